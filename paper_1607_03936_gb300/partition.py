"""Element slabs for a partitioned operator apply over several ranks (one GPU each).

The structured brick is cut along z into slabs of whole element layers, one per rank.  Rank r
owns elements ez in [z0, z1) and the node planes iz in [k z0, k z1) (the last rank also the top
plane k nz); pressure is element-local, so it owns the coefficients of its elements.  Its local
problem is the sub-mesh of elements [e0, e1) = [max(0, z0 - 2), min(nz, z1 + 2)): two ghost
element layers on each interior side.  The library treats every face of a mesh as Dirichlet, so
the sub-mesh's outer ghost planes read and write zero; two layers keep them away from every
element that touches an owned node, and the apply on the sub-mesh is then exact on all owned
nodes and elements without any change to the element kernels.

One apply is: a halo exchange (the neighbour's owned node planes and pressure layers that are this
rank's ghosts, copied into the local vector), the local apply, and the owned part of the result.
Dot products sum over owned entries and reduce over ranks.  The exchange uses torch.distributed
point-to-point messages of contiguous plane blocks (node index ix + NX (iy + NY iz): a z-plane is
contiguous), so it runs on NCCL with device tensors and on gloo with host tensors.

A partitioned solve (SlabOperator, fgmres): the Krylov vectors hold owned entries only; every
operator apply scatters them into the sub-mesh vectors, exchanges the halo and applies locally;
the Arnoldi step orthogonalises by classical Gram-Schmidt applied twice, each pass one batched
all-reduce of the local V^T w, and norms reduce the same way.  With an identical preconditioner
on every rank count (the identity, or any owned-entry-wise map) the iterates equal the one-rank
iterates up to the reduction order.

This module holds the index bookkeeping, the exchange and the distributed Krylov loop (vector
algebra in torch on the ranks' own tensors); the local applies are the library's (wbfbt.Solver
on the sub-mesh) or, in CPU tests, any callable with the same signature.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch


@dataclass
class SlabPartition:
    nx: int
    ny: int
    nz: int
    k: int
    world: int
    rank: int

    def __post_init__(self):
        if self.nz < 2 * self.world:
            raise ValueError("each rank needs at least two element layers")
        base, extra = divmod(self.nz, self.world)
        bounds = [0]
        for r in range(self.world):
            bounds.append(bounds[-1] + base + (1 if r < extra else 0))
        self.bounds = bounds
        self.z0, self.z1 = bounds[self.rank], bounds[self.rank + 1]
        self.e0, self.e1 = max(0, self.z0 - 2), min(self.nz, self.z1 + 2)
        self.NX, self.NY = self.k * self.nx + 1, self.k * self.ny + 1
        self.plane = self.NX * self.NY                      # nodes per z-plane
        self.np_layer = self.nx * self.ny                   # elements per layer

    # ---------------------------------------------------------------- sizes
    @property
    def ext_nz(self) -> int:
        """Element layers of the local (extended) sub-mesh."""
        return self.e1 - self.e0

    @property
    def ext_planes(self) -> int:
        return self.k * self.ext_nz + 1

    def owned_planes(self, r: int | None = None) -> tuple[int, int]:
        """Global node planes [lo, hi) owned by rank r (default: this rank)."""
        r = self.rank if r is None else r
        lo, hi = self.k * self.bounds[r], self.k * self.bounds[r + 1]
        if r == self.world - 1:
            hi += 1
        return lo, hi

    def owned_local_planes(self) -> tuple[int, int]:
        lo, hi = self.owned_planes()
        return lo - self.k * self.e0, hi - self.k * self.e0

    # ---------------------------------------------------------------- vectors
    def local_from_global(self, g: torch.Tensor, ncomp: int) -> torch.Tensor:
        """The sub-mesh part of a global nodal vector [ncomp][NZ][NY][NX] (flat)."""
        NZ = self.k * self.nz + 1
        v = g.reshape(ncomp, NZ, self.plane)
        return v[:, self.k * self.e0: self.k * self.e1 + 1].contiguous().reshape(-1)

    def local_pressure_from_global(self, p: torch.Tensor, npe: int) -> torch.Tensor:
        v = p.reshape(self.nz, self.np_layer * npe)
        return v[self.e0: self.e1].contiguous().reshape(-1)

    def owned_nodes(self, loc: torch.Tensor, ncomp: int) -> torch.Tensor:
        """The owned node planes of a local nodal vector: [ncomp][owned planes][NY][NX]."""
        lo, hi = self.owned_local_planes()
        return loc.reshape(ncomp, self.ext_planes, self.plane)[:, lo:hi]

    def owned_elements(self, loc_p: torch.Tensor, npe: int) -> torch.Tensor:
        v = loc_p.reshape(self.ext_nz, self.np_layer * npe)
        return v[self.z0 - self.e0: self.z1 - self.e0]

    # ---------------------------------------------------------------- exchange
    def halo_exchange(self, loc: torch.Tensor, ncomp: int, loc_p: torch.Tensor | None = None, npe: int = 0):
        """Fill this rank's ghost node planes (and ghost pressure layers) from the neighbours' owned
        data, in place.  Every rank calls it; messages go to r - 1 and r + 1."""
        import torch.distributed as dist

        v = loc.reshape(ncomp, self.ext_planes, self.plane)
        k, e0 = self.k, self.e0
        reqs = []
        recv = []
        for nb in (self.rank - 1, self.rank + 1):
            if nb < 0 or nb >= self.world:
                continue
            # what nb needs from me: my owned planes inside nb's sub-mesh
            nb_e0 = max(0, self.bounds[nb] - 2)
            nb_e1 = min(self.nz, self.bounds[nb + 1] + 2)
            lo, hi = self.owned_planes()
            s_lo, s_hi = max(lo, k * nb_e0), min(hi, k * nb_e1 + 1)
            send = v[:, s_lo - k * e0: s_hi - k * e0].contiguous()
            reqs.append(dist.isend(send, nb))
            # what I need from nb: nb's owned planes inside my sub-mesh
            nlo, nhi = self.owned_planes(nb)
            r_lo, r_hi = max(nlo, k * e0), min(nhi, k * self.e1 + 1)
            buf = torch.empty((ncomp, r_hi - r_lo, self.plane), dtype=loc.dtype, device=loc.device)
            reqs.append(dist.irecv(buf, nb))
            recv.append((buf, r_lo - k * e0, r_hi - k * e0))
            if loc_p is not None:
                pv = loc_p.reshape(self.ext_nz, self.np_layer * npe)
                sl, sh = max(self.z0, nb_e0), min(self.z1, nb_e1)
                reqs.append(dist.isend(pv[sl - e0: sh - e0].contiguous(), nb))
                rl, rh = max(self.bounds[nb], e0), min(self.bounds[nb + 1], self.e1)
                pbuf = torch.empty((rh - rl, self.np_layer * npe), dtype=loc_p.dtype, device=loc_p.device)
                reqs.append(dist.irecv(pbuf, nb))
                recv.append((pbuf, rl - e0, rh - e0, "p"))
        for q in reqs:
            q.wait()
        for item in recv:
            if len(item) == 4:
                buf, a, b, _ = item
                loc_p.reshape(self.ext_nz, -1)[a:b] = buf
            else:
                buf, a, b = item
                v[:, a:b] = buf

    def dot(self, a: torch.Tensor, b: torch.Tensor, ncomp: int) -> torch.Tensor:
        """Sum over owned nodes of a * b, reduced over all ranks (FP64)."""
        import torch.distributed as dist

        s = (self.owned_nodes(a, ncomp).double() * self.owned_nodes(b, ncomp).double()).sum().reshape(1)
        if self.world > 1:
            dist.all_reduce(s)
        return s[0]


def partitioned_apply(part: SlabPartition, u_loc: torch.Tensor, p_loc: torch.Tensor | None, local_apply,
                      npe: int = 0):
    """One partitioned operator apply: halo exchange, the local apply on the sub-mesh, and the owned
    part of the result.  u_loc [3][ext planes][NY][NX] flat (ghost planes overwritten), p_loc the
    sub-mesh pressure or None; local_apply(u_loc, p_loc) -> (yu_loc, yp_loc or None).  Returns the
    owned node planes of yu and the owned element layers of yp."""
    part.halo_exchange(u_loc, 3, p_loc, npe)
    yu, yp = local_apply(u_loc, p_loc)
    return part.owned_nodes(yu, 3), (part.owned_elements(yp, npe) if yp is not None else None)


def library_local_apply(part: SlabPartition, mu_loc: torch.Tensor, lengths, X_loc: torch.Tensor | None = None,
                        **opts):
    """local_apply backed by the CUDA library: a wbfbt.Solver on this rank's sub-mesh (its own GPU),
    applying K = [A B^T; B 0] in FP64.  mu_loc: the sub-mesh's nodal viscosity (device).  X_loc: on
    a mapped mesh, the sub-mesh's node coordinates [3][nodes] (the global coordinates' local planes,
    as for a velocity); the ghost-layer argument is unchanged, since the mapped operators keep the
    node grid's boundary as their Dirichlet set."""
    from . import wbfbt as wb

    h = (lengths[0] / part.nx, lengths[1] / part.ny, lengths[2] / part.nz)
    s = wb.Solver(part.nx, part.k, mu_loc, ny=part.ny, nz=part.ext_nz,
                  lengths=(lengths[0], lengths[1], h[2] * part.ext_nz), **opts)
    if X_loc is not None:
        s.set_geometry(X_loc)

    def apply(u_loc, p_loc):
        y = s.apply_K(torch.cat([u_loc, p_loc]))
        return y[: s.n_u], y[s.n_u:]

    apply.solver = s
    return apply


class SlabOperator:
    """K = [A B^T; B 0] on the owned entries of a slab partition.  An owned vector is the owned
    velocity node planes [3][owned planes][NY][NX] followed by the owned pressure layers
    [owned layers][nx ny][npe], flattened; local_apply(u_loc, p_loc) -> (yu_loc, yp_loc) applies
    the sub-mesh operator."""

    def __init__(self, part: SlabPartition, local_apply, npe: int, dtype=torch.float64, device="cpu"):
        self.part, self.local_apply, self.npe = part, local_apply, npe
        self.dtype, self.device = dtype, device
        lo, hi = part.owned_local_planes()
        self.n_u = 3 * (hi - lo) * part.plane
        self.n_p = (part.z1 - part.z0) * part.np_layer * npe
        self.n = self.n_u + self.n_p

    def apply(self, x: torch.Tensor) -> torch.Tensor:
        part = self.part
        lo, hi = part.owned_local_planes()
        u_loc = torch.zeros((3, part.ext_planes, part.plane), dtype=self.dtype, device=self.device)
        p_loc = torch.zeros((part.ext_nz, part.np_layer * self.npe), dtype=self.dtype, device=self.device)
        u_loc[:, lo:hi] = x[: self.n_u].reshape(3, hi - lo, part.plane)
        p_loc[part.z0 - part.e0: part.z1 - part.e0] = x[self.n_u:].reshape(part.z1 - part.z0, -1)
        yu, yp = partitioned_apply(part, u_loc.reshape(-1), p_loc.reshape(-1), self.local_apply, self.npe)
        return torch.cat([yu.reshape(-1), yp.reshape(-1)])

    def allreduce(self, t: torch.Tensor) -> torch.Tensor:
        import torch.distributed as dist

        if self.part.world > 1:
            dist.all_reduce(t)
        return t

    def norm(self, v: torch.Tensor) -> float:
        return float(torch.sqrt(self.allreduce((v * v).sum().reshape(1)))[0])


def fgmres(op: SlabOperator, b: torch.Tensor, precond=None, restart: int = 50, maxit: int = 1000,
           rtol: float = 1e-6):
    """Right-preconditioned FGMRES(restart) on a SlabOperator, every rank calling it with its owned
    part of b.  precond(v) -> z on owned vectors (identity when None).  Orthogonalisation: classical
    Gram-Schmidt twice (one batched all-reduce per pass), Givens rotations; at a restart the
    residual is recomputed as b - K x.  Returns (x, iterations, relative true residual)."""
    x = torch.zeros_like(b)
    r = b.clone()
    beta0 = op.norm(r)
    if beta0 == 0.0:
        return x, 0, 0.0
    its = 0
    while True:
        beta = op.norm(r)
        m = restart
        V = torch.zeros((m + 1, b.numel()), dtype=b.dtype, device=b.device)
        Z = torch.zeros((m, b.numel()), dtype=b.dtype, device=b.device)
        H = torch.zeros((m + 1, m), dtype=torch.float64)
        cs, sn = torch.zeros(m, dtype=torch.float64), torch.zeros(m, dtype=torch.float64)
        g = torch.zeros(m + 1, dtype=torch.float64)
        g[0] = beta
        V[0] = r / beta
        j_done, converged = 0, False
        for j in range(m):
            Z[j] = V[j] if precond is None else precond(V[j])
            w = op.apply(Z[j])
            for _ in range(2):
                h = op.allreduce(V[: j + 1] @ w)
                w = w - h @ V[: j + 1]
                H[: j + 1, j] += h.cpu().double()
            H[j + 1, j] = op.norm(w)
            if H[j + 1, j] > 0:
                V[j + 1] = w / H[j + 1, j].item()
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = torch.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            j_done = j + 1
            if abs(float(g[j + 1])) <= rtol * beta0 or its >= maxit:
                converged = abs(float(g[j + 1])) <= rtol * beta0
                break
        y = torch.linalg.solve_triangular(H[:j_done, :j_done], g[:j_done].reshape(-1, 1), upper=True).reshape(-1)
        x = x + y.to(b.dtype).to(b.device) @ Z[:j_done]
        r = b - op.apply(x)
        if converged or its >= maxit:
            return x, its, op.norm(r) / beta0

