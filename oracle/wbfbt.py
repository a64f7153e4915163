"""w-BFBT Schur-complement approximation and the Stokes solver around it.

S~^-1 = (B C^-1 B^T)^-1 (B C^-1 A D^-1 B^T) (B D^-1 B^T)^-1          (Eq. wbfbt)
C = M~_u(w_l), D = M~_u(w_r), w_{l,r} = a_{l,r}(e) sqrt(mu)         (Eq. bdramp)
Upper block-triangular right preconditioner [A~ B^T; 0 s S~]^-1     (Eq. precond-stokes)
inside right-preconditioned FGMRES                                   (Sec. 1.3)

Two modes for the inner inverses A~^-1, K_l~^-1, K_r~^-1:
  exact  : sparse LU (the true w-BFBT),
  vcycle : the multigrid of Sec. 6 as restated in `multigrid`.
Pressure vectors are projected Euclidean-orthogonally against 1_psi (the
coefficient vector of the constant function) at S~^-1 entry and exit and
before output; the singular Neumann-type K_w are factored with their first
DOF pinned.  The default s = -1 makes the preconditioner the exact upper
block-LU factor [A B^T; 0 -S] when the blocks are exact (the paper's S is the
negated Schur complement, footnote to Sec. 1.3); s = +1 is the printed block
taken literally.  Both give two iterations with exact blocks (Sec. 1.3).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import krylov
from . import multigrid as mg
from . import operators as op
from . import sinker
from .mesh import Mesh


def default_a_r(mesh: Mesh) -> float:
    """Right boundary amplification following the Table 3 settings: max(1, (N/16) 2^(k-2))."""
    N = max(mesh.nx, mesh.ny, mesh.nz)
    return max(1.0, (N / 16.0) * 2.0 ** (mesh.k - 2))


@dataclass
class Options:
    a_l: float = 1.0
    a_r: float | None = None
    restart: int = 50
    schur_sign: float = -1.0
    mode: str = "vcycle"
    schur: str = "wbfbt"       # "wbfbt" (Eq. wbfbt), "mass" (lumped M_p(1/mu), Eq. lumping),
                               # "mass_diag" (the diagonal of M_p(1/mu))
    weights: str = "sqrt_mu"   # w-BFBT weights: "sqrt_mu" (Eq. wbfbt), "grad" (remark in Sec. 4), or
                               # "diag_a": C = D = diag(A), the diag(A)-BFBT of Sec. 1.3
    kinv_cycles: int = 1       # V-cycles per K~_w^-1 application: x += V(b - K_w x) after the first
    ainv_cycles: int = 1       # V-cycles per A~^-1 application: x += V(b - A x) after the first
    pmg: bool = False          # p-coarsened multigrid (Q_k -> Q1 -> h-levels) for the viscous block


class StokesProblem:
    """Assembled Stokes operators on a brick with per-node viscosity."""

    def __init__(self, mesh: Mesh, mu_nodes: np.ndarray, a_l: float = 1.0, a_r: float | None = None,
                 weights: str = "sqrt_mu"):
        self.mesh = mesh
        self.mu = np.asarray(mu_nodes, dtype=np.float64)
        self.a_l = a_l
        self.a_r = default_a_r(mesh) if a_r is None else a_r
        self.weights = weights
        self.A = op.assemble_A(mesh, op.point_values(mesh, self.mu))
        self.B = op.assemble_B(mesh)
        self.BT = self.B.T.tocsr()
        interior = ~mesh.boundary_node_mask()
        if weights == "diag_a":
            # diag(A)-BFBT (Sec. 1.3): C = D = diag(A), one entry per velocity DOF
            dA = self.A.diagonal()
            free = np.tile(interior, 3)
            self.Cdiag = self.Ddiag = np.where(free, dA, 1.0)
            self.Cinv = self.Dinv = np.where(free, 1.0 / self.Cdiag, 0.0)
        else:
            self.Cdiag = op.lumped_weight_diag(mesh, self.mu, self.a_l, weights)
            self.Ddiag = op.lumped_weight_diag(mesh, self.mu, self.a_r, weights)
            self.Cinv = np.tile(np.where(interior, 1.0 / self.Cdiag, 0.0), 3)
            self.Dinv = np.tile(np.where(interior, 1.0 / self.Ddiag, 0.0), 3)
        self.nu, self.npr = mesh.n_u, mesh.n_p

    def apply_K(self, x: np.ndarray) -> np.ndarray:
        """[A u + B^T p; B u] (Eq. discrete-stokes)."""
        u, p = x[: self.nu], x[self.nu:]
        return np.concatenate([self.A @ u + self.BT @ p, self.B @ u])

    def middle(self, y: np.ndarray) -> np.ndarray:
        """B C^-1 A D^-1 B^T y, the middle factor of Eq. wbfbt."""
        return self.B @ (self.Cinv * (self.A @ (self.Dinv * (self.BT @ y))))


class _PinnedLU:
    """Exact inverse of a singular K_w with null vector 1_psi: pin DOF 0, solve, project."""

    def __init__(self, K: sp.csr_matrix, mesh: Mesh):
        K = K.tolil(copy=True)
        K[0, :] = 0.0
        K[:, 0] = 0.0
        K[0, 0] = 1.0
        self.lu = spla.splu(K.tocsc())
        self.mesh = mesh

    def __call__(self, b):
        bb = b.copy()
        bb[0] = 0.0
        return op.project_pressure(self.mesh, self.lu.solve(bb))


class WBFBT:
    """S~^-1 of Eq. wbfbt with exact or multigrid inner inverses."""

    def __init__(self, prob: StokesProblem, mode: str = "vcycle", kinv_cycles: int = 1):
        self.prob = prob
        m = prob.mesh
        if mode == "exact":
            self.Kl_inv = _PinnedLU(op.assemble_Kw(prob.B, prob.Cdiag, m), m)
            self.Kr_inv = _PinnedLU(op.assemble_Kw(prob.B, prob.Ddiag, m), m)
        elif mode == "vcycle":
            a_l, a_r = (1.0, 1.0) if prob.weights == "diag_a" else (prob.a_l, prob.a_r)
            self.Kl_mg = mg.PressurePoissonMG(m, prob.B, prob.Cdiag, prob.mu, a_l, prob.weights)
            self.Kr_mg = mg.PressurePoissonMG(m, prob.B, prob.Ddiag, prob.mu, a_r, prob.weights)
            self.Kl_inv, self.Kr_inv = self._cycles(self.Kl_mg, kinv_cycles), self._cycles(self.Kr_mg, kinv_cycles)
        else:
            raise ValueError(mode)

    @staticmethod
    def _cycles(pmg, cycles):
        """cycles V-cycles of the two-space multigrid: x = V b, then x += V(b - K_w x)."""
        def apply(b):
            x = pmg.apply(b)
            for _ in range(cycles - 1):
                x = x + pmg.apply(b - pmg.K @ x)
            return x
        return apply

    def apply(self, r: np.ndarray) -> np.ndarray:
        m = self.prob.mesh
        r = op.project_pressure(m, r)
        y = self.Kr_inv(r)
        z = self.prob.middle(y)
        return op.project_pressure(m, self.Kl_inv(z))


class MassSchur:
    """S~^-1 = M~_p(1/mu)^-1, the lumped inverse-viscosity pressure mass of Eq. lumping (the
    Schur approximation w-BFBT is compared against in Sec. 4), with the same projections."""

    def __init__(self, prob: StokesProblem, diag: bool = False):
        self.prob = prob
        if diag:
            self.Sinv = op.diag_mass_schur_inverse(prob.mesh, prob.mu)
        else:
            self.Sinv = op.lumped_mass_schur_inverse(prob.mesh, prob.mu)

    def apply(self, r: np.ndarray) -> np.ndarray:
        m = self.prob.mesh
        return op.project_pressure(m, self.Sinv @ op.project_pressure(m, r))


class BlockPreconditioner:
    """[A~ B^T; 0 s S~]^-1: y_p = s S~^-1 r_p, y_u = A~^-1 (r_u - B^T y_p)."""

    def __init__(self, prob: StokesProblem, mode: str = "vcycle", schur_sign: float = -1.0,
                 schur_inv=None, A_inv=None, schur: str = "wbfbt", kinv_cycles: int = 1, pmg: bool = False,
                 ainv_cycles: int = 1):
        self.prob = prob
        self.sign = schur_sign
        m = prob.mesh
        if A_inv is not None:
            self.A_inv = A_inv
        elif mode == "exact":
            free = np.flatnonzero(m.interior_dof_mask())
            lu = spla.splu(prob.A[free][:, free].tocsc())

            def _ainv(b):
                x = np.zeros_like(b)
                x[free] = lu.solve(b[free])
                return x
            self.A_inv = _ainv
        else:
            self.A_levels = mg.build_hierarchy(m, op.point_values(m, prob.mu), vector=True, pmg=pmg)

            def _vcycles(b):
                # ainv_cycles V-cycles: x = V b, then x += V(b - A x) with the finest level's operator
                x = mg.vcycle(self.A_levels, b)
                for _ in range(ainv_cycles - 1):
                    x = x + mg.vcycle(self.A_levels, b - self.A_levels[0].M @ x)
                return x
            self.A_inv = _vcycles
        if schur_inv is not None:
            self.S_inv = schur_inv
        elif schur in ("mass", "mass_diag"):
            self.S_inv = MassSchur(prob, diag=schur == "mass_diag").apply
        else:
            self.S_inv = WBFBT(prob, mode, kinv_cycles).apply

    def apply(self, v: np.ndarray) -> np.ndarray:
        nu = self.prob.nu
        ru, rp = v[:nu], v[nu:]
        yp = self.sign * self.S_inv(rp)
        yu = self.A_inv(ru - self.prob.BT @ yp)
        return np.concatenate([yu, yp])


def sinker_problem(mesh: Mesh, centres, omega, delta, dr, beta=10.0):
    """Nodal viscosity (n_nodes,) and forcing (n_nodes, 3) of Sec. 2.1."""
    X = mesh.node_coords()
    return sinker.viscosity(X, centres, omega, delta, dr), sinker.forcing(X, centres, omega, delta, beta)


def solve(mesh: Mesh, mu_nodes, f_nodes, opts: Options = Options(), rtol=1e-6, maxit=1000, history=None):
    """FGMRES(restart) solve of the Stokes system; returns (u, p, iters, rel_res, prob)."""
    prob = StokesProblem(mesh, mu_nodes, opts.a_l, opts.a_r, opts.weights)
    pc = BlockPreconditioner(prob, opts.mode, opts.schur_sign, schur=opts.schur, kinv_cycles=opts.kinv_cycles,
                             ainv_cycles=opts.ainv_cycles,
                             pmg=opts.pmg)
    F = np.concatenate([op.load_vector(mesh, f_nodes), np.zeros(mesh.n_p)])
    x, its, rel = krylov.fgmres(prob.apply_K, pc.apply, F, rtol=rtol, restart=opts.restart,
                                maxit=maxit, history=history)
    u = x[: mesh.n_u]
    p = op.project_pressure(mesh, x[mesh.n_u:])
    return u, p, its, rel, prob
