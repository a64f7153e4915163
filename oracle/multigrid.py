"""Geometric multigrid pieces of Sec. 6, restated for fixed-order Q_k h-coarsening.

The paper's HMG (p-, then h-, then algebraic coarsening, then a direct solve)
becomes, in this restatement: Q_k levels N, N/2, ... (coarsen while every
element count is even and the smallest exceeds 4), re-discretised operators
with the coefficient coarsened as the normalised L^2-adjoint of element-wise
multilinear interpolation (Sec. 6; see coarsen_coefficient), nested Q_k interpolation P and restriction P^T,
Chebyshev(3)-accelerated point-Jacobi pre- and post-smoothing (Sec. 6), and a
dense Cholesky solve on the coarsest level (the paper notes a direct solve is
reasonable at 64 elements).  Chebyshev bounds are [0.1, 1.1] x lambda_hat,
lambda_hat from 10 power iterations on D^-1 M from a counter-based SplitMix64
start vector.

The pressure-Poisson V-cycle (Sec. 6, Fig. 5) smooths K_w on the
discontinuous modal space, moves the residual to continuous Q_k with
r_c = M_cd M_d^-1 r_d, runs a Q_k Poisson V-cycle for -div((1/w) grad) with
Neumann conditions, and returns e_d = M_d^-1 M_dc e_c before post-smoothing.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import gll
from . import operators as op
from .mesh import Mesh

POWER_ITERS = 10
CHEB_LO, CHEB_HI = 0.1, 1.1
START_SEED = 0x5EED


# ---------------------------------------------------------------- start vector

def splitmix64_uniform(seed: int, count: int) -> np.ndarray:
    """u_i in [-0.5, 0.5): the (i+1)-th SplitMix64 output of state `seed`, top 53 bits.

    SplitMix64 (Steele, Lea & Flood 2014): s_i = seed + (i+1) * 0x9E3779B97F4A7C15,
    z = (s ^ (s >> 30)) * 0xBF58476D1CE4E5B9, z = (z ^ (z >> 27)) * 0x94D049BB133111EB,
    out = z ^ (z >> 31), all mod 2^64.
    """
    i = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        s = np.uint64(seed) + i * np.uint64(0x9E3779B97F4A7C15)
        z = (s ^ (s >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 2.0 ** 53) - 0.5


def power_lambda(M: sp.spmatrix, dinv: np.ndarray, start: np.ndarray, iters: int = POWER_ITERS) -> float:
    """lambda_hat of D^-1 M: v <- D^-1 M v / ||.||, returning the last norm."""
    v = start / np.linalg.norm(start)
    lam = 0.0
    for _ in range(iters):
        w = dinv * (M @ v)
        lam = np.linalg.norm(w)
        v = w / lam
    return lam


# ------------------------------------------------------------------ smoother

def chebyshev(M, dinv, b, x0, lam_hat, steps=3, want_residual=False):
    """Chebyshev-accelerated point Jacobi on D^-1 M over [0.1, 1.1] lambda_hat.

    The three-term Chebyshev iteration (Saad, Iterative Methods, Alg. 12.1)
    with the diagonal preconditioner.  x0=None means a zero initial guess,
    which saves the first operator apply.  Returns (x, r) where r is the
    recurrence residual after the last step when want_residual, else None.
    """
    lmin, lmax = CHEB_LO * lam_hat, CHEB_HI * lam_hat
    theta, delta = 0.5 * (lmax + lmin), 0.5 * (lmax - lmin)
    sigma = theta / delta
    rho = 1.0 / sigma
    if x0 is None:
        x = np.zeros_like(b)
        r = b.copy()
    else:
        x = x0.copy()
        r = b - M @ x
    d = dinv * r / theta
    for s in range(steps):
        x = x + d
        if s == steps - 1 and not want_residual:
            return x, None
        r = r - M @ d
        if s == steps - 1:
            return x, r
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * (dinv * r)
        rho = rho_new
    return x, r


# ------------------------------------------------------------------ transfers

def prolongation_1d(nc: int, k: int) -> sp.csr_matrix:
    """Nested Q_k interpolation along one axis: (k 2nc + 1) x (k nc + 1).

    A fine node of fine element ef (child s = ef mod 2 of coarse element
    ef // 2) at reference point xi_a maps to coarse reference point
    (xi_a + 2 s - 1) / 2 and takes sum_b l_b(that point) u_c(k (ef // 2) + b).
    """
    xi, _ = gll.gll_nodes_weights(k)
    nf = 2 * nc
    rows, cols, vals = [], [], []
    for i_f in range(k * nf + 1):
        ef = min(i_f // k, nf - 1)
        a = i_f - k * ef
        ec, s = ef // 2, ef % 2
        t = (xi[a] + 2 * s - 1) / 2.0
        lv = gll.lagrange_eval(xi, np.array([t]))[0]
        for b in range(k + 1):
            rows.append(i_f)
            cols.append(k * ec + b)
            vals.append(lv[b])
    return sp.csr_matrix((vals, (rows, cols)), shape=(k * nf + 1, k * nc + 1))


def prolongation_scalar(mc: Mesh) -> sp.csr_matrix:
    """Q_k interpolation from mesh mc to its uniform refinement, P = Pz (x) Py (x) Px."""
    Px = prolongation_1d(mc.nx, mc.k)
    Py = prolongation_1d(mc.ny, mc.k)
    Pz = prolongation_1d(mc.nz, mc.k)
    return sp.kron(Pz, sp.kron(Py, Px)).tocsr()


def prolongation_vector(mc: Mesh) -> sp.csr_matrix:
    P = prolongation_scalar(mc)
    return sp.block_diag([P, P, P], format="csr")


def hat_eval(x: np.ndarray, t: np.ndarray) -> np.ndarray:
    """H[s, i] = hat_i(t_s): piecewise-linear interpolation weights on the node set x."""
    t = np.asarray(t, dtype=np.float64)
    H = np.zeros((t.size, x.size))
    for s, ts in enumerate(t):
        j = min(max(np.searchsorted(x, ts, side="right") - 1, 0), x.size - 2)
        th = (ts - x[j]) / (x[j + 1] - x[j])
        H[s, j] = 1.0 - th
        H[s, j + 1] = th
    return H


def coarsen_coefficient(mf: Mesh, c_fine: np.ndarray) -> np.ndarray:
    """Coefficient coarsening: L^2-adjoint of element-wise multilinear interpolation (Sec. 6).

    c_E(x_q) = sum_{e,q'} W_q' |J_e| phi~_q(x_q') c_e(x_q') / sum_{e,q'} W_q' |J_e| phi~_q(x_q'),
    summed over the 8 children e of coarse element E, where phi~_q is the
    tensor-product piecewise-linear hat of coarse GLL point q.  For k = 1 this
    is exactly the adjoint of trilinear interpolation used by the paper's
    h-coarsening; for k >= 2 the Q_k Lagrange basis would give the adjoint
    negative weights (and negative coarse viscosities at high contrast), the
    hat basis keeps every weight non-negative, and the normalisation keeps
    constants.  c_fine: (n_elem_f, n^3).  Returns (n_elem_c, n^3).
    """
    mc = mf.coarsen()
    n = mf.n
    xi, w = mf.xi, mf.w1
    # One axis of the formula: T[s][i, i'] = w_i' hat_i(t_{s,i'}) / sum_{s'', i''} w_i'' hat_i(t_{s'',i''}),
    # t_{s,i'} = (xi_i' + 2s - 1)/2 the coarse reference coordinate of child s's point i'.
    raw = [(hat_eval(xi, (xi + 2 * s - 1) / 2.0) * w[:, None]).T for s in range(2)]
    den = raw[0].sum(axis=1) + raw[1].sum(axis=1)
    T = [r / den[:, None] for r in raw]
    cf = c_fine.reshape(mf.nz, mf.ny, mf.nx, n, n, n)  # (ez, ey, ex, l', j', i')
    out = np.zeros((mc.nz, mc.ny, mc.nx, n, n, n))
    for sz in range(2):
        for sy in range(2):
            for sx in range(2):
                child = cf[sz::2, sy::2, sx::2]
                out += np.einsum("lL,jJ,iI,zyxLJI->zyxlji", T[sz], T[sy], T[sx], child)
    return out.reshape(mc.n_elem, n ** 3)


# ------------------------------------------------------------------ p-coarsening (Q_k -> Q1)

def p_prolongation_1d(n_el: int, k: int) -> sp.csr_matrix:
    """Trilinear (Q1) functions on a line of n_el elements evaluated at the Q_k GLL nodes of the
    same elements: (k n_el + 1) x (n_el + 1).  Node i of element e (i = k e + a) sits at reference
    point xi_a, where the two Q1 vertex functions are (1 - xi_a)/2 and (1 + xi_a)/2."""
    xi, _ = gll.gll_nodes_weights(k)
    rows, cols, vals = [], [], []
    for i in range(k * n_el + 1):
        e = min(i // k, n_el - 1)
        a = i - k * e
        for v, val in ((e, 0.5 * (1.0 - xi[a])), (e + 1, 0.5 * (1.0 + xi[a]))):
            if val != 0.0:
                rows.append(i)
                cols.append(v)
                vals.append(val)
    return sp.csr_matrix((vals, (rows, cols)), shape=(k * n_el + 1, n_el + 1))


def p_prolongation_vector(mf: Mesh) -> sp.csr_matrix:
    """Q1 -> Q_k on the same mesh, three components: the embedding of trilinear functions."""
    P = sp.kron(p_prolongation_1d(mf.nz, mf.k), sp.kron(p_prolongation_1d(mf.ny, mf.k),
                                                          p_prolongation_1d(mf.nx, mf.k))).tocsr()
    return sp.block_diag([P, P, P], format="csr")


def p_coarsen_coefficient(mf: Mesh, c_fine: np.ndarray) -> np.ndarray:
    """Coefficient at the Q1 points (vertices) of each element from its Q_k point values: the
    normalised L^2-adjoint of element-wise trilinear interpolation (the h-coarsening rule of Sec. 6
    applied within the element), c1(v) = sum_q W_q phi_v(x_q) c(x_q) / sum_q W_q phi_v(x_q) with
    phi_v the trilinear vertex functions and W_q the Q_k GLL weights.  Returns (n_elem, 8)."""
    xi, w = mf.xi, mf.w1
    lin = np.stack([0.5 * (1.0 - xi), 0.5 * (1.0 + xi)])          # (2, n): phi_v at the GLL points
    T = lin * w[None, :]
    T = T / T.sum(axis=1, keepdims=True)
    n = mf.n
    cf = c_fine.reshape(mf.n_elem, n, n, n)                          # (e, l, j, i)
    out = np.einsum("vc,ub,ta,ecba->evut", T, T, T, cf)              # (e, v_z, v_y, v_x)
    return out.reshape(mf.n_elem, 8)


# ------------------------------------------------------------------ levels

def n_levels(m: Mesh) -> int:
    """Number of levels: coarsen while all element counts are even and the smallest exceeds 4."""
    L = 1
    nx, ny, nz = m.nx, m.ny, m.nz
    while nx % 2 == 0 and ny % 2 == 0 and nz % 2 == 0 and min(nx, ny, nz) > 4:
        nx, ny, nz = nx // 2, ny // 2, nz // 2
        L += 1
    return L


class Level:
    """One multigrid level: operator, Jacobi diagonal, lambda_hat, transfer to the next coarser."""

    def __init__(self, mesh, M, vector: bool, coarsest: bool):
        self.mesh, self.M, self.vector, self.coarsest = mesh, M, vector, coarsest
        diag = M.diagonal()
        self.dinv = np.where(diag != 0.0, 1.0 / np.where(diag != 0.0, diag, 1.0), 0.0)
        self.P = None
        if coarsest:
            self._factor()
        else:
            start = splitmix64_uniform(START_SEED, M.shape[0])
            if vector:
                start = start * mesh.interior_dof_mask()
            self.lam = power_lambda(M, self.dinv, start)

    def _factor(self):
        Md = self.M.toarray()
        if self.vector:
            self.free = np.flatnonzero(self.mesh.interior_dof_mask())
            self.chol = sla.cho_factor(Md[np.ix_(self.free, self.free)], lower=True)
        else:
            Md = Md.copy()
            Md[0, :] = 0.0
            Md[:, 0] = 0.0
            Md[0, 0] = 1.0
            self.chol = sla.cho_factor(Md, lower=True)

    def coarse_solve(self, b):
        if self.vector:
            x = np.zeros_like(b)
            x[self.free] = sla.cho_solve(self.chol, b[self.free])
            return x
        bb = b.copy()
        bb[0] = 0.0
        x = sla.cho_solve(self.chol, bb)
        return x - x.mean()


def build_hierarchy(mesh: Mesh, coef_pts: np.ndarray, vector: bool, pmg: bool = False) -> list[Level]:
    """Levels for A (vector, Dirichlet; coef = mu) or L_c (scalar, Neumann; coef = 1/w).

    pmg (vector, k > 1): the p-coarsened hierarchy of Sec. 6 / Fig. 5 -- the Q_k fine level, then
    trilinear Q1 on the same mesh (coefficient by p_coarsen_coefficient, transfer by the Q1 -> Q_k
    embedding), then Q1 h-levels as below."""
    levels = []
    m, c = mesh, coef_pts
    if pmg and vector and mesh.k > 1:
        M = op.assemble_A(m, c)
        lev = Level(m, M, vector, coarsest=False)
        levels.append(lev)
        lev.P = p_prolongation_vector(m)
        c = p_coarsen_coefficient(m, c)
        m = Mesh(m.nx, m.ny, m.nz, 1, m.lx, m.ly, m.lz)
    L = n_levels(m)
    for l in range(L):
        M = op.assemble_A(m, c) if vector else op.assemble_Lc(m, c)
        lev = Level(m, M, vector, coarsest=(l == L - 1))
        levels.append(lev)
        if l < L - 1:
            mc = m.coarsen()
            lev.P = prolongation_vector(mc) if vector else prolongation_scalar(mc)
            c = coarsen_coefficient(m, c)
            m = mc
    return levels


def vcycle(levels: list[Level], b: np.ndarray, l: int = 0) -> np.ndarray:
    """One V-cycle from a zero guess: Chebyshev(3) pre, coarse correction, Chebyshev(3) post."""
    lev = levels[l]
    if lev.coarsest:
        return lev.coarse_solve(b)
    x, r = chebyshev(lev.M, lev.dinv, b, None, lev.lam, want_residual=True)
    e = vcycle(levels, lev.P.T @ r, l + 1)
    x = x + lev.P @ e
    x, _ = chebyshev(lev.M, lev.dinv, b, x, lev.lam)
    return x


class PressurePoissonMG:
    """Approximate inverse of K_w = B C_w^-1 B^T by the two-space V-cycle of Sec. 6."""

    def __init__(self, mesh: Mesh, B, cdiag: np.ndarray, mu_nodes: np.ndarray, a: float, weights: str = "sqrt_mu"):
        self.mesh = mesh
        self.K = op.assemble_Kw(B, cdiag, mesh)
        diag = self.K.diagonal()
        # a zero diagonal (the constant mode of a mesh whose only element has all faces on the
        # Dirichlet boundary) is skipped by the smoother, as Dirichlet rows are
        self.dinv = np.where(diag > 0.0, 1.0 / np.where(diag > 0.0, diag, 1.0), 0.0)
        self.lam = power_lambda(self.K, self.dinv, splitmix64_uniform(START_SEED, self.K.shape[0]))
        amp = op.boundary_amplification(mesh, a)
        c_pts = 1.0 / (amp[:, None] * op.weight_points(mesh, mu_nodes, weights))
        self.levels = build_hierarchy(mesh, c_pts, vector=False)
        Md = op.pressure_mass_element(mesh)
        self.Md_inv = np.linalg.inv(Md)
        self.Mcd = op.mixed_mass(mesh)

    def disc_to_cont(self, r_d):
        """r_c = M_cd M_d^-1 r_d."""
        Np = self.mesh.Np
        v = (r_d.reshape(-1, Np) @ self.Md_inv.T).ravel()
        return self.Mcd @ v

    def cont_to_disc(self, e_c):
        """e_d = M_d^-1 M_dc e_c (L^2 projection onto P_{k-1}^disc)."""
        Np = self.mesh.Np
        v = (self.Mcd.T @ e_c).reshape(-1, Np)
        return (v @ self.Md_inv.T).ravel()

    def apply(self, b_d):
        x, r = chebyshev(self.K, self.dinv, b_d, None, self.lam, want_residual=True)
        e_c = vcycle(self.levels, self.disc_to_cont(r))
        x = x + self.cont_to_disc(e_c)
        x, _ = chebyshev(self.K, self.dinv, b_d, x, self.lam)
        return x
