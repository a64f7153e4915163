"""Stokes operators on mapped (non-affine) hexahedra, and the solve around them.

TEST INFRASTRUCTURE, NOT PRODUCT CODE (see the package header).

The bilinear forms of Sec. 1.2, a(u, v) = int 2 mu eps(u):eps(v) and b(v, q) = -int q div v, on a
mesh whose elements are images of the reference cube under an isoparametric map: element e maps
xi to x(xi) = sum_a X_a l_a(xi), with X_a the physical coordinates of its (k+1)^3 Q_k nodes
(any node placement; the brick is the special case of evenly spaced, axis-aligned nodes).  The
velocity space is the isoparametric Q_k space, which contains every affine field.  At element point
q (a GLL point):

  J_q[d, r]  = dx_d / dxi_r = sum_a D[.][a] X_d along axis r          (Jacobian)
  du/dx_d    = sum_r (J_q^-1)[r, d] du/dxi_r                           (chain rule)
  weight     = W_q det J_q                                             (quadrature)

The pressure space is P_{k-1}^disc in each element's reference coordinates (the mapped space: the
same monomials psi_m(xi) as on the brick).  The Dirichlet set is the boundary of the structured
node grid, as on the brick.

The solve: FGMRES on the mapped Stokes system, right-preconditioned by the w-BFBT block
preconditioner of the undeformed brick with the same nodal viscosity (Eq. precond-stokes,
Eq. wbfbt): the preconditioner's operators stay those of the brick; only the Krylov operator and
the right-hand side carry the geometry.  A second form takes the preconditioner's finest level
from the mapped mesh (its A, B and lumped weights), for comparison.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import krylov
from . import multigrid as mg
from . import operators as op
from . import wbfbt
from .mesh import Mesh


def reference_gradient_op(mesh: Mesh, r: int) -> sp.csr_matrix:
    """Dhat_r: nodal scalar -> d/dxi_r at every element point (the 1-D GLL derivative D along
    reference axis r, identity along the others); (n_elem n^3) x n_nodes."""
    n, n3, E = mesh.n, mesh.n ** 3, mesh.n_elem
    lq = mesh.local_ijk()
    p2n = mesh.point_to_node()
    rows, cols, vals = [], [], []
    for a in range(n):
        lq2 = lq.copy()
        lq2[:, r] = a
        q2 = lq2[:, 0] + n * (lq2[:, 1] + n * lq2[:, 2])
        rows.append(np.arange(E * n3))
        cols.append(p2n[:, q2].ravel())
        vals.append(np.tile(mesh.D1[lq[:, r], a], E))
    G = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(E * n3, mesh.n_nodes))
    G.sum_duplicates()
    return G


def jacobians(mesh: Mesh, X: np.ndarray) -> np.ndarray:
    """J[(e, q), d, r] = dx_d/dxi_r at every element point; X: nodal coordinates (n_nodes, 3)."""
    X = np.asarray(X, dtype=np.float64)
    Dh = [reference_gradient_op(mesh, r) for r in range(3)]
    J = np.empty((mesh.n_elem * mesh.n ** 3, 3, 3))
    for r in range(3):
        for d in range(3):
            J[:, d, r] = Dh[r] @ X[:, d]
    return J


def geometry(mesh: Mesh, X: np.ndarray):
    """Physical gradient operators G_d (list of 3 CSR) and point weights W_q det J_q."""
    J = jacobians(mesh, X)
    detJ = np.linalg.det(J)
    if np.any(detJ <= 0.0):
        raise ValueError("the element map is not orientation-preserving at some point")
    Jinv = np.linalg.inv(J)                       # Jinv[., r, d] = dxi_r / dx_d
    Dh = [reference_gradient_op(mesh, r) for r in range(3)]
    G = []
    for d in range(3):
        Gd = None
        for r in range(3):
            t = sp.diags(Jinv[:, r, d]) @ Dh[r]
            Gd = t if Gd is None else Gd + t
        G.append(Gd.tocsr())
    wq = np.tile(mesh.W, mesh.n_elem) * detJ
    return G, wq


def assemble_A(mesh: Mesh, X: np.ndarray, mu_pts: np.ndarray, mask: bool = True) -> sp.csr_matrix:
    """A from a(u, v) = sum_q W_q det J_q 2 mu_q eps(u):eps(v) on the mapped mesh."""
    G, wq = geometry(mesh, X)
    S = [op.component_selector(mesh, c) for c in range(3)]
    wmu = sp.diags(wq * 2.0 * np.asarray(mu_pts).ravel())
    A = None
    for c in range(3):
        for d in range(3):
            Ecd = 0.5 * (G[d] @ S[c] + G[c] @ S[d])
            term = Ecd.T @ wmu @ Ecd
            A = term if A is None else A + term
    if not mask:
        return A.tocsr()
    M = op.dirichlet_mask(mesh)
    return (M @ A @ M).tocsr()


def assemble_B(mesh: Mesh, X: np.ndarray, mask: bool = True) -> sp.csr_matrix:
    """B from b(v, q) = -sum_q W_q det J_q q(xi_q) div v(x_q); (n_elem Np) x (3 n_nodes)."""
    G, wq = geometry(mesh, X)
    S = [op.component_selector(mesh, c) for c in range(3)]
    div = G[0] @ S[0] + G[1] @ S[1] + G[2] @ S[2]
    B = -(op.pressure_basis(mesh).T @ sp.diags(wq) @ div)
    return (B @ op.dirichlet_mask(mesh)).tocsr() if mask else B.tocsr()


def load_vector(mesh: Mesh, X: np.ndarray, f_nodes: np.ndarray, mask: bool = True) -> np.ndarray:
    """F_c(node) = sum_{(e,q)->node} W_q det J_q f_c(node); Dirichlet rows zero when mask."""
    _, wq = geometry(mesh, X)
    Qt = op.incidence(mesh).T
    p2n = mesh.point_to_node().ravel()
    F = np.concatenate([Qt @ (wq * f_nodes[p2n, c]) for c in range(3)])
    return F * mesh.interior_dof_mask() if mask else F


class MappedStokes:
    """The mapped Stokes system [A B^T; B 0] with per-node viscosity."""

    def __init__(self, mesh: Mesh, X: np.ndarray, mu_nodes: np.ndarray):
        self.mesh = mesh
        self.A = assemble_A(mesh, X, op.point_values(mesh, np.asarray(mu_nodes, dtype=np.float64)))
        self.B = assemble_B(mesh, X)
        self.BT = self.B.T.tocsr()
        self.nu = mesh.n_u

    def apply_K(self, x: np.ndarray) -> np.ndarray:
        u, p = x[: self.nu], x[self.nu:]
        return np.concatenate([self.A @ u + self.BT @ p, self.B @ u])


def lumped_weight_diag(mesh: Mesh, X: np.ndarray, mu_nodes: np.ndarray, a: float) -> np.ndarray:
    """The sqrt(mu) lumped weight of Eq. wbfbt / Eq. bdramp on the mapped mesh: per node, the sum over
    the element points at it of W_q det J_q a(e) sqrt(mu)."""
    _, wq = geometry(mesh, X)
    w = np.sqrt(op.point_values(mesh, np.asarray(mu_nodes, dtype=np.float64))).ravel()
    amp = np.repeat(op.boundary_amplification(mesh, a), mesh.n ** 3)
    return op.incidence(mesh).T @ (wq * amp * w)


def solve(mesh: Mesh, X: np.ndarray, mu_nodes, f_nodes, opts: wbfbt.Options = wbfbt.Options(), rtol=1e-6,
          maxit=1000, history=None, preconditioner: str = "brick"):
    """FGMRES on the mapped system.  Returns (u, p, iters, rel_res) with p projected against 1_psi.

    preconditioner "brick": the brick's w-BFBT block preconditioner (the GPU path's);
    "mapped_fine" (sqrt(mu) weights only): the same with its finest level taken from the mapped
    mesh: A, B, B^T and the lumped weights C, D in the Schur approximation, and the mapped A
    (its Jacobi diagonal and spectral bound) on the finest level of the viscous V-cycle; the coarser
    levels and the pressure-Poisson hierarchies stay the brick's."""
    sysm = MappedStokes(mesh, X, mu_nodes)
    prob = wbfbt.StokesProblem(mesh, mu_nodes, opts.a_l, opts.a_r, opts.weights)
    if preconditioner == "mapped_fine":
        if opts.weights != "sqrt_mu" or opts.mode != "vcycle" or opts.pmg:
            raise ValueError("mapped_fine takes the sqrt(mu) weights and the fixed-order V-cycles")
        interior = ~mesh.boundary_node_mask()
        prob.A, prob.B, prob.BT = sysm.A, sysm.B, sysm.BT
        prob.Cdiag = lumped_weight_diag(mesh, X, mu_nodes, prob.a_l)
        prob.Ddiag = lumped_weight_diag(mesh, X, mu_nodes, prob.a_r)
        prob.Cinv = np.tile(np.where(interior, 1.0 / prob.Cdiag, 0.0), 3)
        prob.Dinv = np.tile(np.where(interior, 1.0 / prob.Ddiag, 0.0), 3)
    elif preconditioner != "brick":
        raise ValueError(preconditioner)
    pc = wbfbt.BlockPreconditioner(prob, opts.mode, opts.schur_sign, schur=opts.schur,
                                   kinv_cycles=opts.kinv_cycles, pmg=opts.pmg, ainv_cycles=opts.ainv_cycles)
    if preconditioner == "mapped_fine":
        fine = pc.A_levels[0]
        lev = mg.Level(mesh, sysm.A, True, coarsest=fine.coarsest)
        lev.P = fine.P
        pc.A_levels[0] = lev
    F = np.concatenate([load_vector(mesh, X, f_nodes), np.zeros(mesh.n_p)])
    x, its, rel = krylov.fgmres(sysm.apply_K, pc.apply, F, rtol=rtol, restart=opts.restart, maxit=maxit,
                                history=history)
    return x[: mesh.n_u], op.project_pressure(mesh, x[mesh.n_u:]), its, rel
