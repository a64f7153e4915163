"""Assembled FP64 operators of the discrete Stokes system (Eq. discrete-stokes).

All matrices are SciPy CSR, built from the bilinear forms with (k+1)^3-point
GLL collocated quadrature on affine hexahedra, J = diag(h/2):

  a(u, v) = sum_e sum_q W_q |J| 2 mu_q eps(u):eps(v)       (viscous stress, A)
  b(v, q) = -sum_e sum_q W_q |J| q(x_q) div v(x_q)          (divergence, B)

Dirichlet velocity DOFs (all nodes on the boundary, Eq. dir-bc) are kept in
storage: their rows and columns are zero, so inputs there are ignored and
outputs there are zero.  Coefficients are given per element quadrature point,
array shape (n_elem, n^3); on the finest mesh they are the nodal values
gathered to the points.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import gll
from .mesh import Mesh


def point_values(mesh: Mesh, nodal: np.ndarray) -> np.ndarray:
    """Gather a nodal scalar field to element points, shape (n_elem, n^3)."""
    return nodal[mesh.point_to_node()]


def incidence(mesh: Mesh) -> sp.csr_matrix:
    """Q: (n_elem n^3) x n_nodes, Q[(e, q), node(e, q)] = 1."""
    p2n = mesh.point_to_node().ravel()
    npts = p2n.size
    return sp.csr_matrix((np.ones(npts), (np.arange(npts), p2n)), shape=(npts, mesh.n_nodes))


def gradient_op(mesh: Mesh, d: int) -> sp.csr_matrix:
    """G_d: nodal scalar -> d/dx_d at every element point, (2/h_d) D along axis d."""
    n, n3, E = mesh.n, mesh.n ** 3, mesh.n_elem
    lq = mesh.local_ijk()
    p2n = mesh.point_to_node()
    rows, cols, vals = [], [], []
    for a in range(n):
        lq2 = lq.copy()
        lq2[:, d] = a
        q2 = lq2[:, 0] + n * (lq2[:, 1] + n * lq2[:, 2])
        rows.append(np.arange(E * n3))
        cols.append(p2n[:, q2].ravel())
        vals.append(np.tile((2.0 / mesh.h[d]) * mesh.D1[lq[:, d], a], E))
    G = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(E * n3, mesh.n_nodes))
    G.sum_duplicates()
    return G


def component_selector(mesh: Mesh, c: int) -> sp.csr_matrix:
    """S_c: component-major velocity vector (3 n_nodes) -> component c (n_nodes)."""
    N = mesh.n_nodes
    return sp.csr_matrix((np.ones(N), (np.arange(N), c * N + np.arange(N))), shape=(N, 3 * N))


def quad_weights(mesh: Mesh) -> np.ndarray:
    """W_q |J| at every element point, flattened (n_elem n^3,)."""
    return np.tile(mesh.W * mesh.detJ, mesh.n_elem)


def dirichlet_mask(mesh: Mesh) -> sp.csr_matrix:
    return sp.diags(mesh.interior_dof_mask().astype(np.float64))


def assemble_A(mesh: Mesh, mu_pts: np.ndarray, mask: bool = True) -> sp.csr_matrix:
    """Viscous stress matrix A from a(u, v) = sum W|J| 2 mu eps(u):eps(v).

    eps_cd(u) = (d_d u_c + d_c u_d) / 2;  A = sum_{c,d} E_cd^T diag(W|J| 2 mu) E_cd.
    """
    G = [gradient_op(mesh, d) for d in range(3)]
    S = [component_selector(mesh, c) for c in range(3)]
    wmu = sp.diags(quad_weights(mesh) * 2.0 * np.asarray(mu_pts).ravel())
    A = None
    for c in range(3):
        for d in range(3):
            Ecd = 0.5 * (G[d] @ S[c] + G[c] @ S[d])
            term = Ecd.T @ wmu @ Ecd
            A = term if A is None else A + term
    if not mask:
        return A.tocsr()
    M = dirichlet_mask(mesh)
    return (M @ A @ M).tocsr()


def pressure_basis(mesh: Mesh) -> sp.csr_matrix:
    """Psi: pressure coefficients (n_elem Np) -> values at element points (n_elem n^3)."""
    psi = gll.pressure_basis_at_points(mesh.k, mesh.ref_pts)  # (n3, Np)
    return sp.block_diag([sp.csr_matrix(psi)] * mesh.n_elem, format="csr")


def assemble_B(mesh: Mesh, mask: bool = True) -> sp.csr_matrix:
    """Divergence matrix B from b(v, q) = -sum W|J| q div v; shape (n_elem Np) x (3 n_nodes)."""
    G = [gradient_op(mesh, d) for d in range(3)]
    S = [component_selector(mesh, c) for c in range(3)]
    div = G[0] @ S[0] + G[1] @ S[1] + G[2] @ S[2]
    B = -(pressure_basis(mesh).T @ sp.diags(quad_weights(mesh)) @ div)
    return (B @ dirichlet_mask(mesh)).tocsr() if mask else B.tocsr()


def boundary_amplification(mesh: Mesh, a: float) -> np.ndarray:
    """Per-element factor of Eq. bdramp: a on elements touching the boundary, else 1."""
    return np.where(mesh.boundary_element_mask(), a, 1.0)


def weight_points(mesh: Mesh, mu_nodes: np.ndarray, weights: str = "sqrt_mu") -> np.ndarray:
    """The w-BFBT weight function at every element point, shape (n_elem, n^3).

    "sqrt_mu": w = sqrt(mu) (Sec. 1.3, Eq. wbfbt).
    "grad":    w = (mu^2 + |grad mu|^2)^(1/4), the viscosity-gradient weights of the remark in
               Sec. 4, with grad mu the gradient of the element's Q_k interpolant of the nodal
               viscosity at the point (discontinuous across elements, so the weight is per
               element point).
    """
    mu_q = point_values(mesh, mu_nodes)
    if weights == "sqrt_mu":
        return np.sqrt(mu_q)
    if weights == "grad":
        g2 = sum((gradient_op(mesh, d) @ mu_nodes) ** 2 for d in range(3)).reshape(mu_q.shape)
        return (mu_q ** 2 + g2) ** 0.25
    if weights == "diag_a":
        # diag(A)-BFBT scales like mu (diag(A) ~ mu); its Poisson surrogate uses the coefficient 1/mu
        return mu_q
    raise ValueError(weights)


def lumped_weight_diag(mesh: Mesh, mu_nodes: np.ndarray, a: float, weights: str = "sqrt_mu") -> np.ndarray:
    """Diagonal of M~_u(w), w = a(e) w(x) (Eq. wbfbt, Eq. bdramp, lumping as Eq. lumping).

    With collocated GLL quadrature the weighted velocity mass matrix is already
    diagonal, so its row sum is sum_{(e,q) -> node} W_q |J| a(e) w_e(x_q), w = sqrt(mu) by default
    (see weight_points).  Returned per node (n_nodes,); the three velocity components share it.
    """
    amp = boundary_amplification(mesh, a)
    vals = (mesh.W * mesh.detJ)[None, :] * amp[:, None] * weight_points(mesh, mu_nodes, weights)
    return incidence(mesh).T @ vals.ravel()


def assemble_Kw(B: sp.csr_matrix, cdiag: np.ndarray, mesh: Mesh) -> sp.csr_matrix:
    """Pressure Poisson matrix K_w = B C_w^-1 B^T (Sec. 6); C_w^-1 zeroed at Dirichlet nodes.
    cdiag per node (n_nodes,), shared by the three components, or per DOF (3 n_nodes,)."""
    bmask = mesh.boundary_node_mask()
    if cdiag.size == 3 * mesh.n_nodes:
        inv = np.where(np.tile(bmask, 3), 0.0, 1.0 / np.where(np.tile(bmask, 3), 1.0, cdiag))
    else:
        inv = np.tile(np.where(bmask, 0.0, 1.0 / cdiag), 3)
    return (B @ sp.diags(inv) @ B.T).tocsr()


def assemble_Lc(mesh: Mesh, c_pts: np.ndarray) -> sp.csr_matrix:
    """Continuous Q_k Poisson matrix L = sum_d G_d^T diag(W|J| c) G_d (Neumann, no masking).

    This is the re-discretisation of -div(c grad) used by the pressure-Poisson
    multigrid (Sec. 6), with c = 1/w per element point.
    """
    G = [gradient_op(mesh, d) for d in range(3)]
    wc = sp.diags(quad_weights(mesh) * np.asarray(c_pts).ravel())
    L = None
    for d in range(3):
        term = G[d].T @ wc @ G[d]
        L = term if L is None else L + term
    return L.tocsr()


def pressure_mass_element(mesh: Mesh) -> np.ndarray:
    """Exact element mass of P_{k-1}: M_d,e = Psi^T diag(W|J|) Psi (Np x Np)."""
    psi = gll.pressure_basis_at_points(mesh.k, mesh.ref_pts)
    return psi.T @ ((mesh.W * mesh.detJ)[:, None] * psi)


def mixed_mass(mesh: Mesh) -> sp.csr_matrix:
    """M_cd: (n_nodes) x (n_elem Np), entries int phi_n psi_m (exact under GLL quadrature)."""
    return (incidence(mesh).T @ sp.diags(quad_weights(mesh)) @ pressure_basis(mesh)).tocsr()


def load_vector(mesh: Mesh, f_nodes: np.ndarray) -> np.ndarray:
    """Right-hand side F_c(node) = sum_{(e,q)->node} W_q |J| f_c(x_node), Dirichlet rows zero.

    f_nodes: (n_nodes, 3).  Returns component-major (3 n_nodes,).
    """
    Qt = incidence(mesh).T
    wq = quad_weights(mesh)
    p2n = mesh.point_to_node().ravel()
    F = np.concatenate([Qt @ (wq * f_nodes[p2n, c]) for c in range(3)])
    return F * mesh.interior_dof_mask()


def constant_pressure(mesh: Mesh) -> np.ndarray:
    """1_psi: coefficient vector of the constant function 1 (Eq. lumping)."""
    v = np.zeros(mesh.n_p)
    v[0::mesh.Np] = 1.0
    return v


def project_pressure(mesh: Mesh, p: np.ndarray) -> np.ndarray:
    """Euclidean projection of p against 1_psi."""
    one = constant_pressure(mesh)
    return p - (one @ p) / (one @ one) * one


# --- element-local evaluation (for sampled outputs at sizes the CSR cannot reach) ---

def element_gradient_mats(mesh: Mesh) -> list[np.ndarray]:
    """Element-local G_d (n^3 x n^3): (2/h_d) D1 along axis d, identity along the others."""
    n = mesh.n
    I = np.eye(n)
    mats = []
    for d in range(3):
        f = [I, I, I]
        f[d] = mesh.D1 * (2.0 / mesh.h[d])
        # local index q = i + n (j + n l): kron order (l, j, i)
        mats.append(np.kron(f[2], np.kron(f[1], f[0])))
    return mats


def element_A(mesh: Mesh, mu_q: np.ndarray) -> np.ndarray:
    """Element stiffness (3 n^3 x 3 n^3), component-major local ordering, no Dirichlet masking."""
    n3 = mesh.n ** 3
    G = element_gradient_mats(mesh)
    Z = np.zeros((n3, n3))
    Sel = [np.hstack([np.eye(n3) if cc == c else Z for cc in range(3)]) for c in range(3)]
    wmu = mesh.W * mesh.detJ * 2.0 * mu_q
    Ae = np.zeros((3 * n3, 3 * n3))
    for c in range(3):
        for d in range(3):
            Ecd = 0.5 * (G[d] @ Sel[c] + G[c] @ Sel[d])
            Ae += Ecd.T @ (wmu[:, None] * Ecd)
    return Ae


def element_B(mesh: Mesh) -> np.ndarray:
    """Element divergence (Np x 3 n^3), no Dirichlet masking."""
    G = element_gradient_mats(mesh)
    psi = gll.pressure_basis_at_points(mesh.k, mesh.ref_pts)
    div = np.hstack(G)
    return -(psi.T @ ((mesh.W * mesh.detJ)[:, None] * div))


def sampled_apply_A(mesh: Mesh, mu_nodes: np.ndarray, u: np.ndarray, nodes: np.ndarray) -> np.ndarray:
    """(A u) at the given global nodes, shape (len(nodes), 3), from element-local matrices.

    Sums the element contributions of the (up to 8) elements around each node;
    Dirichlet inputs are ignored and Dirichlet outputs are zero, as in assemble_A.
    """
    n, N = mesh.n, mesh.n_nodes
    n3 = n ** 3
    bmask = mesh.boundary_node_mask()
    out = np.zeros((len(nodes), 3))
    for r, node in enumerate(np.asarray(nodes)):
        if bmask[node]:
            continue
        g = (node % mesh.NX, (node // mesh.NX) % mesh.NY, node // (mesh.NX * mesh.NY))
        ne = (mesh.nx, mesh.ny, mesh.nz)
        cand = [sorted({min(g[d] // mesh.k, ne[d] - 1), max((g[d] - 1) // mesh.k, 0)}) for d in range(3)]
        for ez in cand[2]:
            for ey in cand[1]:
                for ex in cand[0]:
                    li, lj, ll = g[0] - mesh.k * ex, g[1] - mesh.k * ey, g[2] - mesh.k * ez
                    if not (0 <= li < n and 0 <= lj < n and 0 <= ll < n):
                        continue
                    gi = mesh.k * ex + np.arange(n)
                    gj = mesh.k * ey + np.arange(n)
                    gl = mesh.k * ez + np.arange(n)
                    ids = (gi[None, None, :] + mesh.NX * (gj[None, :, None] + mesh.NY * gl[:, None, None])).ravel()
                    ue = np.concatenate([u[c * N + ids] * (~bmask[ids]) for c in range(3)])
                    ye = element_A(mesh, mu_nodes[ids]) @ ue
                    q = li + n * (lj + n * ll)
                    for c in range(3):
                        out[r, c] += ye[c * n3 + q]
    return out


def nonneg_pressure_basis_at_points(k: int, pts: np.ndarray) -> np.ndarray:
    """phi'_j = prod_d ((1 + xi_d) / 2)^(e_jd) at reference points, same exponents as the solver's
    basis: (n_pts, Np).  Non-negative on the element, so each int_e phi'_j / mu > 0."""
    s = 0.5 * (1.0 + pts)
    return np.stack([s[:, 0] ** a * s[:, 1] ** b * s[:, 2] ** c for a, b, c in gll.pressure_exponents(k)], axis=-1)


def lumped_mass_schur_inverse(mesh: Mesh, mu_nodes: np.ndarray) -> sp.csr_matrix:
    """Inverse of the lumped inverse-viscosity pressure mass (Sec. 1.3, Eq. lumping), block diagonal.

    Steps, per element, in the non-negative basis {phi'_j}:
      M'_e(1/mu) = Phi'^T diag(W_q |J| / mu_q) Phi'       (the pressure mass weighted by 1/mu),
      1'        = coefficients of the constant function 1 in {phi'_j},
      M~'_e     = diag(M'_e(1/mu) 1')                    (Eq. lumping).
    The solver's coefficients p in the centred monomial basis {psi_m} satisfy p = T p' with
    Psi T = Phi' (T found by solving that linear system), so the approximation's inverse in the
    solver's basis is T M~'_e^-1 T^T.  Returned as a sparse (n_p x n_p) matrix.
    """
    psi = gll.pressure_basis_at_points(mesh.k, mesh.ref_pts)          # (n3, Np)
    phi = nonneg_pressure_basis_at_points(mesh.k, mesh.ref_pts)       # (n3, Np)
    T = np.linalg.lstsq(psi, phi, rcond=None)[0]                       # psi @ T = phi
    one = np.linalg.lstsq(phi, np.ones(phi.shape[0]), rcond=None)[0]   # phi @ one = 1
    mu_q = point_values(mesh, mu_nodes)                                # (n_elem, n3)
    blocks = []
    for e in range(mesh.n_elem):
        Me = phi.T @ ((mesh.W * mesh.detJ / mu_q[e])[:, None] * phi)
        d = Me @ one
        blocks.append(T @ np.diag(1.0 / d) @ T.T)
    return sp.csr_matrix(sp.block_diag([sp.csr_matrix(b) for b in blocks], format="csr"))


def diag_mass_schur_inverse(mesh: Mesh, mu_nodes: np.ndarray) -> sp.csr_matrix:
    """Inverse of the diagonal of the inverse-viscosity pressure mass M_p(1/mu) (Sec. 1.3) in the
    solver's centred monomial basis: diag(1 / int_e psi_m^2 / mu) per element, sparse (n_p x n_p)."""
    psi = gll.pressure_basis_at_points(mesh.k, mesh.ref_pts)
    mu_q = point_values(mesh, mu_nodes)
    d = np.stack([np.diag(psi.T @ ((mesh.W * mesh.detJ / mu_q[e])[:, None] * psi)) for e in range(mesh.n_elem)])
    return sp.diags(1.0 / d.ravel()).tocsr()
