"""Pins for the oracle's assembled operators against symbolic integrals and invariants.

Each exactness pin picks fields whose integrand has per-variable degree <= 2k-1,
which (k+1)-point GLL quadrature integrates exactly, so the assembled bilinear
form must equal the sympy integral of the continuous form (Sec. 1.2 operators).
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla
import sympy as sy

from oracle import gll
from oracle import mesh as M
from oracle import operators as op

X, Y, Z = sy.symbols("x y z")
XYZ = (X, Y, Z)


def _integrate(expr, L):
    return float(sy.integrate(expr, (X, 0, L[0]), (Y, 0, L[1]), (Z, 0, L[2])))


def _nodal(mesh, exprs):
    f = sy.lambdify(XYZ, exprs, "numpy")
    P = mesh.node_coords()
    vals = f(P[:, 0], P[:, 1], P[:, 2])
    return [np.broadcast_to(np.asarray(v, dtype=float), (mesh.n_nodes,)) for v in vals]


def _eps(u):
    return [[(sy.diff(u[c], XYZ[d]) + sy.diff(u[d], XYZ[c])) / 2 for d in range(3)] for c in range(3)]


def _a_form(mu, u, v):
    eu, ev = _eps(u), _eps(v)
    return 2 * mu * sum(eu[c][d] * ev[c][d] for c in range(3) for d in range(3))


def test_A_unmasked_matches_symbolic_form_multilinear():
    L = (1.0, 0.7, 1.3)
    m = M.Mesh(2, 3, 2, 2, *L)
    rng = np.random.default_rng(0)
    mono = [1, X, Y, Z, X * Y, Y * Z, X * Z, X * Y * Z]
    u = [sum(float(c) * t for c, t in zip(rng.standard_normal(8), mono)) for _ in range(3)]
    v = [sum(float(c) * t for c, t in zip(rng.standard_normal(8), mono)) for _ in range(3)]
    mu = 1 + X + 2 * Y
    A = op.assemble_A(m, op.point_values(m, _nodal(m, [mu])[0]), mask=False)
    uv, vv = np.concatenate(_nodal(m, u)), np.concatenate(_nodal(m, v))
    assert abs(vv @ A @ uv - _integrate(_a_form(mu, u, v), L)) < 1e-11 * max(1, abs(vv @ A @ uv))


def test_A_masked_matches_symbolic_form_bubble_k3():
    L = (1.0, 1.0, 1.0)
    m = M.Mesh(2, 2, 2, 3)
    b = X * (1 - X) * Y * (1 - Y) * Z * (1 - Z)
    u = [2 * b, -b, 3 * b]
    v = [b, 4 * b, -2 * b]
    mu = 2 + X
    A = op.assemble_A(m, op.point_values(m, _nodal(m, [mu])[0]))
    uv, vv = np.concatenate(_nodal(m, u)), np.concatenate(_nodal(m, v))
    ref = _integrate(_a_form(mu, u, v), L)
    assert abs(vv @ A @ uv - ref) < 1e-12 * abs(ref)


def test_A_kills_rigid_motions_and_is_spd_on_free_dofs():
    m = M.Mesh(3, 2, 2, 2, 1.0, 0.5, 0.8)
    mu = 1 + np.random.default_rng(1).random(m.n_nodes)
    Au = op.assemble_A(m, op.point_values(m, mu), mask=False)
    P = m.node_coords()
    zero = np.zeros(m.n_nodes)
    modes = [np.concatenate([zero + 1, zero, zero]),
             np.concatenate([-P[:, 1], P[:, 0], zero]),
             np.concatenate([zero, -P[:, 2], P[:, 1]]),
             np.concatenate([P[:, 2], zero, -P[:, 0]])]
    for r in modes:
        assert np.abs(Au @ r).max() < 1e-12
    # a non-rigid linear field is not killed (guards against a dropped symmetric part)
    shear = np.concatenate([P[:, 1], zero, zero])
    assert np.abs(Au @ shear).max() > 1e-3
    A = op.assemble_A(m, op.point_values(m, mu))
    assert abs(A - A.T).max() < 1e-13
    free = np.flatnonzero(m.interior_dof_mask())
    ev = np.linalg.eigvalsh(A[free][:, free].toarray())
    assert ev.min() > 0


def _pressure_coeffs(mesh, q_expr):
    """Per-element monomial coefficients of a global linear pressure q."""
    f = sy.lambdify(XYZ, [q_expr, sy.diff(q_expr, X), sy.diff(q_expr, Y), sy.diff(q_expr, Z)], "numpy")
    ec = mesh.element_coords()
    ctr = (ec + 0.5) * mesh.h[None, :]
    vals = [np.broadcast_to(np.asarray(v, dtype=float), (mesh.n_elem,)) for v in f(ctr[:, 0], ctr[:, 1], ctr[:, 2])]
    p = np.zeros((mesh.n_elem, mesh.Np))
    p[:, 0] = vals[0]
    for d in range(3):
        p[:, 1 + d] = vals[1 + d] * mesh.h[d] / 2   # xi_d = 2 (x_d - centre) / h_d
    return p.ravel()


def test_B_matches_symbolic_divergence_form():
    L = (1.0, 0.7, 1.3)
    m = M.Mesh(2, 3, 2, 2, *L)
    b = X * (L[0] - X) * Y * (L[1] - Y) * Z * (L[2] - Z)
    v = [b * 3, -2 * b, b]
    q = 0.5 + 2 * X - Y + 3 * Z
    B = op.assemble_B(m)
    ref = -_integrate(q * sum(sy.diff(v[d], XYZ[d]) for d in range(3)), L)
    got = _pressure_coeffs(m, q) @ B @ np.concatenate(_nodal(m, v))
    assert abs(got - ref) < 1e-12 * abs(ref)


def test_B_adjoint_and_constant_pressure_null():
    m = M.Mesh(3, 3, 2, 2)
    B = op.assemble_B(m)
    rng = np.random.default_rng(2)
    u, p = rng.standard_normal(m.n_u), rng.standard_normal(m.n_p)
    assert abs(p @ (B @ u) - (B.T @ p) @ u) < 1e-12
    assert np.abs(B.T @ op.constant_pressure(m)).max() < 1e-14
    # B ignores Dirichlet inputs
    ub = u * (~m.interior_dof_mask())
    assert np.abs(B @ ub).max() == 0.0


def test_lumped_weight_closed_form():
    n = 4
    m = M.Mesh(n, n, n, 2)
    mu = np.full(m.n_nodes, 9.0)
    a = 5.0
    C = op.lumped_weight_diag(m, mu, a)
    v_bnd = 1.0 - ((n - 2) / n) ** 3
    assert abs(C.sum() - 3.0 * ((1 - v_bnd) + a * v_bnd)) < 1e-12
    # a = 1 and mu = 1: the lumped mass of the cube, total volume 1
    assert abs(op.lumped_weight_diag(m, np.ones(m.n_nodes), 1.0).sum() - 1.0) < 1e-13


def test_Kw_symmetric_psd_with_constant_null():
    m = M.Mesh(3, 3, 3, 2)
    mu = np.exp(np.random.default_rng(3).standard_normal(m.n_nodes))
    B = op.assemble_B(m)
    K = op.assemble_Kw(B, op.lumped_weight_diag(m, mu, 2.0), m)
    assert abs(K - K.T).max() < 1e-14 * abs(K).max()
    assert np.abs(K @ op.constant_pressure(m)).max() < 1e-13 * abs(K).max()
    ev = np.linalg.eigvalsh(K.toarray())
    assert ev[0] > -1e-12 * ev[-1] and ev[1] > 1e-8 * ev[-1]   # one-dimensional null space


def test_Lc_matches_symbolic_form_and_neumann_null():
    L = (1.0, 0.7, 1.3)
    m = M.Mesh(2, 2, 3, 2, *L)
    rng = np.random.default_rng(4)
    mono = [1, X, Y, Z, X * Y, Y * Z, X * Z, X * Y * Z]
    u = sum(float(c) * t for c, t in zip(rng.standard_normal(8), mono))
    v = sum(float(c) * t for c, t in zip(rng.standard_normal(8), mono))
    c = 1 + X + Z
    Lc = op.assemble_Lc(m, op.point_values(m, _nodal(m, [c])[0]))
    uv, vv = _nodal(m, [u])[0], _nodal(m, [v])[0]
    ref = _integrate(c * sum(sy.diff(u, s) * sy.diff(v, s) for s in XYZ), L)
    assert abs(vv @ Lc @ uv - ref) < 1e-12 * max(1, abs(ref))
    assert np.abs(Lc @ np.ones(m.n_nodes)).max() < 1e-12


def test_pressure_mass_and_mixed_mass_exact():
    m = M.Mesh(2, 2, 2, 3, 1.0, 0.5, 2.0)
    Md = op.pressure_mass_element(m)
    ex = gll.pressure_exponents(3)

    def mono_int(p):
        return 0.0 if p % 2 else 2.0 / (p + 1)
    ref = np.array([[mono_int(a + a2) * mono_int(b + b2) * mono_int(c + c2) for (a2, b2, c2) in ex]
                    for (a, b, c) in ex]) * m.detJ
    np.testing.assert_allclose(Md, ref, rtol=1e-13, atol=1e-15)
    # M_dc u = int u psi_m for a Q_k field u (degree 3 per variable times degree <= 2)
    Mcd = op.mixed_mass(m)
    u = X ** 3 * Y + Z ** 2 - X * Y * Z
    uv = _nodal(m, [u])[0]
    got = (Mcd.T @ uv).reshape(m.n_elem, m.Np)
    e = 5   # element (1, 0, 1)
    ec = m.element_coords()[e]
    x0 = ec * m.h
    xi_sub = {X: x0[0] + (sy.Symbol("s") + 1) * m.h[0] / 2}
    s, t, r = sy.symbols("s t r")
    phys = {X: x0[0] + (s + 1) * m.h[0] / 2, Y: x0[1] + (t + 1) * m.h[1] / 2, Z: x0[2] + (r + 1) * m.h[2] / 2}
    ue = u.subs(phys)
    for mi, (a, b, c) in enumerate(ex):
        val = float(sy.integrate(ue * s ** a * t ** b * r ** c, (s, -1, 1), (t, -1, 1), (r, -1, 1))) * m.detJ
        assert abs(got[e, mi] - val) < 1e-13
    del xi_sub


def test_load_vector_exact_against_bubble():
    m = M.Mesh(3, 2, 2, 2)
    f = [1 + X, 2 - Y, Z]
    fn = np.stack(_nodal(m, f), axis=-1)
    F = op.load_vector(m, fn)
    b = X * (1 - X) * Y * (1 - Y) * Z * (1 - Z)
    bv = _nodal(m, [b])[0]
    for c in range(3):
        got = bv @ F[c * m.n_nodes:(c + 1) * m.n_nodes]
        assert abs(got - _integrate(b * f[c], (1, 1, 1))) < 1e-14


def test_sampled_apply_matches_csr():
    m = M.Mesh(3, 4, 2, 2, 1.0, 0.7, 1.3)
    rng = np.random.default_rng(5)
    mu, u = 1 + rng.random(m.n_nodes), rng.standard_normal(m.n_u)
    A = op.assemble_A(m, op.point_values(m, mu))
    nodes = rng.choice(m.n_nodes, 40, replace=False)
    y = op.sampled_apply_A(m, mu, u, nodes)
    ref = (A @ u).reshape(3, -1)[:, nodes].T
    np.testing.assert_allclose(y, ref, atol=1e-13)


def test_schur_complement_positive_definite_on_mean_zero():
    m = M.Mesh(2, 2, 2, 2)
    mu = np.ones(m.n_nodes)
    A = op.assemble_A(m, op.point_values(m, mu))
    B = op.assemble_B(m)
    free = np.flatnonzero(m.interior_dof_mask())
    Af = A[free][:, free].tocsc()
    S = B[:, free] @ spla.splu(Af).solve(B[:, free].T.toarray())
    ev = np.linalg.eigvalsh(0.5 * (S + S.T))
    assert ev[0] > -1e-12 and ev[1] > 1e-6   # S = B A^-1 B^T, kernel = constants only


def test_gradient_weights_on_polynomial_viscosity():
    """Viscosity-gradient w-BFBT weights (remark in Sec. 4): w = (mu^2 + |grad mu|^2)^(1/4).
    Q2 interpolates mu = 1 + x^2 + 3y exactly, so at every element point grad mu = (2x, 3, 0)."""
    from oracle import mesh as Mm
    m = Mm.Mesh(3, 2, 2, 2, 1.5, 1.0, 0.5)
    X = m.node_coords()
    mu = 1.0 + X[:, 0] ** 2 + 3.0 * X[:, 1]
    w = op.weight_points(m, mu, "grad")
    Xq = X[m.point_to_node()]                              # (n_elem, n^3, 3)
    mq = 1.0 + Xq[..., 0] ** 2 + 3.0 * Xq[..., 1]
    np.testing.assert_allclose(w, (mq ** 2 + 4.0 * Xq[..., 0] ** 2 + 9.0) ** 0.25, rtol=1e-12)
    np.testing.assert_allclose(op.weight_points(m, mu, "sqrt_mu"), np.sqrt(mq), rtol=1e-14)
    # a constant viscosity has no gradient: both weights agree
    c = np.full(m.n_nodes, 7.0)
    np.testing.assert_allclose(op.weight_points(m, c, "grad"), op.weight_points(m, c, "sqrt_mu"), rtol=1e-14)
    # the lumped weight sums W |J| a(e) w over the points at a node; the total is the integral
    tot = op.lumped_weight_diag(m, mu, 1.0, "grad").sum()
    np.testing.assert_allclose(tot, (w * (m.W * m.detJ)[None, :]).sum(), rtol=1e-13)


def test_diag_a_bfbt_weights_are_the_viscous_diagonal():
    """diag(A)-BFBT (Sec. 1.3): C = D = diag(A) per DOF; K_w = B diag(A)^-1 B^T equals the dense
    product written out, and the constant pressure mode is in its null space (B^T 1_psi = 0)."""
    from oracle import mesh as Mm
    from oracle import wbfbt as Wb
    m = Mm.Mesh(2, 2, 2, 2)
    mu = 1.0 + m.node_coords()[:, 0]
    prob = Wb.StokesProblem(m, mu, weights="diag_a")
    A = prob.A.toarray()
    free = m.interior_dof_mask()
    np.testing.assert_allclose(prob.Cinv[free], 1.0 / np.diag(A)[free], rtol=1e-14)
    assert np.all(prob.Cinv[~free] == 0.0)
    K = op.assemble_Kw(prob.B, prob.Cdiag, m).toarray()
    Bd = prob.B.toarray()
    np.testing.assert_allclose(K, Bd @ np.diag(prob.Cinv) @ Bd.T, rtol=1e-13, atol=1e-13 * np.abs(K).max())
    np.testing.assert_allclose(K @ op.constant_pressure(m), 0.0, atol=1e-12 * np.abs(K).max())
