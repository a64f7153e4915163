"""Pins for the oracle's multigrid pieces: transfers, coefficient coarsening, Chebyshev, V-cycles."""
import numpy as np
import pytest
import scipy.sparse as sp
import sympy as sy

from oracle import gll
from oracle import mesh as M
from oracle import multigrid as mg
from oracle import operators as op

X, Y, Z = sy.symbols("x y z")


def _nodal(mesh, expr):
    f = sy.lambdify((X, Y, Z), expr, "numpy")
    P = mesh.node_coords()
    return np.broadcast_to(np.asarray(f(P[:, 0], P[:, 1], P[:, 2]), dtype=float), (mesh.n_nodes,)).copy()


@pytest.mark.parametrize("k", [1, 2, 3])
def test_prolongation_reproduces_qk_polynomials(k):
    mc = M.Mesh(2, 3, 2, k, 1.0, 0.7, 1.3)
    mf = M.Mesh(4, 6, 4, k, 1.0, 0.7, 1.3)
    expr = (1 + X ** k) * (2 - Y ** k + Y) * (Z ** k - 3 * Z)   # degree <= k per variable
    P = mg.prolongation_scalar(mc)
    np.testing.assert_allclose(P @ _nodal(mc, expr), _nodal(mf, expr), atol=1e-12)
    # a coarse field vanishing on the boundary stays zero on the fine boundary (Dirichlet kept)
    uc = np.random.default_rng(0).standard_normal(mc.n_nodes) * (~mc.boundary_node_mask())
    assert np.abs((P @ uc)[mf.boundary_node_mask()]).max() < 1e-15


def _brute_coarsen(mf, c_fine, basis):
    """Direct 3-D evaluation of sum_{e,q'} W' |J_e| phi_q(x') c / normaliser."""
    mc = mf.coarsen()
    n = mf.n
    xi, w = mf.xi, mf.w1
    lq = mf.local_ijk()
    out = np.zeros((mc.n_elem, n ** 3))
    ecs = mc.element_coords()
    efs = mf.element_coords()
    for E, ec in enumerate(ecs):
        num = np.zeros(n ** 3)
        den = np.zeros(n ** 3)
        for e, ef in enumerate(efs):
            if not np.all(ef // 2 == ec):
                continue
            s = ef % 2
            for qp in range(n ** 3):
                t = (xi[lq[qp]] + 2 * s - 1) / 2.0          # coarse reference coords of fine point
                wq = w[lq[qp]].prod() * mf.detJ
                for q in range(n ** 3):
                    phi = np.prod([basis(xi, t[d])[lq[q][d]] for d in range(3)])
                    num[q] += wq * phi * c_fine[e, qp]
                    den[q] += wq * phi
        out[E] = num / den if basis is _hat else num / (w[lq].prod(axis=1) * mc.detJ)
    return out


def _hat(x, t):
    return mg.hat_eval(x, np.array([t]))[0]


def _lagrange(x, t):
    return gll.lagrange_eval(x, np.array([t]))[0]


def test_coefficient_coarsening_k1_is_the_l2_adjoint_of_trilinear_interpolation():
    # for k = 1 the hat basis is the trilinear Lagrange basis and the normaliser is W_q |J_E|
    mf = M.Mesh(4, 2, 2, 1, 1.0, 0.7, 1.3)
    c = np.random.default_rng(1).random((mf.n_elem, 8)) + 0.1
    np.testing.assert_allclose(mg.coarsen_coefficient(mf, c), _brute_coarsen(mf, c, _lagrange), rtol=1e-13)


@pytest.mark.parametrize("k", [2, 3])
def test_coefficient_coarsening_brute_force_and_properties(k):
    mf = M.Mesh(2, 2, 2, k)
    rng = np.random.default_rng(k)
    c = np.exp(3 * rng.standard_normal((mf.n_elem, (k + 1) ** 3)))
    got = mg.coarsen_coefficient(mf, c)
    np.testing.assert_allclose(got, _brute_coarsen(mf, c, _hat), rtol=1e-12)
    assert got.min() >= c.min() and got.max() <= c.max()      # convex combinations
    ones = np.ones_like(c)
    np.testing.assert_allclose(mg.coarsen_coefficient(mf, ones), 1.0, rtol=1e-14)


def test_chebyshev_error_polynomial():
    lam = np.linspace(0.05, 2.0, 40)
    Mx = sp.diags(lam)
    lam_hat = 2.0 / 1.1
    b = np.random.default_rng(2).standard_normal(lam.size)
    xstar = b / lam
    lo, hi = 0.1 * lam_hat, 1.1 * lam_hat
    th, de = (hi + lo) / 2, (hi - lo) / 2

    def T3(t):
        return 4 * t ** 3 - 3 * t
    factor = T3((th - lam) / de) / T3(th / de)
    x, r = mg.chebyshev(Mx, np.ones(lam.size), b, None, lam_hat, want_residual=True)
    np.testing.assert_allclose(xstar - x, factor * xstar, atol=1e-12)
    np.testing.assert_allclose(r, b - Mx @ x, atol=1e-12)
    x0 = np.random.default_rng(3).standard_normal(lam.size)
    x1, _ = mg.chebyshev(Mx, np.ones(lam.size), b, x0, lam_hat)
    np.testing.assert_allclose(xstar - x1, factor * (xstar - x0), atol=1e-12)


def test_power_iteration_estimates_top_eigenvalue():
    lam = np.linspace(0.1, 3.0, 200)
    est = mg.power_lambda(sp.diags(lam), np.ones(200), mg.splitmix64_uniform(mg.START_SEED, 200))
    assert 0.85 * 3.0 < est <= 3.0


def _sinker_mu(m, dr=1e4):
    from oracle import sinker
    from paper_1607_03936_gb300 import inputs
    return sinker.viscosity(m.node_coords(), inputs.sinker_centres(0, 4), 0.1, 200.0, dr)


def test_vcycle_is_symmetric_and_converges():
    m = M.Mesh(8, 8, 8, 2)
    mu = _sinker_mu(m)
    levels = mg.build_hierarchy(m, op.point_values(m, mu), vector=True)
    assert len(levels) == 2
    rng = np.random.default_rng(4)
    mask = m.interior_dof_mask()
    x, y = rng.standard_normal(m.n_u) * mask, rng.standard_normal(m.n_u) * mask
    a, b = y @ mg.vcycle(levels, x), x @ mg.vcycle(levels, y)
    assert abs(a - b) < 1e-11 * abs(a)
    # the V-cycle output is zero on Dirichlet DOFs
    assert np.abs(mg.vcycle(levels, x)[~mask]).max() == 0.0


def test_single_level_vcycle_is_the_direct_solve():
    m = M.Mesh(4, 4, 4, 2)
    mu = _sinker_mu(m)
    levels = mg.build_hierarchy(m, op.point_values(m, mu), vector=True)
    assert len(levels) == 1
    b = np.random.default_rng(5).standard_normal(m.n_u) * m.interior_dof_mask()
    x = mg.vcycle(levels, b)
    A = levels[0].M
    np.testing.assert_allclose(A @ x, b, atol=1e-9 * np.abs(b).max())


def test_disc_cont_transfers_are_adjoint_and_project_exactly():
    m = M.Mesh(3, 2, 2, 3)
    mu = 1 + np.random.default_rng(6).random(m.n_nodes)
    B = op.assemble_B(m)
    pp = mg.PressurePoissonMG(m, B, op.lumped_weight_diag(m, mu, 1.0), mu, 1.0)
    rng = np.random.default_rng(7)
    xc, yd = rng.standard_normal(m.n_nodes), rng.standard_normal(m.n_p)
    assert abs(xc @ pp.disc_to_cont(yd) - pp.cont_to_disc(xc) @ yd) < 1e-12
    # a global polynomial of total degree k-1 = 2 survives Q_k -> P_{k-1}^disc projection exactly
    expr = 1 + 2 * X - Y + X * Z + 3 * Y ** 2
    pd = pp.cont_to_disc(_nodal(m, expr)).reshape(m.n_elem, m.Np)
    ex = gll.pressure_exponents(3)
    e = 7
    ctr = (m.element_coords()[e] + 0.5) * m.h
    s, t, r = sy.symbols("s t r")
    loc = sy.Poly(sy.expand(expr.subs({X: ctr[0] + s * m.h[0] / 2, Y: ctr[1] + t * m.h[1] / 2,
                                       Z: ctr[2] + r * m.h[2] / 2})), s, t, r)
    want = [float(loc.coeff_monomial(s ** a * t ** b * r ** c)) for (a, b, c) in ex]
    np.testing.assert_allclose(pd[e], want, atol=1e-12)


def test_pressure_poisson_vcycle_symmetric():
    m = M.Mesh(8, 8, 8, 2)
    mu = _sinker_mu(m)
    B = op.assemble_B(m)
    pp = mg.PressurePoissonMG(m, B, op.lumped_weight_diag(m, mu, 2.0), mu, 2.0)
    rng = np.random.default_rng(8)
    x = op.project_pressure(m, rng.standard_normal(m.n_p))
    y = op.project_pressure(m, rng.standard_normal(m.n_p))
    a, b = y @ op.project_pressure(m, pp.apply(x)), x @ op.project_pressure(m, pp.apply(y))
    assert abs(a - b) < 1e-10 * abs(a)


def test_single_element_mesh_pressure_poisson_is_finite():
    """Degenerate case: one element, every face Dirichlet; the constant mode has a zero K_w diagonal."""
    m = M.Mesh(1, 1, 1, 2)
    mu = np.ones(m.n_nodes)
    B = op.assemble_B(m)
    pp = mg.PressurePoissonMG(m, B, op.lumped_weight_diag(m, mu, 1.0), mu, 1.0)
    assert pp.dinv[0] == 0.0 and np.all(pp.dinv[1:] > 0)
    y = pp.apply(op.project_pressure(m, np.arange(m.n_p, dtype=float)))
    assert np.all(np.isfinite(y))


def test_p_prolongation_embeds_trilinear_functions():
    """Q1 vertex values of a trilinear function, carried to the Q2 (and Q3) nodes of the same mesh,
    equal that function at those nodes (the embedding Q1 in Q_k is exact)."""
    from oracle import mesh as Mm
    for k in (2, 3):
        mf = Mm.Mesh(3, 2, 2, k, 1.5, 1.0, 0.5)
        m1 = Mm.Mesh(3, 2, 2, 1, 1.5, 1.0, 0.5)
        f = lambda X: 1.0 + 2.0 * X[:, 0] - X[:, 1] + 0.5 * X[:, 2] + 3.0 * X[:, 0] * X[:, 1] * X[:, 2]
        P = mg.p_prolongation_vector(mf)
        u1 = np.concatenate([f(m1.node_coords())] * 3)
        np.testing.assert_allclose(P @ u1, np.concatenate([f(mf.node_coords())] * 3), rtol=1e-13, atol=1e-13)


def test_p_coarsen_coefficient_weights():
    """k = 2: per axis the vertex weights are W_a phi_v(x_a) normalised, W = (1/3, 4/3, 1/3), phi_0 =
    (1, 1/2, 0): (1/3, 2/3, 0) -- a coefficient equal to the reference coordinate xi along x gives
    -1/3 at the left vertices and +1/3 at the right; constants are kept."""
    from oracle import mesh as Mm
    m = Mm.Mesh(1, 1, 1, 2)
    xi = m.ref_pts[:, 0]
    c1 = mg.p_coarsen_coefficient(m, xi[None, :]).reshape(2, 2, 2)    # (vz, vy, vx)
    np.testing.assert_allclose(c1[..., 0], -1.0 / 3.0, rtol=1e-14)
    np.testing.assert_allclose(c1[..., 1], 1.0 / 3.0, rtol=1e-14)
    const = mg.p_coarsen_coefficient(m, np.full((1, 27), 2.5))
    np.testing.assert_allclose(const, 2.5, rtol=1e-14)


def test_p_coarsened_hierarchy_levels():
    """pmg: Q2 on 8^3, Q1 on 8^3, Q1 on 4^3 (coarsest); the Q1 operator on the same mesh equals the
    Galerkin-free re-discretisation with the p-coarsened coefficient (symmetric, SPD on free DOFs)."""
    from oracle import mesh as Mm
    from oracle import operators as opx
    m = Mm.Mesh(8, 8, 8, 2)
    mu = 1.0 + m.node_coords()[:, 0] ** 2
    lv = mg.build_hierarchy(m, opx.point_values(m, mu), True, pmg=True)
    assert [(l.mesh.nx, l.mesh.k) for l in lv] == [(8, 2), (8, 1), (4, 1)]
    M1 = lv[1].M
    assert abs(M1 - M1.T).max() < 1e-12 * abs(M1).max()
    assert lv[0].P.shape == (3 * 17 ** 3, 3 * 9 ** 3)
