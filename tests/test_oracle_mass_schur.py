"""Pins of the oracle's lumped inverse-viscosity pressure mass (Sec. 1.3, Eq. lumping).

M~_p(1/mu) = diag(M_p(1/mu) 1_psi), lumped in the element basis phi'_j = s^a t^b u^c,
s = (1 + xi)/2 (non-negative), and carried to the solver's centred monomials psi_m by p = T p'.
Expected values are integrals worked out by hand:  int_0^1 s^a ds = 1/(a + 1).
"""
import numpy as np

from oracle import mesh as M
from oracle import operators as op
from oracle import wbfbt as W

# k = 2: psi = (1, xi, eta, zeta), phi' = (1, s, t, u), s = (1 + xi)/2 = psi_0/2 + psi_1/2, ...
T2 = np.array([[1.0, 0.5, 0.5, 0.5],
               [0.0, 0.5, 0.0, 0.0],
               [0.0, 0.0, 0.5, 0.0],
               [0.0, 0.0, 0.0, 0.5]])


def blocks(S, m):
    S = S.toarray()
    return [S[e * m.Np:(e + 1) * m.Np, e * m.Np:(e + 1) * m.Np] for e in range(m.n_elem)]


def test_constant_viscosity_single_element_q2():
    m = M.Mesh(1, 1, 1, 2, 0.5, 1.0, 2.0)          # volume 1
    mu0 = 4.0
    S = op.lumped_mass_schur_inverse(m, np.full(m.n_nodes, mu0))
    # d' = vol / mu0 (1, 1/2, 1/2, 1/2); S = T diag(1/d') T^T = (mu0 / vol) x the matrix below
    expect = mu0 * np.array([[2.5, 0.5, 0.5, 0.5],
                             [0.5, 0.5, 0.0, 0.0],
                             [0.5, 0.0, 0.5, 0.0],
                             [0.5, 0.0, 0.0, 0.5]])
    np.testing.assert_allclose(blocks(S, m)[0], expect, rtol=1e-13, atol=1e-13)


def test_linear_inverse_viscosity_two_elements_q2():
    # 1/mu = 1 + x on [0,1] x [0,1] x [0,1] split in two along x: elements [0, .5] and [.5, 1]
    m = M.Mesh(2, 1, 1, 2)
    X = m.node_coords()
    S = op.lumped_mass_schur_inverse(m, 1.0 / (1.0 + X[:, 0]))
    # element 0: x = s/2, vol 1/2:  d'_0 = 1/2 int (1 + s/2) = 0.625, d'_s = 1/2 int s (1 + s/2) = 1/3,
    #            d'_t = d'_u = 1/2 (1/2)(1.25) = 0.3125
    # element 1: x = 1/2 + s/2:    d'_0 = 0.875, d'_s = 1/2 (3/4 + 1/6) = 11/24, d'_t = d'_u = 0.4375
    d = [np.array([0.625, 1.0 / 3.0, 0.3125, 0.3125]), np.array([0.875, 11.0 / 24.0, 0.4375, 0.4375])]
    for e, Be in enumerate(blocks(S, m)):
        np.testing.assert_allclose(Be, T2 @ np.diag(1.0 / d[e]) @ T2.T, rtol=1e-13, atol=1e-13)


def test_constant_mode_keeps_the_exact_inverse_viscosity_integral():
    """In the solver's basis the lumped matrix S~_e = T^-T diag(d') T^-1 gives e_0^T S~_e e_0 =
    d'_0 = int_e 1/mu: the constant pressure mode sees the exact weighted mass (any k, any mu)."""
    for k in (2, 3, 4):
        m = M.Mesh(2, 1, 1, k)
        X = m.node_coords()
        S = op.lumped_mass_schur_inverse(m, 1.0 / (1.0 + X[:, 0]))
        for e, Be in enumerate(blocks(S, m)):
            St = np.linalg.inv(Be)
            # int over [e/2, (e+1)/2] x [0,1]^2 of (1 + x) dx = 1/2 + (2e + 1)/8
            np.testing.assert_allclose(St[0, 0], 0.5 + (2 * e + 1) / 8.0, rtol=1e-12)
            assert np.allclose(Be, Be.T) and np.all(np.linalg.eigvalsh(Be) > 0)


def test_q3_constant_viscosity_diagonal_in_the_nonnegative_basis():
    """k = 3, constant mu: d'_j = vol / mu0 x prod_d 1/(e_jd + 1) for phi'_j = s^a t^b u^c."""
    m = M.Mesh(1, 1, 1, 3)
    mu0 = 0.5
    S = blocks(op.lumped_mass_schur_inverse(m, np.full(m.n_nodes, mu0)), m)[0]
    psi = op.gll.pressure_basis_at_points(3, m.ref_pts)
    phi = op.nonneg_pressure_basis_at_points(3, m.ref_pts)
    T = np.linalg.lstsq(psi, phi, rcond=None)[0]
    d = np.linalg.inv(T) @ S @ np.linalg.inv(T.T)     # = diag(1/d')
    exps = op.gll.pressure_exponents(3)
    want = np.array([mu0 * (a + 1) * (b + 1) * (c + 1) for a, b, c in exps])
    np.testing.assert_allclose(np.diag(d), want, rtol=1e-12)
    np.testing.assert_allclose(d - np.diag(np.diag(d)), 0.0, atol=1e-11)


def test_diag_mass_constant_viscosity_q2():
    """Diagonal variant, k = 2, constant mu0: int_e psi_m^2 / mu0 = vol / mu0 (1, 1/3, 1/3, 1/3)."""
    m = M.Mesh(2, 1, 1, 2, 1.0, 0.5, 0.5)        # two elements of volume 1/8
    S = op.diag_mass_schur_inverse(m, np.full(m.n_nodes, 2.0)).toarray()
    np.testing.assert_allclose(np.diag(S), np.tile([16.0, 48.0, 48.0, 48.0], 2), rtol=1e-13)
    assert np.count_nonzero(S - np.diag(np.diag(S))) == 0


def test_mass_schur_solves_converge_and_wbfbt_is_faster_on_sinkers():
    """All three Schur approximations solve the 4^3 multi-sinker problem at DR 1e2; w-BFBT needs
    the fewest iterations (the trend of Table 1)."""
    from paper_1607_03936_gb300 import inputs
    m = M.Mesh(4, 4, 4, 2)
    c = inputs.sinker_centres(0, 4)
    mu, f = W.sinker_problem(m, c, 0.1, 200.0, 1e2)
    its = {}
    for schur in ("mass", "mass_diag", "wbfbt"):
        _, _, its[schur], rel, _ = W.solve(m, mu, f, W.Options(schur=schur), maxit=1000)
        assert rel <= 1e-6, schur
    assert its["wbfbt"] < its["mass_diag"] <= its["mass"], its
