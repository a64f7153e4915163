"""Pins of the oracle's multi-sinker viscosity and forcing (Sec. 2.1) against closed forms.

Sec. 2.1 fixes: mu = (mu_max - mu_min)(1 - chi) + mu_min with mu_min = DR^(-1/2),
mu_max = DR^(1/2); chi = prod_i [1 - exp(-delta max(0, |c_i - x| - omega/2)^2)];
f = (0, 0, beta (chi - 1)), beta = 10.  The expected values below are worked out by
hand (exponentials written as decimal literals), so a swapped mu_min/mu_max, omega in
place of omega/2, a wrong sign of beta (chi - 1) or a sum in place of the product fails.
"""
import numpy as np

from oracle import sinker

E_M1 = 0.36787944117144233     # e^-1
E_M2 = 0.1353352832366127      # e^-2
E_M4 = 0.01831563888873418     # e^-4


def test_inside_sinker_attains_mu_max_and_full_downward_force():
    c = np.array([[0.5, 0.5, 0.5]])
    omega, delta, dr = 0.1, 200.0, 1e4
    # points at distance 0, 0.02, 0.0499 from the centre: inside the radius omega/2 = 0.05
    x = np.array([[0.5, 0.5, 0.5], [0.52, 0.5, 0.5], [0.5, 0.5, 0.5499]])
    mu = sinker.viscosity(x, c, omega, delta, dr)
    np.testing.assert_allclose(mu, 100.0, rtol=1e-15)           # DR^(1/2) = 100
    f = sinker.forcing(x, c, omega, delta)
    np.testing.assert_allclose(f[:, 2], -10.0, rtol=1e-15)      # beta (0 - 1)
    assert np.all(f[:, :2] == 0.0)


def test_far_field_tends_to_mu_min_and_zero_force():
    c = np.array([[0.2, 0.2, 0.2]])
    omega, delta, dr = 0.1, 200.0, 1e6
    x = np.array([[0.95, 0.95, 0.95]])                         # |x - c| = 1.299, s^2 delta ~ 311
    mu = sinker.viscosity(x, c, omega, delta, dr)
    np.testing.assert_allclose(mu, 1e-3, rtol=1e-12)            # DR^(-1/2)
    f = sinker.forcing(x, c, omega, delta)
    assert abs(f[0, 2]) < 1e-100


def test_hand_computed_single_sinker_value():
    # distance 0.15 from the centre, omega/2 = 0.05, so s = 0.1; delta s^2 = 2
    c = np.array([[0.3, 0.4, 0.5]])
    x = np.array([[0.3, 0.55, 0.5], [0.3, 0.4, 0.35]])
    omega, delta, dr = 0.1, 200.0, 1e4
    chi = sinker.indicator(x, c, omega, delta)
    np.testing.assert_allclose(chi, 1.0 - E_M2, rtol=1e-14)
    mu = sinker.viscosity(x, c, omega, delta, dr)
    np.testing.assert_allclose(mu, 99.99 * E_M2 + 0.01, rtol=1e-14)
    f = sinker.forcing(x, c, omega, delta)
    np.testing.assert_allclose(f[:, 2], -10.0 * E_M2, rtol=1e-14)


def test_radius_is_half_the_diameter():
    # a point at distance 0.75 omega: outside the plateau of radius omega/2
    # (delta s^2 = 400 * 0.025^2 = 0.25), inside it were the radius omega
    c = np.array([[0.5, 0.5, 0.5]])
    x = np.array([[0.575, 0.5, 0.5]])
    omega, delta, dr = 0.1, 400.0, 1e2
    chi = sinker.indicator(x, c, omega, delta)
    e_m025 = 0.7788007830714049  # e^-0.25
    np.testing.assert_allclose(chi, 1.0 - e_m025, rtol=1e-14)
    mu = sinker.viscosity(x, c, omega, delta, dr)
    np.testing.assert_allclose(mu, 9.9 * e_m025 + 0.1, rtol=1e-14)


def test_two_sinkers_multiply():
    # s1 = 0.1 from sinker 1 (delta s^2 = 1), s2 = 0.2 from sinker 2 (delta s^2 = 4)
    c = np.array([[0.2, 0.5, 0.5], [0.65, 0.5, 0.5]])
    x = np.array([[0.35, 0.5, 0.5]])        # |x - c1| = 0.15, |x - c2| = 0.30
    omega, delta, dr = 0.1, 100.0, 1e8
    chi = sinker.indicator(x, c, omega, delta)
    # second factor: s2 = 0.30 - 0.05 = 0.25, delta s^2 = 6.25; written out: e^-6.25
    expect = (1.0 - E_M1) * (1.0 - 0.0019304541362277093)
    np.testing.assert_allclose(chi, expect, rtol=1e-14)
    mu = sinker.viscosity(x, c, omega, delta, dr)
    np.testing.assert_allclose(mu, (1e4 - 1e-4) * (1.0 - expect) + 1e-4, rtol=1e-13)
    f = sinker.forcing(x, c, omega, delta, beta=10.0)
    np.testing.assert_allclose(f[0], [0.0, 0.0, 10.0 * (expect - 1.0)], rtol=1e-14, atol=0)


def test_range_and_reciprocal_extremes():
    rng = np.random.default_rng(3)
    c = rng.uniform(0.1, 0.9, size=(12, 3))
    x = rng.uniform(0.0, 1.0, size=(4000, 3))
    for dr in (1e4, 1e6, 1e10):
        mu = sinker.viscosity(x, c, 0.1, 200.0, dr)
        mu_min, mu_max = mu.min(), mu.max()
        assert dr ** -0.5 * (1 - 1e-12) <= mu_min and mu_max <= dr ** 0.5 * (1 + 1e-12)
    # DR = 1e10: mu_min * mu_max = 1, ratio DR
    x2 = np.array(c[:1]) + 0.0                          # a centre: mu_max
    x3 = np.array([[0.0, 0.0, 0.0]]) - 5.0               # far away: mu_min
    a = sinker.viscosity(x2, c, 0.1, 200.0, 1e10)[0]
    b = sinker.viscosity(x3, c, 0.1, 200.0, 1e10)[0]
    np.testing.assert_allclose(a, 1e5, rtol=1e-15)
    np.testing.assert_allclose(b, 1e-5, rtol=1e-12)


def test_decay_factor_e_minus_4():
    c = np.array([[0.5, 0.5, 0.5]])
    x = np.array([[0.5, 0.5, 0.75]])         # s = 0.25 - 0.05 = 0.2, delta s^2 = 100 * 0.04 = 4
    chi = sinker.indicator(x, c, 0.1, 100.0)
    np.testing.assert_allclose(chi, 1.0 - E_M4, rtol=1e-14)
