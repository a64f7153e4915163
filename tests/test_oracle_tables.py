"""Pins for the oracle's reference-element tables, sizes and generators (CPU only)."""
import os

import numpy as np
import pytest

from oracle import gll
from oracle import mesh as M
from oracle import multigrid as mg
from paper_1607_03936_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_gll_closed_forms():
    x, w = gll.gll_nodes_weights(2)
    np.testing.assert_allclose(x, [-1, 0, 1], atol=1e-15)
    np.testing.assert_allclose(w, [1 / 3, 4 / 3, 1 / 3], rtol=1e-14)
    x, w = gll.gll_nodes_weights(3)
    s = 1 / np.sqrt(5)
    np.testing.assert_allclose(x, [-1, -s, s, 1], atol=1e-15)
    np.testing.assert_allclose(w, [1 / 6, 5 / 6, 5 / 6, 1 / 6], rtol=1e-14)
    x, w = gll.gll_nodes_weights(4)
    t = np.sqrt(3 / 7)
    np.testing.assert_allclose(x, [-1, -t, 0, t, 1], atol=1e-15)
    np.testing.assert_allclose(w, [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10], rtol=1e-14)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_gll_quadrature_exact_to_degree_2k_minus_1(k):
    x, w = gll.gll_nodes_weights(k)
    for p in range(2 * k):
        exact = 0.0 if p % 2 else 2.0 / (p + 1)
        assert abs(w @ x ** p - exact) < 1e-13
    # and not exact at degree 2k (GLL loses one degree against Gauss)
    assert abs(w @ x ** (2 * k) - 2.0 / (2 * k + 1)) > 1e-6


@pytest.mark.parametrize("k", [2, 3, 4])
def test_derivative_matrix_exact_on_polynomials(k):
    x, _ = gll.gll_nodes_weights(k)
    D = gll.derivative_matrix(x)
    for p in range(k + 1):
        d_exact = p * x ** (p - 1) if p > 0 else 0 * x
        np.testing.assert_allclose(D @ x ** p, d_exact, atol=1e-12)
    # negative-antisymmetry of GLL differentiation: D[i,j] = -D[n-1-i, n-1-j]
    np.testing.assert_allclose(D, -D[::-1, ::-1], atol=1e-13)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 8])
def test_pressure_mode_count(k):
    ex = gll.pressure_exponents(k)
    assert len(ex) == k * (k + 1) * (k + 2) // 6
    assert ex[0] == (0, 0, 0)
    assert len(set(ex)) == len(ex)
    assert all(sum(e) <= k - 1 for e in ex)
    if k == 2:
        assert ex == [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]


def test_table3_dof_counts():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table3_dof_counts.txt")) if not l.startswith("#")]
    assert len(rows) == 13
    for r in rows:
        level, k = int(r[0]), int(r[1])
        nu, npr = M.table3_dof_counts(level, k)
        assert abs(nu / 1e6 - float(r[3])) <= 0.0101, r
        assert abs(npr / 1e6 - float(r[4])) <= 0.0101, r
        assert abs((nu + npr) / 1e6 - float(r[5])) <= 0.0101, r


def test_splitmix64_published_outputs():
    vals = [int(l, 16) for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) if not l.startswith("#")]
    assert inputs.splitmix64_stream(0, 3) == vals
    # the oracle's vectorised counter form gives the same stream (top 53 bits)
    u = mg.splitmix64_uniform(0, 3) + 0.5
    np.testing.assert_array_equal(u, np.array([(v >> 11) / 2.0 ** 53 for v in vals]))


def test_sinker_centres_in_box_and_seeded():
    c = inputs.sinker_centres(7, 16)
    assert c.shape == (16, 3)
    assert c.min() >= 0.1 and c.max() <= 0.9
    np.testing.assert_array_equal(c, inputs.sinker_centres(7, 16))
    assert not np.array_equal(c, inputs.sinker_centres(8, 16))


def test_level_counts():
    assert mg.n_levels(M.Mesh(32, 32, 32, 2)) == 4
    assert mg.n_levels(M.Mesh(8, 8, 8, 2)) == 2
    assert mg.n_levels(M.Mesh(24, 24, 24, 3)) == 4   # 24, 12, 6, 3
    assert mg.n_levels(M.Mesh(64, 64, 64, 2)) == 5
    assert mg.n_levels(M.Mesh(4, 4, 4, 2)) == 1
