"""Pins of the mapped-hexahedron oracle (isoparametric Q_k geometry, the forms of Sec. 1.2).

Each pin fixes the mapped operators by something other than the oracle's own formula:
  - an axis-aligned, evenly spaced node placement is the brick, whose operators (2/h-scaled
    derivatives, constant |J|) are computed by other code;
  - affine fields are in the isoparametric space, so for u = G x the energy u^T A u is
    2 mu |sym G|^2 vol(Omega) and the constant-pressure row of B u is -tr(G) vol(Omega), exactly
    on straight-edged (trilinear) elements, where the (k+1)-point GLL rule integrates det J;
  - rigid motions c + w x x have eps = 0 and div = 0 at every point of any geometry, and the
    unmasked A has exactly six zero eigenvalues (no spurious kernel);
  - a rotation of mesh and field leaves energies and divergences unchanged, a dilation by s scales
    A by s and B by s^2;
  - a planted transposition of J^-1 fails the patch test.
"""
import numpy as np
import pytest

from oracle import mapped as mp
from oracle import operators as op
from oracle import sinker, wbfbt
from oracle.mesh import Mesh
from paper_1607_03936_gb300 import inputs

LEN = (1.0, 0.7, 1.3)


def mesh_and_coords(kind, k=2, n=(3, 2, 4), amp=None, seed=1):
    m = Mesh(*n, k, *LEN)
    X0 = m.node_coords()
    if kind == "brick":
        return m, X0
    if kind == "trilinear":
        return m, inputs.deform_vertices(X0, n, LEN, 0.15 if amp is None else amp, seed)
    return m, inputs.deform_smooth(X0, LEN, 0.1 if amp is None else amp)


def relmax(a, b):
    return abs(a - b).max() / abs(b).max()


@pytest.mark.parametrize("k", [2, 3, 4])
def test_axis_aligned_nodes_give_the_brick_operators(k):
    m, X = mesh_and_coords("brick", k=k)
    mu = np.random.default_rng(0).uniform(1.0, 5.0, m.n_nodes)
    mu_pts = op.point_values(m, mu)
    assert relmax(mp.assemble_A(m, X, mu_pts), op.assemble_A(m, mu_pts)) < 1e-13
    assert relmax(mp.assemble_B(m, X), op.assemble_B(m)) < 1e-13
    f = np.random.default_rng(1).standard_normal((m.n_nodes, 3))
    assert relmax(mp.load_vector(m, X, f), op.load_vector(m, f)) < 1e-13
    assert relmax(mp.lumped_weight_diag(m, X, mu, 2.0), op.lumped_weight_diag(m, mu, 2.0)) < 1e-13


@pytest.mark.parametrize("k", [2, 3, 4])
def test_affine_fields_patch_test_on_trilinear_elements(k):
    m, X = mesh_and_coords("trilinear", k=k)
    vol = LEN[0] * LEN[1] * LEN[2]
    mu0 = 1.7
    A = mp.assemble_A(m, X, np.full((m.n_elem, m.n ** 3), mu0), mask=False)
    B = mp.assemble_B(m, X, mask=False)
    one = op.constant_pressure(m)
    rng = np.random.default_rng(3)
    for _ in range(3):
        G = rng.standard_normal((3, 3))
        u = (X @ G.T).T.ravel()                      # component-major nodal values of G x
        sG = 0.5 * (G + G.T)
        assert abs(u @ (A @ u) - 2.0 * mu0 * vol * np.sum(sG * sG)) < 1e-11 * (1.0 + abs(u @ (A @ u)))
        assert abs(one @ (B @ u) + np.trace(G) * vol) < 1e-12 * (1.0 + abs(np.trace(G)))
    # volume through the load vector of f = e_x
    f = np.zeros((m.n_nodes, 3))
    f[:, 0] = 1.0
    assert abs(mp.load_vector(m, X, f, mask=False).sum() - vol) < 1e-13


def test_planted_jacobian_transposition_fails_the_patch_test(monkeypatch):
    m, X = mesh_and_coords("trilinear")
    real_inv = np.linalg.inv
    monkeypatch.setattr(mp.np.linalg, "inv", lambda a: np.swapaxes(real_inv(a), -1, -2))
    A = mp.assemble_A(m, X, np.ones((m.n_elem, m.n ** 3)), mask=False)
    G = np.array([[0.3, 1.1, -0.4], [0.2, -0.7, 0.9], [1.3, 0.1, 0.5]])
    u = (X @ G.T).T.ravel()
    sG = 0.5 * (G + G.T)
    assert abs(u @ (A @ u) - 2.0 * np.prod(LEN) * np.sum(sG * sG)) > 1e-3


@pytest.mark.parametrize("kind", ["trilinear", "smooth"])
def test_rigid_motions_are_the_kernel(kind):
    m, X = mesh_and_coords(kind)
    mu = op.point_values(m, np.random.default_rng(4).uniform(1.0, 10.0, m.n_nodes))
    A = mp.assemble_A(m, X, mu, mask=False)
    B = mp.assemble_B(m, X, mask=False)
    rng = np.random.default_rng(5)
    for _ in range(3):
        w, c = rng.standard_normal(3), rng.standard_normal(3)
        ur = (c + np.cross(w, X)).T.ravel()
        assert np.abs(A @ ur).max() < 1e-13 * abs(A).max() * np.abs(ur).max()
        assert np.abs(B @ ur).max() < 1e-13 * abs(B).max() * np.abs(ur).max()


def test_unmasked_A_has_exactly_six_zero_eigenvalues_on_curved_elements():
    m, X = mesh_and_coords("smooth", n=(2, 2, 2), amp=0.1)
    A = mp.assemble_A(m, X, np.ones((m.n_elem, m.n ** 3)), mask=False).toarray()
    ev = np.linalg.eigvalsh(A)
    assert np.all(ev > -1e-12 * ev[-1])
    assert np.all(ev[:6] < 1e-12 * ev[-1])
    assert ev[6] > 1e-4 * ev[-1]


@pytest.mark.parametrize("kind", ["trilinear", "smooth"])
def test_rotation_and_dilation(kind):
    m, X = mesh_and_coords(kind)
    mu = op.point_values(m, np.random.default_rng(6).uniform(1.0, 10.0, m.n_nodes))
    A = mp.assemble_A(m, X, mu, mask=False)
    B = mp.assemble_B(m, X, mask=False)
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th), 0.0], [np.sin(th), np.cos(th), 0.0], [0.0, 0.0, 1.0]])
    ax = np.array([1.0, 2.0, -1.0]) / np.sqrt(6.0)
    K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
    R = (np.eye(3) + np.sin(0.4) * K + (1 - np.cos(0.4)) * K @ K) @ R
    XR = X @ R.T + np.array([0.3, -1.0, 2.0])
    AR = mp.assemble_A(m, XR, mu, mask=False)
    BR = mp.assemble_B(m, XR, mask=False)
    u = np.random.default_rng(7).standard_normal((m.n_nodes, 3))
    uR = u @ R.T
    uv, uRv = u.T.ravel(), uR.T.ravel()
    assert abs(uRv @ (AR @ uRv) - uv @ (A @ uv)) < 1e-12 * abs(uv @ (A @ uv))
    assert relmax(BR @ uRv, B @ uv) < 1e-12
    s = 2.5
    assert relmax(mp.assemble_A(m, s * X, mu, mask=False), s * A) < 1e-13
    assert relmax(mp.assemble_B(m, s * X, mask=False), s * s * B) < 1e-13


def test_inverted_element_is_rejected():
    m, X = mesh_and_coords("brick", n=(2, 2, 2))
    X = X.copy()
    centre = np.argmin(np.linalg.norm(X - np.array([0.5, 0.35, 0.65]), axis=1))
    X[centre] += np.array([0.9, 0.0, 0.0])         # past the neighbouring vertex: det J < 0
    with pytest.raises(ValueError):
        mp.geometry(m, X)


def test_mapped_solve_on_the_brick_is_the_brick_solve():
    m = Mesh(4, 4, 4, 2)
    X = m.node_coords()
    c = inputs.sinker_centres(0, 3)
    mu, f = wbfbt.sinker_problem(m, c, 0.2, 200.0, 1e3)
    u0, p0, it0, _, _ = wbfbt.solve(m, mu, f, rtol=1e-8)
    u1, p1, it1, _ = mp.solve(m, X, mu, f, rtol=1e-8)
    assert it0 == it1
    assert relmax(u1, u0) < 1e-10 and relmax(p1, p0) < 1e-8


def test_mapped_solve_converges_to_the_mapped_system():
    m = Mesh(4, 4, 4, 2)
    X = inputs.deform_vertices(m.node_coords(), (4, 4, 4), (1.0, 1.0, 1.0), 0.15, 2)
    c = inputs.sinker_centres(0, 3)
    mu = sinker.viscosity(X, c, 0.2, 200.0, 1e3)
    f = sinker.forcing(X, c, 0.2, 200.0)
    u, p, its, rel = mp.solve(m, X, mu, f, rtol=1e-8)
    S = mp.MappedStokes(m, X, mu)
    F = np.concatenate([mp.load_vector(m, X, f), np.zeros(m.n_p)])
    r = F - S.apply_K(np.concatenate([u, p]))
    assert np.linalg.norm(r) < 1e-7 * np.linalg.norm(F)
    assert its < 200


def test_fine_level_mapped_preconditioner_solves_the_same_system():
    """The preconditioner whose finest level is the mapped mesh's converges to the same solution of
    the mapped system as the brick's, in no more iterations on a distorted mesh (it only changes
    the preconditioner, not the system)."""
    m = Mesh(8, 8, 8, 2)
    X = inputs.deform_vertices(m.node_coords(), (8, 8, 8), (1.0, 1.0, 1.0), 0.15, 7)
    c = inputs.sinker_centres(0, 4)
    mu = sinker.viscosity(X, c, 0.1, 200.0, 1e4)
    f = sinker.forcing(X, c, 0.1, 200.0)
    u0, p0, it0, _ = mp.solve(m, X, mu, f, rtol=1e-9)
    u1, p1, it1, _ = mp.solve(m, X, mu, f, rtol=1e-9, preconditioner="mapped_fine")
    assert it1 <= it0
    assert relmax(u1, u0) < 1e-6 and relmax(p1, p0) < 1e-5
