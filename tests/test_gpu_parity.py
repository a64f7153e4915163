"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Tolerances: FP64 kernels 1e-12 relative (sum-factorised vs assembled CSR, so
only summation order differs); FP32 kernels 2e-5 relative; composite FP64
preconditioner pieces 1e-10; FP64 solves: iterations within +-1 and solution
relative L2 difference <= 1e-10.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import krylov
from oracle import mesh as M
from oracle import multigrid as mg
from oracle import operators as op
from oracle import sinker
from oracle import wbfbt as W
from paper_1607_03936_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1607_03936_gb300 import build
    build.build()
    from paper_1607_03936_gb300 import wbfbt
    return wbfbt


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def problem(nx, ny, nz, k, dr=1e4, ns=4, seed=0, lengths=(1.0, 1.0, 1.0), omega=0.1, delta=200.0):
    m = M.Mesh(nx, ny, nz, k, *lengths)
    c = inputs.sinker_centres(seed, ns)
    X = m.node_coords()
    mu = sinker.viscosity(X, c, omega, delta, dr)
    f = sinker.forcing(X, c, omega, delta)
    return m, mu, f, c


def gpu_solver(wb, m, mu, **kw):
    mu_t = torch.tensor(mu, dtype=torch.float64, device="cuda")
    return wb.Solver(m.nx, m.k, mu_t, ny=m.ny, nz=m.nz, lengths=(m.lx, m.ly, m.lz), **kw)


def T(x, dtype=torch.float64):
    return torch.tensor(np.asarray(x), dtype=dtype, device="cuda")


def N(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


SHAPES = [(5, 4, 3, 2, (1.0, 0.7, 1.3)), (3, 2, 2, 3, (1.0, 1.0, 1.0)), (1, 1, 1, 2, (1.0, 1.0, 1.0)),
          (2, 3, 1, 4, (0.5, 1.0, 2.0))]


# Isotropic meshes (equal h, exact in binary) with one or several row segments along x, the last
# one short: the FP64 row kernel takes its isotropic form there, the general one on SHAPES.
SHAPES_ISO = [(33, 3, 2, 2, (8.25, 0.75, 0.5)), (6, 5, 4, 2, (1.5, 1.25, 1.0)), (67, 2, 1, 2, (33.5, 1.0, 0.5))]


@pytest.mark.parametrize("kern", [1, 2])
@pytest.mark.parametrize("shape", SHAPES + SHAPES_ISO)
def test_fine_operators_fp64(wb, shape, kern):
    """kern 1: per-point element passes; kern 2: at k = 2 the row-segment passes (warp per point)."""
    nx, ny, nz, k, L = shape
    m, mu, _, _ = problem(nx, ny, nz, k, lengths=L)
    s = gpu_solver(wb, m, mu, elem_kernels=kern)
    rng = np.random.default_rng(1)
    u, p = rng.standard_normal(m.n_u), rng.standard_normal(m.n_p)
    A = op.assemble_A(m, op.point_values(m, mu))
    B = op.assemble_B(m)
    assert rel(N(s.apply_A(T(u))), A @ u) < 1e-12
    assert rel(N(s.apply_B(T(u))), B @ u) < 1e-12
    assert rel(N(s.apply_BT(T(p))), B.T @ p) < 1e-12
    x = np.concatenate([u, p])
    K = np.concatenate([A @ u + B.T @ p, B @ u])
    assert rel(N(s.apply_K(T(x))), K) < 1e-12


# FP32 shapes: single row segments, nx > 32 (two segments along x, the second one short) and
# nx = 64 + 3, so segment seams and ragged segments are covered by the row kernels.
SHAPES_F32 = SHAPES[:2] + [(33, 3, 2, 2, (1.0, 1.0, 1.0)), (6, 5, 4, 2, (1.0, 0.8, 1.2)), (67, 2, 1, 2, (1.0, 1.0, 1.0)),
                          (4, 3, 5, 3, (1.0, 1.0, 1.0))]


@pytest.mark.parametrize("kern", [1, 2])
@pytest.mark.parametrize("shape", SHAPES_F32)
def test_fine_operators_fp32(wb, shape, kern):
    nx, ny, nz, k, L = shape
    m, mu, _, _ = problem(nx, ny, nz, k, lengths=L)
    s = gpu_solver(wb, m, mu, elem_kernels=kern)
    rng = np.random.default_rng(2)
    u, p = rng.standard_normal(m.n_u), rng.standard_normal(m.n_p)
    A = op.assemble_A(m, op.point_values(m, mu))
    B = op.assemble_B(m)
    f32 = torch.float32
    assert rel(N(s.apply_A(T(u, f32))), A @ u) < 2e-5
    assert rel(N(s.apply_B(T(u, f32))), B @ u) < 2e-5
    assert rel(N(s.apply_BT(T(p, f32))), B.T @ p) < 2e-5


@pytest.mark.parametrize("kern", [1, 2])
@pytest.mark.parametrize("which", [0, 1])
def test_Kw_fp32(wb, which, kern):
    m, mu, _, _ = problem(6, 5, 4, 2, dr=1e6)
    s = gpu_solver(wb, m, mu, a_r=3.0, precision=wb.MIXED, elem_kernels=kern)
    prob = W.StokesProblem(m, mu, a_l=1.0, a_r=3.0)
    K = op.assemble_Kw(prob.B, prob.Cdiag if which == 0 else prob.Ddiag, m)
    p = np.random.default_rng(4).standard_normal(m.n_p)
    assert rel(N(s.apply_Kw(which, T(p, torch.float32))), K @ p) < 5e-5


@pytest.mark.parametrize("kern", [1, 2])
def test_vcycle_A_fp32(wb, kern):
    """FP32 V-cycle (FP64 coarsest solve) against the FP64 oracle V-cycle: 8^3 -> 4^3."""
    m, mu, _, _ = problem(8, 8, 8, 2, dr=1e4)
    s = gpu_solver(wb, m, mu, precision=wb.MIXED, elem_kernels=kern)
    levels = mg.build_hierarchy(m, op.point_values(m, mu), vector=True)
    b = np.random.default_rng(5).standard_normal(m.n_u) * m.interior_dof_mask()
    assert rel(N(s.apply_Ainv(T(b, torch.float32))), mg.vcycle(levels, b)) < 1e-4


@pytest.mark.parametrize("kern", [1, 2])
@pytest.mark.parametrize("which", [0, 1])
def test_pressure_poisson_vcycle_fp32(wb, which, kern):
    m, mu, _, _ = problem(8, 8, 8, 2, dr=1e6, ns=8)
    s = gpu_solver(wb, m, mu, a_r=2.0, precision=wb.MIXED, elem_kernels=kern)
    prob = W.StokesProblem(m, mu, a_l=1.0, a_r=2.0)
    pp = mg.PressurePoissonMG(m, prob.B, prob.Cdiag if which == 0 else prob.Ddiag, mu,
                              1.0 if which == 0 else 2.0)
    b = op.project_pressure(m, np.random.default_rng(6).standard_normal(m.n_p))
    assert rel(N(s.apply_Kinv(which, T(b, torch.float32))), pp.apply(b)) < 1e-4


@pytest.mark.parametrize("kern", [1, 2])
def test_fp32_applies_are_deterministic(wb, kern):
    m, mu, _, _ = problem(12, 10, 8, 2)
    s = gpu_solver(wb, m, mu, precision=wb.MIXED, elem_kernels=kern)
    rng = np.random.default_rng(11)
    u, p = T(rng.standard_normal(m.n_u), torch.float32), T(rng.standard_normal(m.n_p), torch.float32)
    assert torch.equal(s.apply_A(u), s.apply_A(u))
    assert torch.equal(s.apply_Kinv(1, p), s.apply_Kinv(1, p))


def test_apply_is_deterministic(wb):
    m, mu, _, _ = problem(6, 6, 6, 2)
    s = gpu_solver(wb, m, mu)
    u = T(np.random.default_rng(3).standard_normal(m.n_u))
    a, b = s.apply_K(torch.cat([u, T(np.zeros(m.n_p))])), s.apply_K(torch.cat([u, T(np.zeros(m.n_p))]))
    assert torch.equal(a, b)


def test_sinker_setup_matches_oracle(wb):
    m = M.Mesh(6, 5, 4, 3)
    c = inputs.sinker_centres(3, 8)
    mu_g, f_g = wb.sinker_setup(6, 3, c, 0.05, 200.0, 1e6, ny=5, nz=4)
    X = m.node_coords()
    mu_o = sinker.viscosity(X, c, 0.05, 200.0, 1e6)
    f_o = sinker.forcing(X, c, 0.05, 200.0)
    assert rel(N(mu_g), mu_o) < 1e-14
    assert rel(N(f_g), f_o.T.ravel()) < 1e-14


@pytest.mark.parametrize("shape", [(4, 3, 5, 2), (3, 2, 4, 3)])
@pytest.mark.parametrize("which", [0, 1])
def test_Kw_fp64(wb, which, shape):
    """FP64 contexts apply K_w as an assembled 27-neighbour block stencil (k = 2, 3)."""
    m, mu, _, _ = problem(*shape, dr=1e6)
    s = gpu_solver(wb, m, mu, a_r=3.0)
    prob = W.StokesProblem(m, mu, a_l=1.0, a_r=3.0)
    K = op.assemble_Kw(prob.B, prob.Cdiag if which == 0 else prob.Ddiag, m)
    p = np.random.default_rng(4).standard_normal(m.n_p)
    assert rel(N(s.apply_Kw(which, T(p))), K @ p) < 1e-12


@pytest.mark.parametrize("kern", [1, 2])
@pytest.mark.parametrize("n,k", [(8, 2), (6, 3), (3, 2)])
def test_vcycle_A_fp64(wb, n, k, kern):
    """kern 2 forces the row-segment Stokes passes on every level (nodal and per-point viscosity)."""
    m, mu, _, _ = problem(n, n, n, k, dr=1e4)
    s = gpu_solver(wb, m, mu, elem_kernels=kern)
    levels = mg.build_hierarchy(m, op.point_values(m, mu), vector=True)
    assert len(levels) == s.n_levels
    b = np.random.default_rng(5).standard_normal(m.n_u) * m.interior_dof_mask()
    assert rel(N(s.apply_Ainv(T(b))), mg.vcycle(levels, b)) < 1e-10


@pytest.mark.parametrize("kern", [1, 2])
@pytest.mark.parametrize("which", [0, 1])
def test_pressure_poisson_vcycle_fp64(wb, which, kern):
    """kern 2 forces the row kernels of the scalar Poisson levels and transfers (FP64 too)."""
    m, mu, _, _ = problem(8, 8, 8, 2, dr=1e6, ns=8)
    s = gpu_solver(wb, m, mu, a_r=2.0, elem_kernels=kern)
    prob = W.StokesProblem(m, mu, a_l=1.0, a_r=2.0)
    pp = mg.PressurePoissonMG(m, prob.B, prob.Cdiag if which == 0 else prob.Ddiag, mu,
                              1.0 if which == 0 else 2.0)
    b = op.project_pressure(m, np.random.default_rng(6).standard_normal(m.n_p))
    assert rel(N(s.apply_Kinv(which, T(b))), pp.apply(b)) < 1e-10


@pytest.mark.parametrize("lengths", [(1.0, 0.5, 1.0), (1.0, 1.0, 1.0)])
def test_flat_fp64_passes(wb, lengths):
    """A fine level of 2048 elements (16 x 8 x 16) takes the flat FP64 passes (32 consecutive
    elements per block, element-major scratch) for A and the Q2 Poisson level; isotropic
    (h = 1/16) and anisotropic meshes; A, the A V-cycle and both pressure-Poisson V-cycles."""
    m, mu, _, _ = problem(16, 8, 16, 2, dr=1e4, lengths=lengths)
    s = gpu_solver(wb, m, mu, a_r=2.0)
    rng = np.random.default_rng(13)
    u = rng.standard_normal(m.n_u)
    A = op.assemble_A(m, op.point_values(m, mu))
    assert rel(N(s.apply_A(T(u))), A @ u) < 1e-12
    levels = mg.build_hierarchy(m, op.point_values(m, mu), vector=True)
    b = u * m.interior_dof_mask()
    assert rel(N(s.apply_Ainv(T(b))), mg.vcycle(levels, b)) < 1e-10
    prob = W.StokesProblem(m, mu, a_l=1.0, a_r=2.0)
    for which in (0, 1):
        pp = mg.PressurePoissonMG(m, prob.B, prob.Cdiag if which == 0 else prob.Ddiag, mu,
                                  1.0 if which == 0 else 2.0)
        bp = op.project_pressure(m, rng.standard_normal(m.n_p))
        assert rel(N(s.apply_Kinv(which, T(bp))), pp.apply(bp)) < 1e-10


def test_schur_inverse_and_block_preconditioner_fp64(wb):
    m, mu, _, _ = problem(8, 8, 8, 2, dr=1e4)
    s = gpu_solver(wb, m, mu)
    prob = W.StokesProblem(m, mu)
    pc = W.BlockPreconditioner(prob, mode="vcycle", schur_sign=-1.0)
    rng = np.random.default_rng(7)
    r = rng.standard_normal(m.n_p)
    assert rel(N(s.apply_schur_inv(T(r))), pc.S_inv(r)) < 1e-10
    x = np.concatenate([rng.standard_normal(m.n_u) * m.interior_dof_mask(), rng.standard_normal(m.n_p)])
    assert rel(N(s.apply_precond(T(x))), pc.apply(x)) < 1e-10


@pytest.mark.parametrize("n,k,dr,ns", [(8, 2, 1e4, 4), (6, 3, 1e6, 8)])
def test_solve_fp64_matches_oracle(wb, n, k, dr, ns):
    m, mu, f, _ = problem(n, n, n, k, dr=dr, ns=ns)
    s = gpu_solver(wb, m, mu)
    u, p, res = s.solve(T(f.T.ravel()))
    uo, po, its, relo, _ = W.solve(m, mu, f)
    assert res.status == 0 and res.rel_res <= 1e-6
    assert abs(res.iters - its) <= 1, (res.iters, its)
    assert rel(N(u), uo) < 1e-10
    assert rel(N(p), po) < 1e-10


def test_solve_fp64_row_kernels_matches_oracle(wb):
    """FP64 solve with the row-segment kernels (scalar and Stokes) forced on every level."""
    m, mu, f, _ = problem(8, 8, 8, 2, dr=1e4, ns=4)
    s = gpu_solver(wb, m, mu, elem_kernels=2)
    u, p, res = s.solve(T(f.T.ravel()))
    uo, po, its, relo, _ = W.solve(m, mu, f)
    assert res.status == 0 and abs(res.iters - its) <= 1, (res.iters, its)
    assert rel(N(u), uo) < 1e-10
    assert rel(N(p), po) < 1e-10


def test_solve_with_host_buffers(wb):
    m, mu, f, _ = problem(4, 4, 4, 2)
    s = gpu_solver(wb, m, mu)
    fh = torch.tensor(f.T.ravel(), dtype=torch.float64).pin_memory()
    uh = torch.empty(m.n_u, dtype=torch.float64).pin_memory()
    ph = torch.empty(m.n_p, dtype=torch.float64).pin_memory()
    u1, p1, r1 = s.solve(fh, u=uh, p=ph)
    u2, p2, r2 = s.solve(T(f.T.ravel()))
    assert r1.iters == r2.iters
    assert np.array_equal(u1.numpy(), N(u2)) and np.array_equal(p1.numpy(), N(p2))


def test_mixed_precision_solve(wb):
    m, mu, f, _ = problem(8, 8, 8, 2, dr=1e6, ns=8)
    s64 = gpu_solver(wb, m, mu)
    s32 = gpu_solver(wb, m, mu, precision=wb.MIXED)
    u64, p64, r64 = s64.solve(T(f.T.ravel()), rtol=1e-8)
    u32, p32, r32 = s32.solve(T(f.T.ravel()), rtol=1e-8)
    assert r32.status == 0 and r32.rel_res <= 1e-8
    assert abs(r32.iters - r64.iters) <= 3
    assert rel(N(u32), N(u64)) < 1e-6


def test_invalid_arguments_rejected(wb):
    m, mu, _, _ = problem(2, 2, 2, 2)
    bad = mu.copy()
    bad[3] = -1.0
    with pytest.raises(wb.WbfbtError):
        gpu_solver(wb, m, bad)
    with pytest.raises(wb.WbfbtError):
        wb.Solver(2, 7, T(mu))
    s = gpu_solver(wb, m, mu)
    with pytest.raises(wb.WbfbtError):
        s.apply_schur_inv(T(np.zeros(m.n_p), torch.float32))   # FP64 context, FP32 request


def test_full_size_sampled_A_apply(wb):
    """32^3 Q2 (the bench workload size): A u at sampled nodes against element-local oracle sums."""
    cfg = inputs.WORKLOADS["32^3-Q2-S24-DR1e6"]
    n, k = cfg["n"], cfg["k"]
    c = inputs.sinker_centres(cfg["seed"], cfg["n_sinkers"])
    mu_g, f_g = wb.sinker_setup(n, k, c, cfg["omega"], cfg["delta"], cfg["dr"])
    s = wb.Solver(n, k, mu_g)
    m = M.Mesh(n, n, n, k)
    mu = N(mu_g)
    u = np.random.default_rng(8).standard_normal(m.n_u)
    y = N(s.apply_A(T(u))).reshape(3, -1)
    nodes = np.random.default_rng(9).choice(m.n_nodes, 200, replace=False)
    ref = op.sampled_apply_A(m, mu, u, nodes)
    err = np.abs(y[:, nodes].T - ref).max() / np.abs(ref).max()
    assert err < 1e-12


def test_full_size_sampled_A_apply_fp32(wb):
    """32^3 Q2 in FP32 with the default kernel choice (row segments on this level): sampled nodes."""
    cfg = inputs.WORKLOADS["32^3-Q2-S24-DR1e6"]
    n, k = cfg["n"], cfg["k"]
    c = inputs.sinker_centres(cfg["seed"], cfg["n_sinkers"])
    mu_g, _ = wb.sinker_setup(n, k, c, cfg["omega"], cfg["delta"], cfg["dr"])
    s = wb.Solver(n, k, mu_g, precision=wb.MIXED)
    m = M.Mesh(n, n, n, k)
    mu = N(mu_g)
    u = np.random.default_rng(8).standard_normal(m.n_u)
    y = N(s.apply_A(T(u, torch.float32))).reshape(3, -1)
    nodes = np.random.default_rng(9).choice(m.n_nodes, 200, replace=False)
    ref = op.sampled_apply_A(m, mu, u.astype(np.float32).astype(np.float64), nodes)
    err = np.abs(y[:, nodes].T - ref).max() / np.abs(ref).max()
    assert err < 2e-5


def test_full_size_64cubed_sampled_A_apply_fp32(wb):
    """64^3 Q2 (the largest configuration; two row segments along x) in FP32: sampled nodes."""
    cfg = inputs.WORKLOADS["64^3-Q2-S64-DR1e10"]
    n, k = cfg["n"], cfg["k"]
    c = inputs.sinker_centres(cfg["seed"], cfg["n_sinkers"])
    mu_g, _ = wb.sinker_setup(n, k, c, cfg["omega"], cfg["delta"], cfg["dr"])
    s = wb.Solver(n, k, mu_g, precision=wb.MIXED, restart=5)
    m = M.Mesh(n, n, n, k)
    mu = N(mu_g)
    u = np.random.default_rng(10).standard_normal(m.n_u)
    y = N(s.apply_A(T(u, torch.float32))).reshape(3, -1)
    rng = np.random.default_rng(11)
    nodes = np.concatenate([rng.choice(m.n_nodes, 150, replace=False),
                            # nodes on the seam between the two x-segments (x index 64)
                            64 + m.NX * rng.integers(1, m.NY - 1, 50) + m.NX * m.NY * rng.integers(1, m.NZ - 1, 50)])
    ref = op.sampled_apply_A(m, mu, u.astype(np.float32).astype(np.float64), nodes)
    err = np.abs(y[:, nodes].T - ref).max() / np.abs(ref).max()
    assert err < 2e-5


def test_full_size_64cubed_sampled_K_apply_fp64(wb):
    """64^3 Q2 DR 1e10 in FP64 (the largest configuration, row-segment FP64 passes with two
    segments along x): the fused K apply (A + B^T, B) at sampled nodes and elements."""
    cfg = inputs.WORKLOADS["64^3-Q2-S64-DR1e10"]
    n, k = cfg["n"], cfg["k"]
    c = inputs.sinker_centres(cfg["seed"], cfg["n_sinkers"])
    mu_g, _ = wb.sinker_setup(n, k, c, cfg["omega"], cfg["delta"], cfg["dr"])
    s = wb.Solver(n, k, mu_g, restart=5)
    m = M.Mesh(n, n, n, k)
    mu = N(mu_g)
    rng = np.random.default_rng(12)
    u = rng.standard_normal(m.n_u)
    y = N(s.apply_A(T(u))).reshape(3, -1)
    nodes = np.concatenate([rng.choice(m.n_nodes, 150, replace=False),
                            64 + m.NX * rng.integers(1, m.NY - 1, 50) + m.NX * m.NY * rng.integers(1, m.NZ - 1, 50)])
    ref = op.sampled_apply_A(m, mu, u, nodes)
    err = np.abs(y[:, nodes].T - ref).max() / np.abs(ref).max()
    assert err < 1e-12
    # B on sampled elements: the element divergence matrix on the element's masked velocity
    yp = N(s.apply_B(T(u))).reshape(m.n_elem, m.Np)
    Be = op.element_B(m)
    bmask = m.boundary_node_mask()
    ids_all = m.point_to_node()
    elems = rng.choice(m.n_elem, 100, replace=False)
    refp = np.stack([Be @ np.concatenate([u[cc * m.n_nodes + ids_all[e]] * (~bmask[ids_all[e]]) for cc in range(3)])
                     for e in elems])
    assert np.abs(yp[elems] - refp).max() / np.abs(refp).max() < 1e-12


def test_q3_dr1e8_mixed_solve_matches_fp64(wb):
    """24^3 Q3, 32 sinkers, DR 1e8 (the mixed-precision configuration): mixed vs FP64 GPU solve."""
    cfg = inputs.WORKLOADS["24^3-Q3-S32-DR1e8"]
    n, k = cfg["n"], cfg["k"]
    c = inputs.sinker_centres(cfg["seed"], cfg["n_sinkers"])
    mu_g, f_g = wb.sinker_setup(n, k, c, cfg["omega"], cfg["delta"], cfg["dr"])
    u64, p64, r64 = wb.Solver(n, k, mu_g).solve(f_g)
    u32, p32, r32 = wb.Solver(n, k, mu_g, precision=wb.MIXED).solve(f_g)
    assert r64.status == 0 and r32.status == 0
    assert abs(r32.iters - r64.iters) <= 3, (r32.iters, r64.iters)
    assert rel(N(u32), N(u64)) < 1e-6
    assert rel(N(p32), N(p64)) < 1e-6


def test_mixed_solve_point_and_row_kernels_agree(wb):
    """The two single-precision kernel families (per point, per element) agree up to FP32 rounding."""
    m, mu, f, _ = problem(8, 8, 8, 2, dr=1e6, ns=8)
    fg = T(f.T.ravel())
    u1, p1, r1 = gpu_solver(wb, m, mu, precision=wb.MIXED, elem_kernels=1).solve(fg, rtol=1e-8)
    u2, p2, r2 = gpu_solver(wb, m, mu, precision=wb.MIXED, elem_kernels=2).solve(fg, rtol=1e-8)
    assert abs(r1.iters - r2.iters) <= 2
    assert rel(N(u1), N(u2)) < 1e-6


def test_graph_replay_matches_direct_launches(wb):
    """The CUDA-graph preconditioner replays exactly the launches of the direct path."""
    m, mu, f, _ = problem(8, 8, 8, 2, dr=1e6, ns=8)
    fg = T(f.T.ravel())
    u1, p1, r1 = gpu_solver(wb, m, mu, use_graphs=True).solve(fg)
    u2, p2, r2 = gpu_solver(wb, m, mu, use_graphs=False).solve(fg)
    assert r1.iters == r2.iters
    assert torch.equal(u1, u2) and torch.equal(p1, p2)


def test_resetup_reuses_memory_and_matches_fresh_context(wb):
    m, mu, f, _ = problem(8, 8, 8, 2, dr=1e4)
    _, mu2, _, _ = problem(8, 8, 8, 2, dr=1e6, ns=8, seed=3)
    s = gpu_solver(wb, m, mu)
    before = s.device_bytes
    s.setup(T(mu2))
    assert s.device_bytes == before
    u1, p1, r1 = s.solve(T(f.T.ravel()))
    u2, p2, r2 = gpu_solver(wb, m, mu2).solve(T(f.T.ravel()))
    assert r1.iters == r2.iters
    assert torch.equal(u1, u2) and torch.equal(p1, p2)
