"""GPU parity of the single-kernel FP32 Q2 A apply (element arithmetic of Sec. 1.2 with the node
sums formed on chip and a fix-up pass over tile-surface nodes), on levels large enough to take it.

The shapes have a short last 32-element segment along x and, where the layer count does not
divide, a short last chunk along z, so the sampled nodes include tile seams, edges and corners
(every shape must also coarsen to a small dense level, which rules out a short last 4-row tile
along y: the index arithmetic of that case is checked on the host by a model of the kernels).  References: the oracle's element-local sums at sampled nodes (2e-5 relative, the
FP32 bound used elsewhere), the two-pass row kernels of the same context type on the full vector
(same element arithmetic, another summation order: 1e-6), and for the in-place epilogues of the
Chebyshev smoother the FP64 V-cycle (1e-4, as for every FP32 V-cycle).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mesh as M
from oracle import operators as op
from oracle import sinker
from paper_1607_03936_gb300 import inputs

pytestmark = pytest.mark.gpu

ELEM_AUTO, ELEM_ROW = 0, 2
SHAPES = [(80, 64, 32), (48, 48, 64), (64, 64, 40)]


@pytest.fixture(scope="module")
def wb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1607_03936_gb300 import build
    build.build()
    from paper_1607_03936_gb300 import wbfbt
    return wbfbt


def N(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def setup(wb, shape, restart=5, **kw):
    nx, ny, nz = shape
    m = M.Mesh(nx, ny, nz, 2, 1.0, ny / nx, nz / nx)
    c = inputs.sinker_centres(3, 6)
    mu = sinker.viscosity(m.node_coords(), c, 0.1, 200.0, 1e6)
    mu_t = torch.tensor(mu, device="cuda")
    s = wb.Solver(nx, 2, mu_t, ny=ny, nz=nz, lengths=(1.0, ny / nx, nz / nx), precision=wb.MIXED, restart=restart, **kw)
    return m, mu, s


def seam_nodes(m, rng):
    """Random nodes plus every node of small boxes around tile seams and the domain's edges."""
    xs = [0, 1, 63, 64, 65, m.NX - 2, m.NX - 1]
    ys = [0, 7, 8, 9, m.NY - 2, m.NY - 1]
    zs = [0, 1, 2, 3, 4, 5, m.NZ // 2, m.NZ // 2 + 1, m.NZ - 3, m.NZ - 2, m.NZ - 1]
    box = [x + m.NX * (y + m.NY * z) for z in zs for y in ys for x in xs if x < m.NX and y < m.NY]
    return np.unique(np.concatenate([rng.choice(m.n_nodes, 200, replace=False), np.array(box)]))


@pytest.mark.parametrize("shape", SHAPES)
def test_fused_A_apply_matches_oracle_and_two_pass(wb, shape):
    m, mu, s = setup(wb, shape)
    _, _, s_row = setup(wb, shape, elem_kernels=ELEM_ROW)
    rng = np.random.default_rng(sum(shape))
    u = rng.standard_normal(m.n_u).astype(np.float32)
    ut = torch.tensor(u, device="cuda")
    y = N(s.apply_A(ut))
    y_row = N(s_row.apply_A(ut))
    assert rel(y, y_row) < 1e-6
    nodes = seam_nodes(m, rng)
    ref = op.sampled_apply_A(m, mu, u.astype(np.float64), nodes)
    got = y.reshape(3, -1)[:, nodes].T
    assert np.abs(got - ref).max() / np.abs(ref).max() < 2e-5
    # bitwise reproducible: a second apply gives the same bits
    assert np.array_equal(N(s.apply_A(ut)), y)


@pytest.mark.parametrize("shape", SHAPES[:2])
def test_fused_A_vcycle_matches_fp64(wb, shape):
    """The A V-cycle's fine-level Chebyshev steps (in-place epilogues on the fused path) against the
    FP64 V-cycle of the same problem, and against the two-pass FP32 V-cycle."""
    m, mu, s = setup(wb, shape)
    _, _, s_row = setup(wb, shape, elem_kernels=ELEM_ROW)
    nx, ny, nz = shape
    s64 = wb.Solver(nx, 2, torch.tensor(mu, device="cuda"), ny=ny, nz=nz, lengths=(1.0, ny / nx, nz / nx),
                    restart=5)
    r = np.random.default_rng(5).standard_normal(m.n_u)
    bmask = np.tile(m.boundary_node_mask(), 3)
    r[bmask] = 0.0
    z64 = N(s64.apply_Ainv(torch.tensor(r, device="cuda")))
    r32 = torch.tensor(r, dtype=torch.float32, device="cuda")
    z = N(s.apply_Ainv(r32))
    z_row = N(s_row.apply_Ainv(r32))
    assert rel(z, z64) < 1e-4
    assert rel(z, z_row) < 1e-4


def test_fused_mixed_solve_matches_two_pass(wb):
    """A mixed-precision Stokes solve whose fine level takes the fused apply against the same solve
    on the two-pass row kernels: same iteration count within one, solutions within the solve
    tolerance."""
    shape = (48, 48, 64)
    m, mu, s = setup(wb, shape, restart=50)
    _, _, s_row = setup(wb, shape, restart=50, elem_kernels=ELEM_ROW)
    f = sinker.forcing(m.node_coords(), inputs.sinker_centres(3, 6), 0.1, 200.0)
    ft = torch.tensor(f.T.ravel(), device="cuda")
    u, p, res = s.solve(ft, rtol=1e-6)
    u2, p2, res2 = s_row.solve(ft, rtol=1e-6)
    assert res.status == 0 and res2.status == 0
    assert abs(res.iters - res2.iters) <= 1, (res.iters, res2.iters)
    assert rel(N(u), N(u2)) < 1e-5


@pytest.mark.parametrize("shape", SHAPES[:2])
def test_fused_BT_and_Kw_match_two_pass(wb, shape):
    """B^T p (the fused gradient pass), B u and K_w p = B C^-1 B^T p against the two-pass row
    kernels; the K_w V-cycle (fused K_w and Poisson
    smoothing steps) against FP64 and the two-pass V-cycle."""
    m, mu, s = setup(wb, shape)
    _, _, s_row = setup(wb, shape, elem_kernels=ELEM_ROW)
    rng = np.random.default_rng(7)
    p = torch.tensor(rng.standard_normal(m.n_p), dtype=torch.float32, device="cuda")
    assert rel(N(s.apply_BT(p)), N(s_row.apply_BT(p))) < 1e-6
    # B u (the element-local pass both contexts share) on the same shapes
    u = torch.tensor(rng.standard_normal(m.n_u), dtype=torch.float32, device="cuda")
    assert rel(N(s.apply_B(u)), N(s_row.apply_B(u))) < 1e-6
    for which in (0, 1):
        assert rel(N(s.apply_Kw(which, p)), N(s_row.apply_Kw(which, p))) < 1e-5
    nx, ny, nz = shape
    s64 = wb.Solver(nx, 2, torch.tensor(mu, device="cuda"), ny=ny, nz=nz, lengths=(1.0, ny / nx, nz / nx),
                    restart=5)
    r = op.project_pressure(m, rng.standard_normal(m.n_p))
    z64 = N(s64.apply_Kinv(1, torch.tensor(r, device="cuda")))
    r32 = torch.tensor(r, dtype=torch.float32, device="cuda")
    z = N(s.apply_Kinv(1, r32))   # fused B^T and fused Poisson smoothing on the fine levels
    assert rel(z, z64) < 1e-4
    assert rel(z, N(s_row.apply_Kinv(1, r32))) < 1e-4


@pytest.mark.parametrize("shape", SHAPES[:2])
def test_tiled_transfers_fp64_match_per_node(wb, shape):
    """The tiled Q2 restriction and prolongation (coarse grids of >= 100000 nodes under the automatic
    kernel choice) against the per-node kernels, through FP64 V-cycles of both hierarchies: the two
    differ only in summation order."""
    nx, ny, nz = shape
    m = M.Mesh(nx, ny, nz, 2, 1.0, ny / nx, nz / nx)
    mu = sinker.viscosity(m.node_coords(), inputs.sinker_centres(3, 6), 0.1, 200.0, 1e6)
    kw = dict(ny=ny, nz=nz, lengths=(1.0, ny / nx, nz / nx), restart=5)
    s = wb.Solver(nx, 2, torch.tensor(mu, device="cuda"), **kw)
    s_row = wb.Solver(nx, 2, torch.tensor(mu, device="cuda"), elem_kernels=ELEM_ROW, **kw)
    rng = np.random.default_rng(11)
    r = rng.standard_normal(m.n_u)
    r[np.tile(m.boundary_node_mask(), 3)] = 0.0
    rt = torch.tensor(r, device="cuda")
    assert rel(N(s.apply_Ainv(rt)), N(s_row.apply_Ainv(rt))) < 1e-11
    q = torch.tensor(op.project_pressure(m, rng.standard_normal(m.n_p)), device="cuda")
    for which in (0, 1):
        assert rel(N(s.apply_Kinv(which, q)), N(s_row.apply_Kinv(which, q))) < 1e-11


def test_fused_apply_on_a_coarse_level_128cubed(wb):
    """128^3 Q2 (the paper's level-7 size): the second level of the viscous hierarchy (64^3) also
    takes the single-kernel A apply, there with the viscosity per element point; the FP32 A and
    K_w V-cycles against the two-pass kernels (1e-4, as for every FP32 V-cycle)."""
    cfg = inputs.WORKLOADS["128^3-Q2-S16-DR1e6"]
    n, k = cfg["n"], cfg["k"]
    c = inputs.sinker_centres(cfg["seed"], cfg["n_sinkers"])
    mu, _ = wb.sinker_setup(n, k, c, cfg["omega"], cfg["delta"], cfg["dr"])
    s = wb.Solver(n, k, mu, precision=wb.MIXED, restart=5)
    rng = torch.Generator(device="cuda").manual_seed(4)
    r = torch.randn(s.n_u, device="cuda", generator=rng).float()
    q = torch.randn(s.n_p, device="cuda", generator=rng).float()
    z = N(s.apply_Ainv(r))
    zk = N(s.apply_Kinv(1, q))
    s.close()
    s_row = wb.Solver(n, k, mu, precision=wb.MIXED, restart=5, elem_kernels=ELEM_ROW)
    assert rel(z, N(s_row.apply_Ainv(r))) < 1e-4
    assert rel(zk, N(s_row.apply_Kinv(1, q))) < 1e-4
    s_row.close()
