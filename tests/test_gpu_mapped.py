"""GPU parity of the mapped-hexahedron path (isoparametric Q_k geometry) against the oracle.

The CUDA element pass forms J = dx/dxi per point from the nodal coordinates and applies the forms
of Sec. 1.2 on the mapped element; the oracle assembles the same operators as CSR matrices with
J^-1 from a library inverse.  Tolerances as for the brick: FP64 applies 1e-12 relative, FP32 2e-5,
FP64 solves iterations within +-1 and solution within 1e-10.  Shapes leave a ragged last block of
elements, and one shape has more element batches than the launch's blocks (grid-stride loop).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mapped as mp
from oracle import mesh as M
from oracle import operators as op
from oracle import sinker
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


def T(x, dtype=torch.float64):
    return torch.tensor(np.asarray(x), dtype=dtype, device="cuda")


def N(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def mapped_problem(n, k, kind, lengths=(1.0, 1.0, 1.0), amp=None, dr=1e4, ns=4, seed=3):
    m = M.Mesh(*n, k, *lengths)
    X0 = m.node_coords()
    if kind == "trilinear":
        X = inputs.deform_vertices(X0, n, lengths, 0.15 if amp is None else amp, seed)
    elif kind == "smooth":
        X = inputs.deform_smooth(X0, lengths, 0.1 if amp is None else amp)
    else:
        X = X0
    c = inputs.sinker_centres(seed, ns)
    mu = sinker.viscosity(X, c, 0.1, 200.0, dr)
    f = sinker.forcing(X, c, 0.1, 200.0)
    return m, X, mu, f


def solver(wb, m, X, mu, **kw):
    s = wb.Solver(m.nx, m.k, T(mu), ny=m.ny, nz=m.nz, lengths=(m.lx, m.ly, m.lz), **kw)
    s.set_geometry(T(X.T.ravel()))
    return s


CASES = [((6, 5, 7), 2, "trilinear"), ((6, 5, 7), 2, "smooth"), ((4, 3, 5), 3, "trilinear"),
         ((3, 3, 2), 4, "smooth")]


@pytest.mark.parametrize("n,k,kind", CASES)
def test_mapped_applies_match_oracle(wb, n, k, kind):
    lengths = (1.0, 0.8, 1.2)
    m, X, mu, _ = mapped_problem(n, k, kind, lengths=lengths)
    s = solver(wb, m, X, mu)
    A = mp.assemble_A(m, X, op.point_values(m, mu))
    B = mp.assemble_B(m, X)
    rng = np.random.default_rng(sum(n) + k)
    u = rng.standard_normal(m.n_u)
    p = rng.standard_normal(m.n_p)
    assert rel(N(s.apply_A(T(u))), A @ u) < 1e-12
    assert rel(N(s.apply_B(T(u))), B @ u) < 1e-12
    assert rel(N(s.apply_BT(T(p))), B.T @ p) < 1e-12
    x = np.concatenate([u, p])
    yk = N(s.apply_K(T(x)))
    assert rel(yk[: m.n_u], A @ u + B.T @ p) < 1e-12
    assert rel(yk[m.n_u:], B @ u) < 1e-12
    # FP32 applies of the same context
    assert rel(N(s.apply_A(T(u, torch.float32))), A @ u) < 2e-5
    assert rel(N(s.apply_B(T(u, torch.float32))), B @ u) < 2e-5
    assert rel(N(s.apply_BT(T(p, torch.float32))), B.T @ p) < 2e-5


def patch_values(m, X, mu, u, p, vertex):
    """A u and B^T p at one interior element vertex from the oracle's mapped operators assembled on
    the 2 x 2 x 2 elements around it (every element that holds the node), with the velocity of the
    global mesh's Dirichlet nodes read as zero."""
    k = m.k
    pm = M.Mesh(2, 2, 2, k)
    lo = [k * (v - 1) for v in vertex]
    ii = np.arange(2 * k + 1)
    iz, iy, ix = np.meshgrid(ii + lo[2], ii + lo[1], ii + lo[0], indexing="ij")
    gn = (ix + m.NX * (iy + m.NY * iz)).ravel()          # global node of each patch node
    uu = u.reshape(3, -1)[:, gn] * (~m.boundary_node_mask()[gn])
    ez, ey, ex = np.meshgrid(np.arange(2) + vertex[2] - 1, np.arange(2) + vertex[1] - 1,
                             np.arange(2) + vertex[0] - 1, indexing="ij")
    ge = (ex + m.nx * (ey + m.ny * ez)).ravel()          # global element of each patch element
    pp = p.reshape(-1, m.Np)[ge].ravel()
    A = mp.assemble_A(pm, X[gn], op.point_values(pm, mu[gn]), mask=False)
    B = mp.assemble_B(pm, X[gn], mask=False)
    c = k + pm.NX * (k + pm.NY * k)                      # the patch's centre node
    ya, yb = (A @ uu.ravel()).reshape(3, -1), (B.T @ pp).reshape(3, -1)
    return ya[:, c], yb[:, c]


def test_mapped_applies_on_a_row_kernel_grid_sampled(wb):
    """32 x 32 x 24 Q2 elements: more element batches than the launch's blocks (the grid-stride
    loop), on a grid whose brick applies take the row-segment kernels.  A u and B^T p at sampled
    interior vertices (including the last elements) against the oracle's patch operators at 1e-12
    of the largest sampled entry; with the brick's own coordinates the mapped apply equals the
    brick's row kernels to 1e-13."""
    n = (32, 32, 24)
    m, X, mu, _ = mapped_problem(n, 2, "trilinear", amp=0.12)
    s = solver(wb, m, X, mu)
    rng = np.random.default_rng(11)
    u = rng.standard_normal(m.n_u)
    p = rng.standard_normal(m.n_p)
    ya = N(s.apply_A(T(u))).reshape(3, -1)
    yb = N(s.apply_BT(T(p))).reshape(3, -1)
    verts = [tuple(rng.integers(1, [n[0], n[1], n[2]])) for _ in range(24)]
    verts += [(n[0] - 1, n[1] - 1, n[2] - 1), (1, 1, 1), (n[0] - 1, 1, n[2] - 1), (1, n[1] - 1, n[2] - 1)]
    got_a, got_b, ref_a, ref_b = [], [], [], []
    for v in verts:
        node = 2 * v[0] + m.NX * (2 * v[1] + m.NY * 2 * v[2])
        ra, rb = patch_values(m, X, mu, u, p, v)
        got_a.append(ya[:, node]); got_b.append(yb[:, node]); ref_a.append(ra); ref_b.append(rb)
    got_a, got_b, ref_a, ref_b = map(np.array, (got_a, got_b, ref_a, ref_b))
    assert np.abs(got_a - ref_a).max() < 1e-12 * np.abs(ref_a).max()
    assert np.abs(got_b - ref_b).max() < 1e-12 * np.abs(ref_b).max()
    # the brick's coordinates through the mapped kernels against the brick's row kernels
    X0 = m.node_coords()
    s.set_geometry(T(X0.T.ravel()))
    y_mapped = N(s.apply_A(T(u)))
    s.set_geometry(None)
    assert rel(y_mapped, N(s.apply_A(T(u)))) < 1e-13


def test_brick_coordinates_reproduce_the_brick_and_none_restores_it(wb):
    m, X, mu, _ = mapped_problem((5, 4, 6), 2, "brick", lengths=(1.0, 0.7, 1.3))
    s = solver(wb, m, X, mu)
    rng = np.random.default_rng(2)
    u = T(rng.standard_normal(m.n_u))
    y_mapped = N(s.apply_A(u))
    s.set_geometry(None)
    y_brick = N(s.apply_A(u))
    assert rel(y_mapped, y_brick) < 1e-13


def test_inverted_geometry_is_rejected_and_the_brick_kept(wb):
    m, X, mu, _ = mapped_problem((2, 2, 2), 2, "brick")
    s = wb.Solver(2, 2, T(mu))
    u = T(np.random.default_rng(3).standard_normal(m.n_u))
    y0 = N(s.apply_A(u))
    Xb = X.copy()
    centre = np.argmin(np.linalg.norm(Xb - 0.5, axis=1))
    Xb[centre, 0] += 0.9                                   # past the neighbouring vertex: det J < 0
    with pytest.raises(wb.WbfbtError):
        s.set_geometry(T(Xb.T.ravel()))
    Xn = X.copy()
    Xn[centre, 1] = np.nan
    with pytest.raises(wb.WbfbtError):
        s.set_geometry(T(Xn.T.ravel()))
    assert np.array_equal(N(s.apply_A(u)), y0)


@pytest.mark.parametrize("kind,n,k", [("trilinear", 8, 2), ("smooth", 8, 2), ("smooth", 6, 3)])
def test_mapped_solve_fp64_matches_oracle(wb, kind, n, k):
    m, X, mu, f = mapped_problem((n, n, n), k, kind, dr=1e4, ns=4)
    s = solver(wb, m, X, mu)
    u, p, res = s.solve(T(f.T.ravel()))
    uo, po, its, relo = mp.solve(m, X, mu, f)
    assert res.status == 0 and res.rel_res <= 1e-6
    assert abs(res.iters - its) <= 1, (res.iters, its)
    assert rel(N(u), uo) < 1e-10
    assert rel(N(p), po) < 1e-10
    with pytest.raises(wb.WbfbtError):
        s.solve_block(wb.BLOCK_A, T(f.T.ravel()))


def test_mapped_solve_mixed_precision(wb):
    """FP32 preconditioner with the FP64 mapped Krylov operator, and with the FP32 mapped Arnoldi
    apply as well, against the oracle's FP64 solve: the FP64 true residual decides convergence
    (<= 1e-6); solutions within 1e-6 (FP64 Arnoldi) and 1e-5 (FP32 Arnoldi) of the oracle's, the
    bounds of the brick's mixed solves."""
    m, X, mu, f = mapped_problem((8, 8, 8), 2, "trilinear", dr=1e6, ns=8)
    uo, po, its, _ = mp.solve(m, X, mu, f)
    for arn in (wb.F64, wb.F32):
        s = solver(wb, m, X, mu, precision=wb.MIXED, arnoldi_precision=arn)
        u, p, res = s.solve(T(f.T.ravel()))
        assert res.status == 0 and res.rel_res <= 1e-6
        assert abs(res.iters - its) <= 3, (arn, res.iters, its)
        tol = 1e-6 if arn == wb.F64 else 1e-5
        assert rel(N(u), uo) < tol and rel(N(p), po) < tol


def test_setup_entry_points_reject_host_buffers(wb):
    """Host memory where device arrays are required is refused before any device work."""
    import ctypes
    lib = wb.lib()
    mesh = wb.Mesh(2, 2, 2, 1.0, 1.0, 1.0)
    host = torch.zeros(3 * 125, dtype=torch.float64)
    dev = torch.zeros(125, dtype=torch.float64, device="cuda")
    c = torch.tensor([[0.5, 0.5, 0.5]], dtype=torch.float64)
    assert lib.wbfbt_node_coords(ctypes.byref(mesh), 2, ctypes.c_void_p(host.data_ptr()), None) == -1
    assert lib.wbfbt_sinker_setup_at(ctypes.byref(mesh), 2, ctypes.c_void_p(host.data_ptr()),
                                     ctypes.c_void_p(c.data_ptr()), 1, 0.1, 200.0, 1e4, 10.0,
                                     ctypes.c_void_p(dev.data_ptr()), None, None) == -1


def test_node_coords_and_sinker_fields_at_mapped_nodes(wb):
    """The library's brick node positions against the oracle mesh's (k = 3: GLL nodes that are not
    evenly spaced), and the fields of Sec. 2.1 evaluated at moved nodes against the oracle's."""
    lengths = (1.0, 0.7, 1.3)
    m = M.Mesh(5, 4, 6, 3, *lengths)
    X0 = m.node_coords()
    Xg = N(wb.node_coords(5, 3, ny=4, nz=6, lengths=lengths))
    assert np.abs(Xg - X0.T.ravel()).max() < 1e-15
    X = inputs.deform_smooth(X0, lengths, 0.1)
    c = inputs.sinker_centres(4, 6)
    mu, f = wb.sinker_setup_at(T(X.T.ravel()), 5, 3, c, 0.1, 200.0, 1e6, ny=4, nz=6, lengths=lengths)
    assert rel(N(mu), sinker.viscosity(X, c, 0.1, 200.0, 1e6)) < 1e-14
    assert rel(N(f), sinker.forcing(X, c, 0.1, 200.0).T.ravel()) < 1e-14
