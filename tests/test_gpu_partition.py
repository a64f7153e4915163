"""The slab partition's local applies on the CUDA path: each rank's sub-mesh (its slab plus two
ghost element layers per interior side) applied by the library gives, on the owned node planes and
element layers, exactly the global apply.  The ranks run one after the other on this GPU (their
kernels do not wait on each other); the ghost values come from the global vector, which is what
the halo exchange delivers (that exchange is tested on gloo ranks in test_partition_gloo.py)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

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


@pytest.mark.parametrize("nx,ny,nz,k,world,dtype", [(6, 5, 12, 2, 3, torch.float64), (6, 5, 12, 2, 3, torch.float32),
                                                      (4, 4, 8, 3, 2, torch.float64), (33, 2, 8, 2, 4, torch.float64)])
def test_partitioned_K_apply_on_the_gpu(wb, nx, ny, nz, k, world, dtype):
    from paper_1607_03936_gb300 import partition
    L = (1.0, 0.8, 1.6)
    c = inputs.sinker_centres(3, 6)
    mu, _ = wb.sinker_setup(nx, k, c, 0.1, 200.0, 1e4, ny=ny, nz=nz, lengths=L)
    prec = wb.MIXED if dtype == torch.float32 else wb.F64
    glob = wb.Solver(nx, k, mu, ny=ny, nz=nz, lengths=L, precision=prec)
    gen = torch.Generator(device="cuda").manual_seed(4)
    x = torch.randn(glob.n_u + glob.n_p, dtype=torch.float64, device="cuda", generator=gen)
    y = glob.apply_K(x.to(dtype))
    yu = y[: glob.n_u].reshape(3, k * nz + 1, -1)
    yp = y[glob.n_u:].reshape(nz, -1)
    npe = glob.np
    got_u, got_p = [], []
    for r in range(world):
        part = partition.SlabPartition(nx, ny, nz, k, world, r)
        u_loc = part.local_from_global(x[: glob.n_u], 3).to(dtype)
        p_loc = part.local_pressure_from_global(x[glob.n_u:], npe).to(dtype)
        mu_loc = part.local_from_global(mu, 1)
        apply = partition.library_local_apply(part, mu_loc, L, precision=prec)
        ou, op_ = apply(u_loc, p_loc)
        got_u.append(part.owned_nodes(ou, 3))
        got_p.append(part.owned_elements(op_, npe))
        apply.solver.close()
    gu, gp = torch.cat(got_u, dim=1), torch.cat(got_p, dim=0)
    tol = 1e-12 if dtype == torch.float64 else 2e-5
    assert (gu - yu).abs().max().item() <= tol * yu.abs().max().item()
    assert (gp - yp).abs().max().item() <= tol * yp.abs().max().item()


@pytest.mark.parametrize("nx,ny,nz,k,world", [(6, 5, 12, 2, 3), (4, 4, 8, 3, 2)])
def test_partitioned_mapped_K_apply_on_the_gpu(wb, nx, ny, nz, k, world):
    """The same on a mapped mesh (interior vertices moved, the sinker fields at the moved nodes):
    each rank's sub-mesh takes its local planes of the global coordinates."""
    from paper_1607_03936_gb300 import partition
    L = (1.0, 0.8, 1.6)
    X0 = wb.node_coords(nx, k, ny=ny, nz=nz, lengths=L).view(3, -1).T.cpu().numpy()
    Xh = inputs.deform_vertices(X0, (nx, ny, nz), L, 0.12, 5)
    X = torch.tensor(np.ascontiguousarray(Xh.T).ravel(), device="cuda")
    c = inputs.sinker_centres(3, 6)
    mu, _ = wb.sinker_setup_at(X, nx, k, c, 0.1, 200.0, 1e4, ny=ny, nz=nz, lengths=L)
    glob = wb.Solver(nx, k, mu, ny=ny, nz=nz, lengths=L)
    glob.set_geometry(X)
    gen = torch.Generator(device="cuda").manual_seed(6)
    x = torch.randn(glob.n_u + glob.n_p, dtype=torch.float64, device="cuda", generator=gen)
    y = glob.apply_K(x)
    yu = y[: glob.n_u].reshape(3, k * nz + 1, -1)
    yp = y[glob.n_u:].reshape(nz, -1)
    npe = glob.np
    got_u, got_p = [], []
    for r in range(world):
        part = partition.SlabPartition(nx, ny, nz, k, world, r)
        apply = partition.library_local_apply(part, part.local_from_global(mu, 1), L,
                                              X_loc=part.local_from_global(X, 3))
        ou, op_ = apply(part.local_from_global(x[: glob.n_u], 3), part.local_pressure_from_global(x[glob.n_u:], npe))
        got_u.append(part.owned_nodes(ou, 3))
        got_p.append(part.owned_elements(op_, npe))
        apply.solver.close()
    gu, gp = torch.cat(got_u, dim=1), torch.cat(got_p, dim=0)
    assert (gu - yu).abs().max().item() <= 1e-12 * yu.abs().max().item()
    assert (gp - yp).abs().max().item() <= 1e-12 * yp.abs().max().item()
