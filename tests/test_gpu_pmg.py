"""p-coarsened multigrid for the viscous block (Sec. 6, Fig. 5: Q_k -> Q1 on the same mesh, then Q1
h-levels) through the C ABI against the oracle: one V-cycle (FP64 1e-10, FP32 1e-4), the A block
alone and the Stokes solve (iterations +-1, solution 1e-10)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import krylov
from oracle import mesh as M
from oracle import multigrid as mg
from oracle import operators as op
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
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def N(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def problem(n, k, dr=1e4, ns=4, lengths=(1.0, 1.0, 1.0), ny=None, nz=None):
    m = M.Mesh(n, ny or n, nz or n, k, *lengths)
    c = inputs.sinker_centres(1, ns)
    mu, f = W.sinker_problem(m, c, 0.1, 200.0, dr)
    return m, mu, f


@pytest.mark.parametrize("shape", [(8, 2, (1.0, 1.0, 1.0), None, None), (8, 3, (1.0, 1.0, 1.0), None, None),
                                   (16, 2, (1.0, 0.75, 1.25), 12, 8)])
def test_pmg_vcycle_matches_oracle(wb, shape):
    n, k, L, ny, nz = shape
    m, mu, _ = problem(n, k, lengths=L, ny=ny, nz=nz)
    levels = mg.build_hierarchy(m, op.point_values(m, mu), vector=True, pmg=True)
    b = np.random.default_rng(3).standard_normal(m.n_u) * m.interior_dof_mask()
    ref = mg.vcycle(levels, b)
    mu_t = torch.tensor(mu, device="cuda")
    s64 = wb.Solver(n, k, mu_t, ny=ny, nz=nz, lengths=L, pmg=True)
    assert rel(N(s64.apply_Ainv(torch.tensor(b, device="cuda"))), ref) < 1e-10
    s32 = wb.Solver(n, k, mu_t, ny=ny, nz=nz, lengths=L, pmg=True, precision=wb.MIXED)
    assert rel(N(s32.apply_Ainv(torch.tensor(b, dtype=torch.float32, device="cuda"))), ref) < 1e-4


def test_pmg_A_alone_and_solve_match_oracle(wb):
    m, mu, f = problem(8, 2)
    prob = W.StokesProblem(m, mu)
    levels = mg.build_hierarchy(m, op.point_values(m, mu), vector=True, pmg=True)
    b = op.load_vector(m, f)
    xo, its, _ = krylov.fgmres(lambda x: prob.A @ x, lambda v: mg.vcycle(levels, v), b, rtol=1e-8)
    s = wb.Solver(8, 2, torch.tensor(mu, device="cuda"), pmg=True)
    x, res = s.solve_block(wb.BLOCK_A, torch.tensor(b, device="cuda"), rtol=1e-8)
    assert res.status == 0 and abs(res.iters - its) <= 1, (res.iters, its)
    assert rel(N(x), xo) < 1e-10
    uo, po, its, _, _ = W.solve(m, mu, f, W.Options(pmg=True))
    u, p, res = s.solve(torch.tensor(f.T.ravel(), device="cuda"))
    assert res.status == 0 and abs(res.iters - its) <= 1, (res.iters, its)
    assert rel(N(u), uo) < 1e-10 and rel(N(p), po) < 1e-10
