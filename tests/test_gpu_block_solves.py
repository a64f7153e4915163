"""The preconditioner's blocks solved on their own (the "alone" iteration counts of Table 3, Sec. 7)
through wbfbt_solve_block, against the oracle's FGMRES with the same V-cycles: iterations +-1 and
solution 1e-10 (FP64); the mixed-precision context converges to the same tolerance."""
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


@pytest.fixture(scope="module")
def case():
    m = M.Mesh(8, 8, 8, 2)
    c = inputs.sinker_centres(4, 8)
    mu, f = W.sinker_problem(m, c, 0.1, 200.0, 1e4)
    return m, mu, f


def test_A_alone_matches_oracle(wb, case):
    m, mu, f = case
    prob = W.StokesProblem(m, mu)
    levels = mg.build_hierarchy(m, op.point_values(m, mu), vector=True)
    b = op.load_vector(m, f)
    xo, its, relo = krylov.fgmres(lambda x: prob.A @ x, lambda v: mg.vcycle(levels, v), b, rtol=1e-8)
    s = wb.Solver(8, 2, torch.tensor(mu, device="cuda"))
    x, res = s.solve_block(wb.BLOCK_A, torch.tensor(b, device="cuda"), rtol=1e-8)
    assert res.status == 0 and abs(res.iters - its) <= 1, (res.iters, its)
    assert rel(N(x), xo) < 1e-10
    sm = wb.Solver(8, 2, torch.tensor(mu, device="cuda"), precision=wb.MIXED)
    xm, rm = sm.solve_block(wb.BLOCK_A, torch.tensor(b, device="cuda"), rtol=1e-6)
    assert rm.status == 0 and rm.rel_res <= 1e-6 and rm.iters <= its + 3   # its: the count to 1e-8


@pytest.mark.parametrize("which", [1, 2])
def test_Kw_alone_matches_oracle(wb, case, which):
    m, mu, f = case
    prob = W.StokesProblem(m, mu)
    cd, a = (prob.Cdiag, prob.a_l) if which == 1 else (prob.Ddiag, prob.a_r)
    K = op.assemble_Kw(prob.B, cd, m)
    pp = mg.PressurePoissonMG(m, prob.B, cd, mu, a)
    b = op.project_pressure(m, inputs.normal_vector(9, m.n_p))
    pc = lambda v: op.project_pressure(m, pp.apply(op.project_pressure(m, v)))
    xo, its, relo = krylov.fgmres(lambda x: K @ x, pc, b, rtol=1e-8)
    s = wb.Solver(8, 2, torch.tensor(mu, device="cuda"))
    x, res = s.solve_block(which, torch.tensor(b, device="cuda"), rtol=1e-8)
    assert res.status == 0 and abs(res.iters - its) <= 1, (res.iters, its)
    assert rel(N(x), op.project_pressure(m, xo)) < 1e-10


def test_block_solve_rejects_bad_arguments(wb, case):
    m, mu, f = case
    s = wb.Solver(8, 2, torch.tensor(mu, device="cuda"))
    b = torch.zeros(3 * m.n_nodes, dtype=torch.float64, device="cuda")
    with pytest.raises(wb.WbfbtError):
        s.solve_block(3, b)
    with pytest.raises(wb.WbfbtError):
        s.solve_block(wb.BLOCK_A, b.cpu())
