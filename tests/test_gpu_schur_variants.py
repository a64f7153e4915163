"""GPU parity of the inverse-viscosity pressure-mass Schur approximations (Sec. 1.3, Eq. lumping),
the baseline that Sec. 4 / Table 1 compares w-BFBT against, through the C ABI.

Tolerances as elsewhere: FP64 applies 1e-12 relative, FP32 2e-5; FP64 solves iterations +-1
and solution 1e-10.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mesh as M
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


def problem(n, k, dr, ns, lengths=(1.0, 1.0, 1.0), ny=None, nz=None):
    m = M.Mesh(n, ny or n, nz or n, k, *lengths)
    c = inputs.sinker_centres(2, ns)
    mu, f = W.sinker_problem(m, c, 0.1, 200.0, dr)
    return m, mu, f


VARIANTS = [("mass", 1), ("mass_diag", 2)]


@pytest.mark.parametrize("name,code", VARIANTS)
@pytest.mark.parametrize("shape", [(4, 2, (1.0, 1.0, 1.0), 3, 5), (3, 3, (1.0, 0.8, 1.2), 2, 2), (2, 4, (1.0, 1.0, 1.0), 2, 2)])
def test_mass_schur_apply_matches_oracle(wb, name, code, shape):
    n, k, L, ny, nz = shape
    m, mu, _ = problem(n, k, 1e4, 4, L, ny, nz)
    mu_t = torch.tensor(mu, device="cuda")
    prob = W.StokesProblem(m, mu)
    ref = W.MassSchur(prob, diag=name == "mass_diag")
    r = np.random.default_rng(3).standard_normal(m.n_p)
    s64 = wb.Solver(n, k, mu_t, ny=ny, nz=nz, lengths=L, schur=code)
    assert rel(N(s64.apply_schur_inv(torch.tensor(r, device="cuda"))), ref.apply(r)) < 1e-12
    s32 = wb.Solver(n, k, mu_t, ny=ny, nz=nz, lengths=L, schur=code, precision=wb.MIXED)
    y32 = N(s32.apply_schur_inv(torch.tensor(r, dtype=torch.float32, device="cuda")))
    assert rel(y32, ref.apply(r.astype(np.float32).astype(np.float64))) < 2e-5


@pytest.mark.parametrize("name,code", VARIANTS)
def test_mass_schur_solve_matches_oracle(wb, name, code):
    m, mu, f = problem(8, 2, 1e2, 4)
    uo, po, its, relo, _ = W.solve(m, mu, f, W.Options(schur=name), maxit=2000)
    s = wb.Solver(8, 2, torch.tensor(mu, device="cuda"), schur=code)
    u, p, res = s.solve(torch.tensor(f.T.ravel(), device="cuda"), maxit=2000)
    assert res.status == 0 and abs(res.iters - its) <= 1, (res.iters, its)
    assert rel(N(u), uo) < 1e-10 and rel(N(p), po) < 1e-10


def test_invalid_schur_option_rejected(wb):
    m, mu, _ = problem(2, 2, 1e2, 1)
    with pytest.raises(wb.WbfbtError):
        wb.Solver(2, 2, torch.tensor(mu, device="cuda"), schur=3)


# ------------------------------------------------------------------ viscosity-gradient weights
# w = (mu^2 + |grad mu|^2)^(1/4) in place of sqrt(mu) (remark in Sec. 4): the weighted lumped
# masses C, D, the K_w operators, their V-cycles and the solve against the oracle.

def test_gradient_weights_Kw_and_vcycle_match_oracle(wb):
    from oracle import multigrid as mg
    m, mu, _ = problem(8, 2, 1e4, 4)
    prob = W.StokesProblem(m, mu, a_l=1.0, a_r=2.0, weights="grad")
    r = op.project_pressure(m, np.random.default_rng(5).standard_normal(m.n_p))
    s64 = wb.Solver(8, 2, torch.tensor(mu, device="cuda"), a_r=2.0, weights=wb.WEIGHTS_GRAD)
    s32 = wb.Solver(8, 2, torch.tensor(mu, device="cuda"), a_r=2.0, weights=wb.WEIGHTS_GRAD, precision=wb.MIXED)
    for which, cd, a in ((0, prob.Cdiag, 1.0), (1, prob.Ddiag, 2.0)):
        K = op.assemble_Kw(prob.B, cd, m)
        assert rel(N(s64.apply_Kw(which, torch.tensor(r, device="cuda"))), K @ r) < 1e-12
        y32 = N(s32.apply_Kw(which, torch.tensor(r, dtype=torch.float32, device="cuda")))
        assert rel(y32, K @ r.astype(np.float32).astype(np.float64)) < 5e-5
        pp = mg.PressurePoissonMG(m, prob.B, cd, mu, a, "grad")
        assert rel(N(s64.apply_Kinv(which, torch.tensor(r, device="cuda"))), pp.apply(r)) < 1e-10


def test_gradient_weights_solve_matches_oracle(wb):
    m, mu, f = problem(8, 2, 1e6, 8)
    uo, po, its, relo, _ = W.solve(m, mu, f, W.Options(weights="grad"))
    s = wb.Solver(8, 2, torch.tensor(mu, device="cuda"), weights=wb.WEIGHTS_GRAD)
    u, p, res = s.solve(torch.tensor(f.T.ravel(), device="cuda"))
    assert res.status == 0 and abs(res.iters - its) <= 1, (res.iters, its)
    assert rel(N(u), uo) < 1e-10 and rel(N(p), po) < 1e-10


def test_several_kinv_cycles_match_oracle(wb):
    """kinv_cycles = 3: each K~_w^-1 runs three residual-correcting V-cycles, on both sides."""
    m, mu, f = problem(8, 2, 1e6, 8)
    uo, po, its, relo, _ = W.solve(m, mu, f, W.Options(kinv_cycles=3))
    s = wb.Solver(8, 2, torch.tensor(mu, device="cuda"), kinv_cycles=3)
    r = op.project_pressure(m, np.random.default_rng(6).standard_normal(m.n_p))
    prob = W.StokesProblem(m, mu)
    ref = W.WBFBT(prob, "vcycle", 3)
    assert rel(N(s.apply_schur_inv(torch.tensor(r, device="cuda"))), ref.apply(r)) < 1e-10
    u, p, res = s.solve(torch.tensor(f.T.ravel(), device="cuda"))
    assert res.status == 0 and abs(res.iters - its) <= 1, (res.iters, its)
    assert rel(N(u), uo) < 1e-10 and rel(N(p), po) < 1e-10


def test_several_ainv_cycles_match_oracle(wb):
    """ainv_cycles = 3: each A~^-1 of the block preconditioner runs three residual-correcting
    V-cycles, on both sides: the block preconditioner at 1e-10 (FP64), the FP64 solve +-1 its and
    1e-10, the mixed solve within 1e-6 of the oracle's."""
    m, mu, f = problem(8, 2, 1e6, 8)
    uo, po, its, relo, _ = W.solve(m, mu, f, W.Options(ainv_cycles=3))
    s = wb.Solver(8, 2, torch.tensor(mu, device="cuda"), ainv_cycles=3)
    prob = W.StokesProblem(m, mu)
    pc = W.BlockPreconditioner(prob, "vcycle", -1.0, ainv_cycles=3)
    rng = np.random.default_rng(9)
    x = np.concatenate([rng.standard_normal(m.n_u) * m.interior_dof_mask(), rng.standard_normal(m.n_p)])
    assert rel(N(s.apply_precond(torch.tensor(x, device="cuda"))), pc.apply(x)) < 1e-10
    u, p, res = s.solve(torch.tensor(f.T.ravel(), device="cuda"))
    assert res.status == 0 and abs(res.iters - its) <= 1, (res.iters, its)
    assert rel(N(u), uo) < 1e-10 and rel(N(p), po) < 1e-10
    s32 = wb.Solver(8, 2, torch.tensor(mu, device="cuda"), ainv_cycles=3, precision=wb.MIXED)
    u, p, res = s32.solve(torch.tensor(f.T.ravel(), device="cuda"))
    assert res.status == 0 and abs(res.iters - its) <= 3, (res.iters, its)
    assert rel(N(u), uo) < 1e-6 and rel(N(p), po) < 1e-6


# ------------------------------------------------------------------ diag(A)-BFBT (Sec. 1.3)

def test_diag_a_bfbt_matches_oracle(wb):
    from oracle import multigrid as mg
    m, mu, f = problem(8, 2, 1e4, 4)
    prob = W.StokesProblem(m, mu, weights="diag_a")
    r = op.project_pressure(m, np.random.default_rng(8).standard_normal(m.n_p))
    s64 = wb.Solver(8, 2, torch.tensor(mu, device="cuda"), weights=wb.WEIGHTS_DIAG_A)
    s32 = wb.Solver(8, 2, torch.tensor(mu, device="cuda"), weights=wb.WEIGHTS_DIAG_A, precision=wb.MIXED)
    K = op.assemble_Kw(prob.B, prob.Cdiag, m)
    for which in (0, 1):
        assert rel(N(s64.apply_Kw(which, torch.tensor(r, device="cuda"))), K @ r) < 1e-12
        y32 = N(s32.apply_Kw(which, torch.tensor(r, dtype=torch.float32, device="cuda")))
        assert rel(y32, K @ r.astype(np.float32).astype(np.float64)) < 5e-5
    pp = mg.PressurePoissonMG(m, prob.B, prob.Cdiag, mu, 1.0, "diag_a")
    assert rel(N(s64.apply_Kinv(1, torch.tensor(r, device="cuda"))), pp.apply(r)) < 1e-10
    ref = W.WBFBT(prob, "vcycle")
    assert rel(N(s64.apply_schur_inv(torch.tensor(r, device="cuda"))), ref.apply(r)) < 1e-10
    uo, po, its, relo, _ = W.solve(m, mu, f, W.Options(weights="diag_a"), maxit=2000)
    u, p, res = s64.solve(torch.tensor(f.T.ravel(), device="cuda"), maxit=2000)
    assert res.status == 0 and abs(res.iters - its) <= 1, (res.iters, its)
    assert rel(N(u), uo) < 1e-10 and rel(N(p), po) < 1e-10
