"""GPU solves of the benchmark configurations against the FP64 CPU oracle, and the solver's
failure statuses.

32^3 Q2, 24 sinkers, omega 0.05, delta 200, DR 1e6 (the plain-method FP64 configuration,
Sec. 2.1 multi-sinker problem; Table 3a row l = 5 has the same size): the GPU FP64 solve must
take the oracle's iteration count +-1 and match its solution to 1e-10 relative L2 (velocity and
pressure, pressure modulo the constant); the mixed-precision solve (FP32 preconditioner) must
match the oracle to 1e-6.  The oracle runs its V-cycle mode (assembled CSR operators), about
1.5 minutes on one host core.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mesh as M
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


def N(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def T(x, dtype=torch.float64):
    return torch.tensor(np.asarray(x), dtype=dtype, device="cuda")


def oracle_solve(cfg, **kw):
    m = M.Mesh(cfg["n"], cfg["n"], cfg["n"], cfg["k"])
    c = inputs.sinker_centres(cfg["seed"], cfg["n_sinkers"])
    mu, f = W.sinker_problem(m, c, cfg["omega"], cfg["delta"], cfg["dr"])
    u, p, its, relres, _ = W.solve(m, mu, f, **kw)
    return dict(mesh=m, centres=c, mu=mu, f=f, u=u, p=p, its=its, rel=relres)


@pytest.fixture(scope="module")
def config_b():
    return oracle_solve(inputs.WORKLOADS["32^3-Q2-S24-DR1e6"])


def gpu_config(wb, cfg, centres, **kw):
    mu_g, f_g = wb.sinker_setup(cfg["n"], cfg["k"], centres, cfg["omega"], cfg["delta"], cfg["dr"])
    return wb.Solver(cfg["n"], cfg["k"], mu_g, **kw), mu_g, f_g


def test_config_b_fp64_solve_matches_oracle(wb, config_b):
    cfg = inputs.WORKLOADS["32^3-Q2-S24-DR1e6"]
    s, mu_g, f_g = gpu_config(wb, cfg, config_b["centres"])
    # the GPU's own viscosity and forcing (row a1) equal the oracle's
    assert rel(N(mu_g), config_b["mu"]) < 1e-14
    assert rel(N(f_g), config_b["f"].T.ravel()) < 1e-14
    u, p, res = s.solve(f_g)
    assert res.status == 0 and res.rel_res <= 1e-6
    assert abs(res.iters - config_b["its"]) <= 1, (res.iters, config_b["its"])
    eu, ep = rel(N(u), config_b["u"]), rel(N(p), config_b["p"])
    print(f"config B FP64: its gpu {res.iters} oracle {config_b['its']}; rel err u {eu:.2e} p {ep:.2e}")
    assert eu < 1e-10 and ep < 1e-10


def test_config_b_mixed_solve_matches_oracle(wb, config_b):
    cfg = inputs.WORKLOADS["32^3-Q2-S24-DR1e6"]
    s, _, f_g = gpu_config(wb, cfg, config_b["centres"], precision=wb.MIXED)
    u, p, res = s.solve(f_g)
    assert res.status == 0 and res.rel_res <= 1e-6
    eu, ep = rel(N(u), config_b["u"]), rel(N(p), config_b["p"])
    print(f"config B mixed: its gpu {res.iters} oracle {config_b['its']}; rel err u {eu:.2e} p {ep:.2e}")
    assert abs(res.iters - config_b["its"]) <= 3
    assert eu < 1e-6 and ep < 1e-6


def test_config_b_mixed_fp32_arnoldi_matches_oracle(wb, config_b):
    """Mixed precision with the K apply inside the Arnoldi process in FP32 as well: the FP64 true
    residual decides convergence (<= 1e-6).  The FP32 error of the Arnoldi relation moves the
    iterate within the set of vectors with that residual, so the solution is held to 1e-5 of the
    oracle here (measured 1.5e-6), not to the 1e-6 of the default mixed form."""
    cfg = inputs.WORKLOADS["32^3-Q2-S24-DR1e6"]
    s, _, f_g = gpu_config(wb, cfg, config_b["centres"], precision=wb.MIXED, arnoldi_precision=wb.F32)
    u, p, res = s.solve(f_g)
    assert res.status == 0 and res.rel_res <= 1e-6
    eu, ep = rel(N(u), config_b["u"]), rel(N(p), config_b["p"])
    print(f"config B mixed, FP32 Arnoldi: its gpu {res.iters} oracle {config_b['its']}; rel err u {eu:.2e} p {ep:.2e}")
    assert abs(res.iters - config_b["its"]) <= 3
    assert eu < 1e-5 and ep < 1e-5


def test_fp32_arnoldi_needs_a_mixed_context(wb):
    s, mu_g, _ = small(wb)
    with pytest.raises(wb.WbfbtError):
        wb.Solver(4, 2, mu_g, arnoldi_precision=wb.F32)


@pytest.mark.parametrize("n,k,dr,ns", [(8, 2, 1e6, 8), (6, 3, 1e4, 4)])
def test_small_mixed_solve_matches_oracle(wb, n, k, dr, ns):
    """Mixed precision on 8^3 Q2 DR 1e6 and 6^3 Q3 DR 1e4 against the oracle's FP64 solve (on meshes this
    coarse, DR 1e8 sinkers of width 0.1 are unresolved and neither side converges in 1000 iterations)."""
    cfg = dict(n=n, k=k, n_sinkers=ns, omega=0.1, delta=200.0, dr=dr, seed=0)
    o = oracle_solve(cfg)
    for arn in (wb.F64, wb.F32):
        s, _, f_g = gpu_config(wb, cfg, o["centres"], precision=wb.MIXED, arnoldi_precision=arn)
        u, p, res = s.solve(f_g)
        assert res.status == 0 and res.rel_res <= 1e-6
        assert abs(res.iters - o["its"]) <= 3, (arn, res.iters, o["its"])
        tol = 1e-6 if arn == wb.F64 else 1e-5
        assert rel(N(u), o["u"]) < tol and rel(N(p), o["p"]) < tol


# ------------------------------------------------------------------ failure statuses
# Every failure is made on the host (a NaN in an input, an iteration limit): no kernel is
# driven into a fault.

def small(wb, **kw):
    cfg = dict(n=4, k=2, n_sinkers=4, omega=0.1, delta=200.0, dr=1e4, seed=0)
    c = inputs.sinker_centres(0, 4)
    return gpu_config(wb, cfg, c, **kw)


def test_nan_in_force_returns_nonfinite(wb):
    s, _, f_g = small(wb)
    f = f_g.clone()
    f[2 * s.n_nodes + s.n_nodes // 2] = float("nan")
    _, _, res = s.solve(f, check=False)
    assert res.status == wb.ERR_NONFINITE
    # the context stays usable: a clean solve afterwards converges
    _, _, res2 = s.solve(f_g)
    assert res2.status == 0


def test_iteration_limit_returns_maxit_with_iterate(wb):
    s, _, f_g = small(wb)
    u_ref, p_ref, full = s.solve(f_g)
    u, p, res = s.solve(f_g, maxit=2)
    assert res.status == wb.ERR_MAXIT
    assert res.iters == 2 and res.rel_res > 1e-6
    # the iterate after two steps is written: nonzero, finite, and not yet the solution
    un = N(u)
    assert np.all(np.isfinite(un)) and np.linalg.norm(un) > 0
    assert 1e-8 < rel(un, N(u_ref)) < 10.0
    with pytest.raises(wb.WbfbtError):
        s.solve(f_g, maxit=0)


@pytest.mark.parametrize("bad", [float("nan"), float("inf"), 0.0, -1.0])
def test_bad_viscosity_rejected_at_create_and_setup(wb, bad):
    s, mu_g, _ = small(wb)
    mu = mu_g.clone()
    mu[7] = bad
    with pytest.raises(wb.WbfbtError) as e:
        wb.Solver(4, 2, mu)
    assert e.value.status == wb.ERR_INVALID
    with pytest.raises(wb.WbfbtError) as e2:
        s.setup(mu)
    assert e2.value.status == wb.ERR_INVALID
    s.setup(mu_g)      # a valid viscosity afterwards restores the context
    _, _, res = s.solve(small(wb)[2])
    assert res.status == 0


def test_amplified_q3_solve_matches_oracle(wb):
    """Boundary amplification a_r = 4 (Eq. bdramp, the Table 2 / 3b setting for k = 3) on 6^3 Q3:
    iterations +-1 and solution 1e-10 against the oracle."""
    cfg = dict(n=6, k=3, n_sinkers=4, omega=0.1, delta=200.0, dr=1e4, seed=0)
    o = oracle_solve(cfg, opts=W.Options(a_r=4.0))
    s, _, f_g = gpu_config(wb, cfg, o["centres"], a_r=4.0)
    u, p, res = s.solve(f_g)
    assert res.status == 0 and abs(res.iters - o["its"]) <= 1, (res.iters, o["its"])
    assert rel(N(u), o["u"]) < 1e-10 and rel(N(p), o["p"]) < 1e-10
