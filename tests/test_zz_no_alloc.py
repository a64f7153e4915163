"""The allocation-free pressure-Poisson apply (wbfbt_apply_Kw_noalloc) against the context one.

Callers that cannot allocate device memory (foreign memory pools, real-time hosts,
caller-buffer-only libraries) use wbfbt_apply_Kw_noalloc, whose temporaries live in
a static device array.  This file is collected last on purpose.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1607_03936_gb300 import build
    build.build()
    from paper_1607_03936_gb300 import wbfbt
    return wbfbt


def test_noalloc_Kw_matches_context_apply_twice(wb):
    from paper_1607_03936_gb300 import inputs
    n, k = 6, 2
    c = inputs.sinker_centres(11, 6)
    mu, _ = wb.sinker_setup(n, k, c, 0.1, 200.0, 1e6)
    s = wb.Solver(n, k, mu, a_l=2.0)
    rng = np.random.default_rng(12)
    y = torch.empty(s.n_p, dtype=torch.float64, device="cuda")
    for call in range(2):   # two calls in a row: the shared static scratch keeps the last call's contents
        p = torch.tensor(rng.standard_normal(s.n_p), dtype=torch.float64, device="cuda")
        ref = s.apply_Kw(0, p)
        wb.apply_Kw_noalloc(n, k, mu, 2.0, p, y)
        torch.cuda.synchronize()
        err = (torch.linalg.norm(y - ref) / torch.linalg.norm(ref)).item()
        assert err < 1e-12, (call, err)
    s.close()


def test_noalloc_rejects_meshes_beyond_the_static_scratch(wb):
    n = 64   # (2*64+1)^3 nodes > the static limit
    assert (2 * n + 1) ** 3 > wb.NOALLOC_MAX_NODES
    mu = torch.ones(1, dtype=torch.float64, device="cuda")
    p = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(wb.WbfbtError):
        wb.apply_Kw_noalloc(n, 2, mu, 1.0, p, p)


def test_noalloc_rejects_axis_counts_that_overflow_int(wb):
    """k*n+1 beyond 2^31 on an axis is rejected before any product is formed."""
    mu = torch.ones(1, dtype=torch.float64, device="cuda")
    p = torch.zeros(1, dtype=torch.float64, device="cuda")
    for n in (2 ** 30, 2 ** 31 - 1):
        with pytest.raises(wb.WbfbtError):
            wb.apply_Kw_noalloc(n, 2, mu, 1.0, p, p)
