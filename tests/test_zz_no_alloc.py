"""The allocation-free factor solve (tsnnls_chol_solve_noalloc), GPU.

Callers that may not allocate device memory (their own pool owns the memory
they may use, or their thread cannot take cudaMalloc's latency and possible
device-wide synchronisation) use this entry point: it runs the same
triangular solves as tsnnls_chol_solve with the scratch in a static device
array.  The test calls it through the C ABI twice in a row and checks each
result against tsnnls_chol_solve on the same factor, within the tolerance
the other factor tests use, and against the CPU oracle's textbook Cholesky
solve of the same matrix, within the tolerances of the factor parity tests.
The file name sorts last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_cs_0408029_gb300 as ts

    ts.load()
    ctx = ts.Context(0)
    yield ts, ctx, torch
    ctx.close()


@pytest.mark.parametrize("k,precision,rtol,rtol_oracle", [(700, 0, 1e-5, 1e-2), (257, 1, 1e-12, 1e-9)])
def test_noalloc_matches_context_solve_twice(env, oracle_mod, k, precision, rtol, rtol_oracle):
    ts, ctx, torch = env
    dt = torch.float32 if precision == ts.MIXED else torch.float64
    rng = np.random.default_rng(k)
    a = rng.standard_normal((k + 40, k))
    s = a.T @ a
    S = torch.as_tensor(s.T.copy(), dtype=dt, device="cuda")
    st, info = ctx.cholesky(S, k, k, precision=precision)
    assert st == ts.OK and info == 0
    L_ref = oracle_mod.cholesky(s)
    for call in range(2):
        rhs = rng.standard_normal(k)
        want = torch.as_tensor(rhs, dtype=dt, device="cuda")
        ctx.chol_solve(S, k, k, want, precision=precision)
        got = torch.as_tensor(rhs, dtype=dt, device="cuda")
        assert ts.chol_solve_noalloc(S, k, k, got, precision=precision) == ts.OK, call
        w = want.cpu().numpy().astype(np.float64)
        g = got.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(g - w) <= rtol * np.linalg.norm(w), call
        x_ref = oracle_mod.cholesky_solve(L_ref, rhs)
        assert np.linalg.norm(g - x_ref) <= rtol_oracle * np.linalg.norm(x_ref), call


def test_noalloc_rejects_oversized_k(env):
    ts, ctx, torch = env
    L = torch.ones(4, dtype=torch.float32, device="cuda")
    rhs = torch.ones(4, dtype=torch.float32, device="cuda")
    big = 65536 + 1
    assert ts.chol_solve_noalloc(L, big, big, rhs) == ts.EINVAL
