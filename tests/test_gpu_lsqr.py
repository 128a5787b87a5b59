"""LSQR path (LSQR on A_F for each pivot, column-scaled, FP32 inner products
with FP64 residual correction), GPU.

Scaled-down instances of the large sparse recipe are compared with the CPU
oracle; the full 2,000,000 x 200,000 instance, far beyond what the oracle can
solve, is checked by the KKT certificate of Eq. 3 (which, with A^T A positive
definite, identifies the unique solution) and against the FP64 LSQR path.
"""
import numpy as np
import pytest

import workloads
from oracle import kkt

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_cs_0408029_gb300 as ts

    ctx = ts.Context(0)
    yield ts, ctx, torch
    ctx.close()


def _scaled_recipe(m, n, seed, spread):
    """The large LSQR recipe at a reduced size, columns scaled by 10^U(-spread, spread)."""
    return workloads.lsqr_large(seed=seed, m=m, n=n, col_spread=spread)


@pytest.mark.parametrize("m,n,seed,spread", [(20000, 2000, 4, 2.0), (20000, 2000, 1, 1.0),
                                             (6000, 900, 2, 0.5), (3001, 401, 3, 1.0)])
def test_lsqr_path_matches_oracle(env, oracle_mod, m, n, seed, spread):
    ts, ctx, torch = env
    p = _scaled_recipe(m, n, seed, spread)
    ref = oracle_mod.bpp_solve(p, final_step=oracle_mod.FINAL_LSQR)
    A = ts.HostCSR.from_problem(p)
    for precision in ("mixed", "fp64"):
        x, y, inF, trace, info = ctx.solve_ex(A, p.b, precision=precision, path="lsqr")
        assert info.path_used == ts.PATH_LSQR
        err = np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x)
        assert err <= 1e-9, (precision, err)
        atb = kkt.atb_norm(p)
        assert kkt.violation(p, x) <= 1e-10 * atb
        band = 1e-10 * atb
        yr = kkt.dual(p, ref.x)
        clear = (np.abs(ref.x) > band) | (np.abs(yr) > band)
        assert np.array_equal(inF[clear], ref.inF[clear])


def test_lsqr_path_agrees_with_factor_path(env):
    ts, ctx, torch = env
    p = workloads.random_sparse(1500, 1000, 0.02, seed=5, zero_frac=0.4, noise=0.05)
    A = ts.HostCSR.from_problem(p)
    xf, _ = ctx.solve(A, p.b, path="factor")
    xl, info = ctx.solve(A, p.b, path="lsqr")
    assert info.path_used == ts.PATH_LSQR
    assert np.linalg.norm(xl - xf) <= 1e-10 * np.linalg.norm(xf)


def test_lsqr_full_size_kkt(env):
    """2e6 x 2e5, 8 nonzeros per row, columns scaled by 10^U(-2,2): AUTO picks
    LSQR (A^T A would not fit), device-resident inputs as in the benchmark."""
    ts, ctx, torch = env
    p = workloads.lsqr_large()
    A = ts.DeviceCSR.from_problem(p)
    b = torch.as_tensor(p.b, device="cuda")
    x, info = ctx.solve(A, b)
    assert info.path_used == ts.PATH_LSQR
    x = x.cpu().numpy()
    atb = kkt.atb_norm(p)
    assert kkt.violation(p, x) <= 1e-10 * atb
    x64, _ = ctx.solve(A, b, precision="fp64")
    x64 = x64.cpu().numpy()
    assert np.linalg.norm(x - x64) <= 1e-9 * np.linalg.norm(x64)
