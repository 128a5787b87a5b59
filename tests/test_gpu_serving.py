"""Serving: continuous batching of arriving requests (GPU).

Requests of mixed sizes arrive (Poisson) while others are on the GPU; they
are admitted by device footprint and run concurrently on the context's
stream lanes.  Each result must equal the same request solved alone, and the
admitted footprints must never exceed the HBM budget.
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_cs_0408029_gb300 as ts
    from paper_cs_0408029_gb300 import serving

    return ts, serving


def test_mix_results_equal_alone_results(env):
    ts, serving = env
    probs = [workloads.serving_request(i, n_hi=1024) for i in range(24)]
    arrivals = workloads.serving_arrivals(len(probs), rate_per_s=2000.0)
    with ts.Context(0) as ctx:
        out = serving.replay(ctx, probs, arrivals)
        assert (out["status"] == ts.OK).all(), out["status"]
        q = out["queue"]
        assert q["completed"] == len(probs)
        assert q["max_active"] > 1  # requests overlapped on the device
        for p, x in zip(probs, out["x"]):
            alone, _ = ctx.solve(ts.HostCSR.from_problem(p), p.b)
            assert np.linalg.norm(x - alone) <= 1e-12 * np.linalg.norm(alone), p.name


def test_admission_respects_budget(env):
    ts, serving = env
    probs = [workloads.serving_request(100 + i, n_lo=256, n_hi=1536) for i in range(12)]
    arrivals = np.zeros(len(probs))  # all at once
    budget = 48 << 20
    with ts.Context(0, hbm_budget=budget) as ctx:
        out = serving.replay(ctx, probs, arrivals)
        assert (out["status"] == ts.OK).all()
        q = out["queue"]
        assert 0 < q["max_in_use_bytes"] <= budget
        # a request whose factor-path state can never fit is refused at submission
        big = workloads.serving_request(7, n_lo=4000, n_hi=4001)
        big_A, big_x = ts.HostCSR.from_problem(big), np.empty(big.n)
        with pytest.raises(ts.TsnnlsError) as e:
            ctx.submit(big_A, big.b, big_x, path="factor")
        assert e.value.status == ts.EADMIT
        # with AUTO the same request falls back to the LSQR path, which fits
        t = ctx.submit(big_A, big.b, big_x)
        st, info = ctx.wait(t)
        assert st == ts.OK and info.path_used == ts.PATH_LSQR


def test_burst_of_factor_solves_has_no_stall(env):
    """A burst of mid-size requests keeps every lane in the tensor-core
    factorisation at once; each solve must stay far below the seconds-long
    bound of the device-side waits (a wait that misses its barrier phase
    would sit out that bound and still return a correct result)."""
    ts, serving = env
    probs = [workloads.serving_request(300 + i, n_lo=1500, n_hi=3500) for i in range(24)]
    with ts.Context(0) as ctx:
        for _ in range(2):
            out = serving.replay(ctx, probs, np.zeros(len(probs)))
            assert (out["status"] == ts.OK).all(), out["status"]
            assert np.nanmax(out["device_ms"]) < 2000.0, np.nanmax(out["device_ms"])
