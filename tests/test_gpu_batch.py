"""Batched dense path (many uneven problems in one persistent launch), GPU.

Each problem of a batch is compared with the CPU oracle (FP64 A built from
the same FP32 values) and with its own solve-alone result through the
single-problem path; the FP64 batch path is checked the same way.
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


def _batch(seed, count, n_lo, n_hi):
    return workloads.batched_uneven(seed=seed, count=count, n_lo=n_lo, n_hi=n_hi)


def _run(ts, ctx, torch, probs, precision):
    a = [torch.as_tensor(p.a, device="cuda") for p in probs]
    b = [torch.as_tensor(p.b, device="cuda") for p in probs]
    x = [torch.empty(p.n, dtype=torch.float64, device="cuda") for p in probs]
    st, stat, info = ctx.solve_batch_dense(a, b, x, precision=precision)
    return st, stat, info, [t.cpu().numpy() for t in x]


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_batch_matches_oracle(env, oracle_mod, precision):
    ts, ctx, torch = env
    probs = _batch(101, 24, 32, 300)
    st, stat, info, xs = _run(ts, ctx, torch, probs, precision)
    assert st == ts.OK and (stat == ts.OK).all(), stat
    assert info.kernel_launches >= 2
    for p, x in zip(probs, xs):
        csr = workloads.dense_to_csr(p.a.astype(np.float64), p.b)
        ref = oracle_mod.bpp_solve(csr)
        err = np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x)
        assert err <= 1e-9, (p.name, err)
        assert kkt.violation(csr, x) <= 1e-10 * kkt.atb_norm(csr)


def test_batch_equals_solve_alone(env):
    ts, ctx, torch = env
    probs = _batch(102, 16, 32, 1024)
    st, stat, info, xs = _run(ts, ctx, torch, probs, "mixed")
    assert st == ts.OK
    for p, x in zip(probs, xs):
        csr = workloads.dense_to_csr(p.a.astype(np.float64), p.b)
        alone, _ = ctx.solve(ts.HostCSR.from_problem(csr), csr.b)
        assert np.linalg.norm(x - alone) <= 1e-9 * np.linalg.norm(alone), p.name


def test_replayed_graph_reads_the_new_problems(env, oracle_mod):
    """A second call of the same shape replays the first call's graph: its
    problems (new values, new buffers) must still be the ones solved."""
    ts, ctx, torch = env
    first = _batch(105, 10, 32, 400)
    second = [workloads.DenseProblem(p.m, p.n, (-1.5 * p.a).astype(np.float32),
                                     -1.5 * p.b + 0.25 * np.linspace(-1, 1, p.m), None, p.name + "_b")
              for p in first]
    for probs in (first, second, first):
        st, stat, info, xs = _run(ts, ctx, torch, probs, "mixed")
        assert st == ts.OK
        for p, x in zip(probs, xs):
            ref = oracle_mod.bpp_solve(workloads.dense_to_csr(p.a.astype(np.float64), p.b))
            assert np.linalg.norm(x - ref.x) <= 1e-9 * max(np.linalg.norm(ref.x), 1e-300), p.name


def test_batch_single_and_ragged_sizes(env, oracle_mod):
    ts, ctx, torch = env
    rng = np.random.default_rng(7)
    probs = []
    for n in (1, 2, 31, 32, 33, 63, 64, 65, 129, 1024):
        m = n + 1 + n // 2
        a = rng.standard_normal((m, n)).astype(np.float32)
        xs = np.where(rng.random(n) < 0.3, 0.0, rng.uniform(0.1, 1.0, n))
        b = a.astype(np.float64) @ xs + 1e-3 * rng.standard_normal(m)
        probs.append(workloads.DenseProblem(m, n, a, b, xs, f"n{n}"))
    st, stat, info, xs = _run(ts, ctx, torch, probs, "mixed")
    assert st == ts.OK, stat
    for p, x in zip(probs, xs):
        csr = workloads.dense_to_csr(p.a.astype(np.float64), p.b)
        ref = oracle_mod.bpp_solve(csr)
        assert np.linalg.norm(x - ref.x) <= 1e-9 * max(np.linalg.norm(ref.x), 1e-300), p.name


def test_batch_rejects_bad_sizes(env):
    ts, ctx, torch = env
    a = [torch.zeros((4, 4), dtype=torch.float32, device="cuda")]
    b = [torch.zeros(4, dtype=torch.float64, device="cuda")]
    x = [torch.zeros(4, dtype=torch.float64, device="cuda")]
    st, _, _ = ctx.solve_batch_dense(a, b, x)
    assert st == ts.EINVAL


def test_autotune_picks_candidate_widths(env):
    ts, ctx, torch = env
    nb = ctx.batch_autotune(ts.MIXED, per_bucket=16)
    assert set(nb.tolist()) <= {8, 16, 32, 48}
    probs = _batch(103, 8, 32, 512)
    st, stat, info, xs = _run(ts, ctx, torch, probs, "mixed")
    assert st == ts.OK


def test_autotune_cache_hit_skips_timing(env, tmp_path):
    """First call tunes and records the widths under this device's key; the
    second finds them; a seeded entry is installed as it stands."""
    ts, ctx, torch = env
    path = str(tmp_path / "widths.json")
    key = ctx.batch_tune_key(ts.MIXED, per_bucket=8)
    assert "sm_10" in key and "mixed" in key
    nb, hit = ctx.batch_autotune_cached(path, ts.MIXED, per_bucket=8)
    assert not hit and list(ts.tune_cache_get(path, key)) == list(nb)
    nb2, hit2 = ctx.batch_autotune_cached(path, ts.MIXED, per_bucket=8)
    assert hit2 and list(nb2) == list(nb)
    seeded = str(tmp_path / "seeded.json")
    ts.tune_cache_put(seeded, key, [16, 16, 16, 16, 16])
    nb3, hit3 = ctx.batch_autotune_cached(seeded, ts.MIXED, per_bucket=8)
    assert hit3 and list(nb3) == [16] * 5
    probs = _batch(104, 8, 32, 300)
    st, stat, info, xs = _run(ts, ctx, torch, probs, "mixed")
    assert st == ts.OK
    ts.Context.batch_set_panel([32] * 5, ts.MIXED)  # the built-in table


def test_batch_traces_match_oracle_and_full_refinement(env, oracle_mod):
    """Every problem's pivot trace equals the oracle's (A rounded to FP32 on
    both sides); refining intermediate pivots only until their signs are
    settled (the default) gives the same traces and x as refining every pivot
    to rel_tol, with fewer refinement steps."""
    ts, ctx, torch = env
    probs = _batch(104, 20, 32, 1024)
    a = [torch.as_tensor(p.a, device="cuda") for p in probs]
    b = [torch.as_tensor(p.b, device="cuda") for p in probs]
    out = {}
    for full in (0, 1):
        x = [torch.empty(p.n, dtype=torch.float64, device="cuda") for p in probs]
        st, stat, info, trs = ctx.solve_batch_dense(a, b, x, trace_cap=400, full_refine=full)
        assert st == ts.OK, stat
        out[full] = ([t.cpu().numpy() for t in x], trs, info.refine_steps)
    assert out[0][2] < out[1][2]
    for i, p in enumerate(probs):
        csr = workloads.dense_to_csr(p.a.astype(np.float64), p.b)
        ref = oracle_mod.bpp_solve(csr)
        assert np.array_equal(out[0][1][i], ref.trace), p.name
        assert np.array_equal(out[1][1][i], ref.trace), p.name
        x0, x1 = out[0][0][i], out[1][0][i]
        assert np.linalg.norm(x0 - x1) <= 1e-12 * np.linalg.norm(x1), p.name


def test_batch_single_exchange_fallback(env, oracle_mod):
    """p_max = 0 on conditioned problems (A rounded to FP32): the persistent
    kernel's single-variable fallback moves the largest infeasible index,
    row by row as the oracle does."""
    ts, ctx, torch = env
    probs = []
    for seed, (m, n) in enumerate([(60, 40), (200, 150), (400, 300)]):
        prob, _, _ = workloads.conditioned_dense(m, n, 1e3, seed=seed + 2, active_frac=1.0)
        a32 = prob.a.astype(np.float32)
        probs.append(workloads.DenseProblem(m, n, a32, prob.b, prob.x_planted, f"cond{n}"))
    a = [torch.as_tensor(p.a, device="cuda") for p in probs]
    b = [torch.as_tensor(p.b, device="cuda") for p in probs]
    x = [torch.empty(p.n, dtype=torch.float64, device="cuda") for p in probs]
    st, stat, info, trs = ctx.solve_batch_dense(a, b, x, trace_cap=400, p_max=0)
    assert st == ts.OK, stat
    singles = 0
    for p, tr, xt in zip(probs, trs, x):
        csr = workloads.dense_to_csr(p.a.astype(np.float64), p.b)
        ref = oracle_mod.bpp_solve(csr, p_max=0)
        assert np.array_equal(tr, ref.trace), p.name
        singles += int((ref.trace[:, 3] == 2).sum())
        xv = xt.cpu().numpy()
        assert np.linalg.norm(xv - ref.x) <= 1e-9 * np.linalg.norm(ref.x), p.name
    assert singles >= 3


def test_batched_full_size_sampled(env, oracle_mod):
    """The bench's configuration: all 512 problems of the batched workload in
    one call (MIXED).  Every result passes the KKT test of Eq. 3; the three
    largest problems and five others drawn with a fixed seed are compared
    with the oracle one by one."""
    ts, ctx, torch = env
    probs = workloads.batched_uneven()
    assert len(probs) == 512
    st, stat, info, xs = _run(ts, ctx, torch, probs, "mixed")
    assert st == ts.OK and (stat == ts.OK).all(), stat
    for p, x in zip(probs, xs):  # dense KKT in numpy, on the FP64 copy of the FP32 values
        a = p.a.astype(np.float64)
        y = a.T @ (a @ x - p.b)
        scale = np.linalg.norm(a.T @ p.b)
        assert x.min() >= 0.0, p.name
        assert -y.min() <= 1e-10 * scale, p.name
        assert np.max(np.abs(x * y) / np.maximum(1.0, np.abs(x))) <= 1e-10 * scale, p.name
    ns = np.array([p.n for p in probs])
    pick = list(np.argsort(-ns, kind="stable")[:3]) + list(np.random.default_rng(7).choice(512, 5, replace=False))
    for i in pick:
        p = probs[int(i)]
        ref = oracle_mod.bpp_solve(workloads.dense_to_csr(p.a.astype(np.float64), p.b))
        err = np.linalg.norm(xs[int(i)] - ref.x) / np.linalg.norm(ref.x)
        assert err <= 1e-9, (p.name, err)
