"""tsnnls_submit_batch: many independent CSR solves under one ticket (GPU).

The members are admitted one by one by device footprint and run beside each
other on the context's lanes.  Each member's x must meet the oracle bar
(relative error 1e-9, KKT violation 1e-10 ||A^T b||) and equal the same
problem solved alone; the ticket's info aggregates the members'.
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

    ts.load()
    return ts, torch


def _members(ts, torch):
    probs = [workloads.serving_request(40 + i, n_hi=1024) for i in range(5)]
    probs.append(workloads.plain_single())
    probs += [workloads.random_sparse(900, 700, 0.05, seed=2, zero_frac=0.4, noise=0.05),
              workloads.random_sparse(130, 97, 0.2, seed=4, zero_frac=0.4, noise=0.05)]
    As, bs, xs = [], [], []
    for i, p in enumerate(probs):
        if i % 3 == 2:  # some members live on the device
            As.append(ts.DeviceCSR.from_problem(p))
            bs.append(torch.as_tensor(p.b, device="cuda"))
            xs.append(torch.empty(p.n, dtype=torch.float64, device="cuda"))
        else:
            As.append(ts.HostCSR.from_problem(p))
            bs.append(np.ascontiguousarray(p.b))
            xs.append(np.empty(p.n))
    return probs, As, bs, xs


def _host(x):
    return x if isinstance(x, np.ndarray) else x.cpu().numpy()


def test_batch_members_match_oracle_and_solve_alone(env, oracle_mod):
    ts, torch = env
    probs, As, bs, xs = _members(ts, torch)
    with ts.Context(0) as ctx:
        t = ctx.submit_batch(As, bs, xs)
        infos = [None] * len(probs)
        while any(i is None for i in infos):  # collect members as they finish, no release
            for i in range(len(probs)):
                if infos[i] is None:
                    st, info = ctx.batch_member_info(t, i)
                    if st != ts.PENDING:
                        assert st == ts.OK, (i, st)
                        infos[i] = info
        st, agg = ctx.wait(t)
        assert st == ts.OK
        assert agg.iters == sum(i.iters for i in infos)
        assert agg.nF == sum(i.nF for i in infos)
        assert agg.kkt_viol == max(i.kkt_viol for i in infos) <= 1e-10
        assert ctx.batch_member_info(t, 0)[0] == ts.EINVAL  # released
        assert ctx.poll(t)[0] == ts.EINVAL
        q = ctx.queue_stats()
        assert q["completed"] == len(probs) and q["max_active"] > 1
        for p, x, info in zip(probs, xs, infos):
            x = _host(x)
            ref = oracle_mod.bpp_solve(p)
            err = np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x)
            assert err <= 1e-9, (p.name, err)
            assert kkt.violation(p, x) <= 1e-10 * kkt.atb_norm(p)
            alone, ainfo = ctx.solve(ts.HostCSR.from_problem(p), p.b)
            assert np.linalg.norm(x - alone) <= 1e-12 * np.linalg.norm(alone), p.name
            assert info.iters == ainfo.iters == ref.iters


def test_batch_is_accepted_whole_or_not_at_all(env):
    ts, torch = env
    good = workloads.plain_single()
    bad = workloads.random_sparse(40, 20, 0.2, seed=3)
    with ts.Context(0) as ctx:
        As = [ts.HostCSR.from_problem(good), ts.HostCSR(20, 20, bad.row_ptr[:21], bad.col_idx, bad.val)]
        with pytest.raises(ts.TsnnlsError) as e:
            ctx.submit_batch(As, [good.b, bad.b[:20]], [np.empty(good.n), np.empty(20)])
        assert e.value.status == ts.EINVAL  # m == n in the second member
        assert ctx.queue_stats()["submitted"] == 0
        with ts.Context(0, hbm_budget=1 << 16) as small:
            with pytest.raises(ts.TsnnlsError) as e:
                small.submit_batch([ts.HostCSR.from_problem(good)], [good.b], [np.empty(good.n)],
                                   path="factor")
            assert e.value.status == ts.EADMIT
