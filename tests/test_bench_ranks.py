"""Host-side replica logic of bench.py on CPU ranks (gloo, world size 2).

On a GPU node every rank solves its own copy of the workload and the ranks
meet only at the barrier around the timed region and in the max over their
times (no collective on the data path).  These tests run that coordination,
and the reference arm's rank-0-only output, as two CPU processes.
"""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out_q, mode):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        if mode == "ranks":
            r = bench.Ranks(*bench.dist_env()[:2], torch.device("cpu"))
            r.barrier()
            slowest = r.max_over_ranks(1.0 + rank)  # rank 1 is the slow one
            out_q.put((rank, slowest, r.value(5, slowest)))
        else:
            # the reference arm with a stub for the oracle's timed solves:
            # rank 0 alone prints its line, the other ranks return without work
            import types

            import numpy as np

            stub = types.SimpleNamespace(iters=3, x=np.zeros(8000))
            bench.oracle_full_solves = lambda prob, count, budget_s, warmup=0: ([0.5, 0.5], stub)

            class Args:
                steps, warmup, ref_budget_s = 2, 0, 60.0

            buf = io.StringIO()
            with redirect_stdout(buf):
                bench.run_reference(Args())
            out_q.put((rank, buf.getvalue()))
    finally:
        dist.destroy_process_group()


def _run(mode):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q, mode)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(res)


def test_max_over_ranks_and_weak_scaling_value():
    res = _run("ranks")
    assert [r[1] for r in res] == [2.0, 2.0]          # both ranks see the slowest time
    assert [r[2] for r in res] == [5.0, 5.0]          # 2 ranks x 5 units / 2 s


def test_reference_arm_prints_on_rank_zero_only():
    pytest.importorskip("workloads")
    res = _run("reference")
    lines0 = [l for l in res[0][1].splitlines() if l.strip()]
    assert len(lines0) == 1 and res[1][1].strip() == ""
    d = json.loads(lines0[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] == pytest.approx(2.0)
    assert d["steps"] == 2 and d["ms_per_step"] == pytest.approx(500.0)
