"""Replay a trace of NNLS requests through the asynchronous C ABI.

Each request is submitted at its arrival time (tsnnls_submit); the context
admits it as soon as its device footprint fits the HBM budget and a stream
lane is free, and runs it concurrently with the requests already on the GPU
(continuous batching).  Latency is measured from arrival to the moment the
completion is observed.  Argument marshalling and timing only: every solve
runs in the library.
"""
from __future__ import annotations

import time

import numpy as np

from . import PENDING, HostCSR


def replay(ctx, problems, arrivals, precision="mixed", poll_s=0.0002, keep_x=True):
    """Submit problems[i] at time arrivals[i] (seconds from the start).

    ``problems`` is a sequence of problems (m, n, row_ptr, col_idx, val, b).
    It may also be a lazy source: indexing may block until request i is
    ready, and if it has a ``release(i)`` method that is called once request
    i has completed, so that a long trace never holds every request in host
    memory at once.  Requests are fetched in arrival order.

    Returns dict with x (list; None entries unless keep_x), status,
    latency_s (per request), wall_s, device_ms (per request), and the queue
    statistics."""
    n = len(arrivals)
    order = np.argsort(arrivals, kind="stable")
    release = getattr(problems, "release", None)
    xs = [None] * n
    lat = np.full(n, np.nan)
    dev_ms = np.full(n, np.nan)
    status = np.full(n, -1, dtype=np.int64)
    pending = {}
    t0 = time.perf_counter()
    nxt = 0

    def drain():
        for t in list(pending):
            st, info = ctx.poll(t)
            if st == PENDING:
                continue
            i, arr, x = pending.pop(t)
            lat[i] = time.perf_counter() - (t0 + arr)
            dev_ms[i] = info.time_ms
            status[i] = st
            if keep_x:
                xs[i] = x
            if release is not None:
                release(i)

    while nxt < n or pending:
        now = time.perf_counter() - t0
        while nxt < n and arrivals[order[nxt]] <= now:
            i = int(order[nxt])
            p = problems[i]
            x = np.empty(p.n)
            t = ctx.submit(HostCSR.from_problem(p), np.ascontiguousarray(p.b, dtype=np.float64), x,
                           precision=precision)
            pending[t] = (i, float(arrivals[i]), x)
            nxt += 1
        drain()
        if nxt < n:
            wait = arrivals[order[nxt]] - (time.perf_counter() - t0)
            time.sleep(min(max(wait, 0.0), poll_s) if pending else max(wait, 0.0))
        elif pending:
            time.sleep(poll_s)
    wall = time.perf_counter() - t0
    return {"x": xs, "status": status, "latency_s": lat, "wall_s": wall, "device_ms": dev_ms,
            "queue": ctx.queue_stats()}
