"""The bounds-checked build (libtsnnls_check.so, -DTSNNLS_CHECK), GPU.

Each case runs in a child process with TSNNLS_CHECK=1 so that the checked
library is the one loaded.  On valid inputs every path must give the
oracle's answer with no index outside its buffer.  On an out-of-range index
that only the kernel sees (a column index of a device CSR handed to
tsnnls_spmv, an F entry handed to tsnnls_gather) the call must return
TSNNLS_EBOUNDS and name the site.  Those inputs sit inside buffers
allocated larger than the bound being checked, so even a missed check
would read memory the process owns."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, sys
import numpy as np, torch
sys.path.insert(0, ROOT)
import paper_cs_0408029_gb300 as ts, workloads, oracle
assert ts.check_build()
out = {}
with ts.Context(0) as ctx:
    # valid inputs through every path: oracle answer, nothing reported
    cases = [("factor", workloads.random_sparse(900, 600, 0.02, seed=41), {}),
             ("sparse", workloads.grid_sparse(24), {"path": "sparse"}),
             ("lsqr", workloads.random_sparse(700, 400, 0.03, seed=42), {"path": "lsqr"})]
    for name, p, kw in cases:
        ref = oracle.bpp_solve(p)
        for prec in ("mixed", "fp64"):
            x, info = ctx.solve(ts.HostCSR.from_problem(p), p.b, precision=prec, **kw)
            err = float(np.linalg.norm(x - ref.x) / max(np.linalg.norm(ref.x), 1e-300))
            out[f"{name}_{prec}"] = [int(info.status), err, ts.check_report()[0]]
    probs = workloads.batched_uneven(seed=43, count=12, n_lo=16, n_hi=300)
    a = [torch.as_tensor(q.a, device="cuda") for q in probs]
    b = [torch.as_tensor(q.b, device="cuda") for q in probs]
    xs = [torch.empty(q.n, dtype=torch.float64, device="cuda") for q in probs]
    st, _, _ = ctx.solve_batch_dense(a, b, xs, precision="mixed")
    out["batch"] = [int(st), ts.check_report()[0]]
    # an out-of-range column index (5 with n = 3); x has 16 entries
    A = ts.DeviceCSR(4, 3, torch.tensor([0, 1, 2, 3, 4], dtype=torch.int64, device="cuda"),
                     torch.tensor([0, 1, 5, 2], dtype=torch.int32, device="cuda"),
                     torch.ones(4, dtype=torch.float64, device="cuda"))
    x = torch.ones(16, dtype=torch.float64, device="cuda")
    try:
        ctx.spmv(A, 0, 1.0, x)
        out["spmv_bad"] = [0, ""]
    except ts.TsnnlsError as e:
        out["spmv_bad"] = [e.status, ts.check_report()[1]]
    # an F entry past the leading dimension (10 with ldg = 8); G has 16 columns
    G = torch.eye(8, 16, dtype=torch.float32, device="cuda").t().contiguous()
    F = torch.tensor([0, 1, 10], dtype=torch.int32, device="cuda")
    try:
        ctx.gather(G, 8, F)
        out["gather_bad"] = [0, ""]
    except ts.TsnnlsError as e:
        out["gather_bad"] = [e.status, ts.check_report()[1]]
print("RESULT " + json.dumps(out))
'''


def test_checked_build_parity_and_reports():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    env = dict(os.environ, TSNNLS_CHECK="1")
    code = CHILD.replace("ROOT", repr(ROOT))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("RESULT ")]
    assert r.returncode == 0 and line, r.stdout[-2000:] + r.stderr[-4000:]
    out = json.loads(line[0][7:])
    import paper_cs_0408029_gb300 as ts

    for name in ("factor", "sparse", "lsqr"):
        for prec in ("mixed", "fp64"):
            st, err, hits = out[f"{name}_{prec}"]
            assert st == ts.OK and hits == 0, (name, prec, out[f"{name}_{prec}"])
            assert err <= 1e-9, (name, prec, err)
    assert out["batch"] == [ts.OK, 0]
    st, what = out["spmv_bad"]
    assert st == ts.EBOUNDS and "sparse.cu" in what and "index 5 outside [0, 3)" in what, out["spmv_bad"]
    st, what = out["gather_bad"]
    assert st == ts.EBOUNDS and "dense.cu" in what and "index 10 outside [0, 8)" in what, out["gather_bad"]
