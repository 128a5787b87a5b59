"""The sparse path: supernodal Cholesky of the sparse (A^T A)_FF (GPU).

Every solve goes through the C ABI with path = TSNNLS_PATH_SPARSE and is
compared with the CPU oracle (dense FP64 Cholesky of the same block, Section
2's method): x within 1e-9, the KKT certificate of Eq. 3, the F/G split
outside the degenerate band, and the pivot trace.  The workload is the grid
problem whose A^T A is below 1 % dense; general sparse and dense-ish Grams
must also come out right (with more fill).
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
    ctx = ts.Context(0)
    yield ts, ctx, torch
    ctx.close()


def _check(p, ref, x, inF):
    err = np.linalg.norm(x - ref.x) / np.linalg.norm(ref.x)
    assert err <= 1e-9, err
    assert kkt.violation(p, x) <= 1e-10 * kkt.atb_norm(p)
    band = 1e-10 * kkt.atb_norm(p)
    y = kkt.dual(p, ref.x)
    clear = (np.abs(ref.x) > band) | (np.abs(y) > band)
    assert np.array_equal(inF[clear], ref.inF[clear])


def _cases():
    return [workloads.grid_sparse(16, seed=11), workloads.grid_sparse(40, seed=12),
            workloads.plain_single(),
            workloads.random_sparse(900, 700, 0.05, seed=2, zero_frac=0.4, noise=0.05)]


@pytest.mark.parametrize("case", range(4))
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_sparse_path_matches_oracle(env, oracle_mod, case, precision):
    ts, ctx, _ = env
    p = _cases()[case]
    ref = oracle_mod.bpp_solve(p)
    x, y, inF, trace, info = ctx.solve_ex(ts.HostCSR.from_problem(p), p.b, precision=precision,
                                          path="sparse")
    assert info.path_used == ts.PATH_SPARSE
    _check(p, ref, x, inF)
    assert np.array_equal(trace, ref.trace)
    assert info.kkt_viol <= 1e-10


def test_sparse_single_exchange_trace(env, oracle_mod):
    """The largest-index fallback (p_max = 0) through the sparse factor."""
    ts, ctx, _ = env
    prob, _, _ = workloads.conditioned_dense(400, 300, 3e3, seed=4, active_frac=1.0)
    p = workloads.dense_to_csr(prob.a, prob.b)
    ref = oracle_mod.bpp_solve(p, p_max=0)
    x, y, inF, trace, info = ctx.solve_ex(ts.HostCSR.from_problem(p), p.b, p_max=0, path="sparse")
    _check(p, ref, x, inF)
    assert np.array_equal(trace, ref.trace)


def test_sparse_equals_dense_path_and_is_deterministic(env):
    ts, ctx, torch = env
    p = workloads.grid_sparse(48, seed=13)
    A = ts.HostCSR.from_problem(p)
    xs, _, fs, trs, _ = ctx.solve_ex(A, p.b, path="sparse")
    xd, _, fd, trd, _ = ctx.solve_ex(A, p.b, path="factor")
    assert np.array_equal(trs, trd) and np.array_equal(fs, fd)
    assert np.linalg.norm(xs - xd) <= 1e-12 * np.linalg.norm(xd)
    xs2, _ = ctx.solve(A, p.b, path="sparse")
    assert np.array_equal(xs, xs2)
    Ad = ts.DeviceCSR.from_problem(p)
    xdev, _ = ctx.solve(Ad, torch.as_tensor(p.b, device="cuda"), path="sparse")
    assert np.array_equal(xs, xdev.cpu().numpy())


def test_sparse_full_size_grid(env):
    """256 x 256 grid (n = 65536, 131072 rows): no oracle at this size; the
    KKT certificate of Eq. 3 and agreement of the mixed and FP64 sparse paths."""
    ts, ctx, torch = env
    p = workloads.grid_sparse(256)
    A = ts.DeviceCSR.from_problem(p)
    b = torch.as_tensor(p.b, device="cuda")
    xm, im = ctx.solve(A, b, path="sparse")
    x64, i64 = ctx.solve(A, b, path="sparse", precision="fp64")
    xm, x64 = xm.cpu().numpy(), x64.cpu().numpy()
    atb = kkt.atb_norm(p)
    assert kkt.violation(p, xm) <= 1e-10 * atb
    assert kkt.violation(p, x64) <= 1e-10 * atb
    assert np.linalg.norm(xm - x64) <= 1e-9 * np.linalg.norm(x64)
    assert im.iters == i64.iters and im.path_used == ts.PATH_SPARSE


def _block_diagonal(p1, p2):
    """A = diag(A1, A2) with b = (b1, b2): two independent problems, so the
    Gram pattern has two components and the supernodal tree two roots."""
    return workloads.CSRProblem(
        m=p1.m + p2.m, n=p1.n + p2.n,
        row_ptr=np.concatenate([p1.row_ptr, p1.row_ptr[-1] + p2.row_ptr[1:]]).astype(np.int64),
        col_idx=np.concatenate([p1.col_idx, p2.col_idx + p1.n]).astype(np.int32),
        val=np.concatenate([p1.val, p2.val]), b=np.concatenate([p1.b, p2.b]),
        x_planted=np.concatenate([p1.x_planted, p2.x_planted]), name="block_diagonal")


def test_sparse_disconnected_gram(env, oracle_mod):
    """Two components: a forest of supernodal trees, each root taken by depth
    0 in the backward solve's order; against the oracle, trace included."""
    ts, ctx, _ = env
    p = _block_diagonal(workloads.grid_sparse(12, seed=21), workloads.grid_sparse(10, seed=22))
    _, parent, _ = ts.sparse_analyze(p.m, p.n, p.row_ptr, p.col_idx)
    assert (parent < 0).sum() >= 2  # the elimination forest has a root per component
    ref = oracle_mod.bpp_solve(p)
    for precision in ("mixed", "fp64"):
        x, y, inF, trace, info = ctx.solve_ex(ts.HostCSR.from_problem(p), p.b, precision=precision,
                                              path="sparse")
        _check(p, ref, x, inF)
        assert np.array_equal(trace, ref.trace)


def test_sparse_shared_update_matrices_match_dense_path(env):
    """A 96 x 96 grid, whose tallest supernodes have update matrices of three
    and more 128 x 128 blocks (shared out to waiting CTAs in the FP32
    factor): the same trace and F as the dense path, x within 1e-12, and
    bitwise repeatable."""
    ts, ctx, _ = env
    p = workloads.grid_sparse(96, seed=23)
    _, _, st = ts.sparse_analyze(p.m, p.n, p.row_ptr, p.col_idx)
    # the tallest supernode (at most 64 columns) has more than 128 rows below:
    # its update matrix spans 2 x 2 block rows, three 128 x 128 blocks or more
    assert st["max_height"] > 128 + 64
    A = ts.HostCSR.from_problem(p)
    xs, _, fs, trs, _ = ctx.solve_ex(A, p.b, path="sparse")
    xd, _, fd, trd, _ = ctx.solve_ex(A, p.b, path="factor")
    assert np.array_equal(trs, trd) and np.array_equal(fs, fd)
    assert np.linalg.norm(xs - xd) <= 1e-12 * np.linalg.norm(xd)
    xs2, _ = ctx.solve(A, p.b, path="sparse")
    assert np.array_equal(xs, xs2)
    assert kkt.violation(p, xs) <= 1e-10 * kkt.atb_norm(p)
