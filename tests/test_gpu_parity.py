"""Parity of the CUDA path with the CPU oracle (GPU).

Every call goes through the C ABI (ctypes binding).  Step-level calls are
compared element by element with the oracle's own routines; full solves are
compared on x (relative error), on the F/G split outside the degenerate band
1e-10 ||A^T b||, on the KKT certificate of Eq. 3, and on the pivot trace.
"""
import numpy as np
import pytest

import workloads
from oracle import kkt

pytestmark = pytest.mark.gpu

REL_TOL = 1e-9        # ||x - x*|| / ||x*|| against the FP64 oracle
KKT_FACTOR = 1e-10    # KKT violation <= 1e-10 ||A^T b||


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def ts(torch_cuda):
    import paper_cs_0408029_gb300 as mod

    mod.load()
    return mod


@pytest.fixture(scope="module")
def ctx(ts):
    c = ts.Context(0)
    yield c
    c.close()


def _check_solution(prob, ref, x, inF=None):
    err = np.linalg.norm(x - ref.x) / max(np.linalg.norm(ref.x), 1e-300)
    assert err <= REL_TOL, err
    assert kkt.violation(prob, x) <= KKT_FACTOR * kkt.atb_norm(prob)
    if inF is not None:
        band = 1e-10 * kkt.atb_norm(prob)
        y = kkt.dual(prob, ref.x)
        clear = (np.abs(ref.x) > band) | (np.abs(y) > band)
        assert np.array_equal(inF[clear], ref.inF[clear])
    return err


# ---------------------------------------------------------------------------
# step level


@pytest.mark.parametrize("m,n,density", [(300, 200, 0.05), (1500, 1100, 0.01), (70, 33, 0.3)])
def test_gram_bit_exact(ts, ctx, torch_cuda, oracle_mod, m, n, density):
    """A^T A and A^T b: same products summed in the same (ascending row)
    order as the oracle's column dot products, so FP64 results are equal bit
    for bit, and the FP32 copy is the rounding of that value."""
    torch = torch_cuda
    p = workloads.random_sparse(m, n, density, seed=m + n)
    A = ts.DeviceCSR.from_problem(p)
    b = torch.as_tensor(p.b, device="cuda")
    g_ref = oracle_mod.gram(p)
    c_ref = oracle_mod.atb(p)
    G, ldg, c = ts.Context.gram(ctx, A, b, precision=ts.FP64)
    Gh = G.cpu().numpy()[:, :n].T  # Gh[i, j] = G(i, j)
    lower = np.tril(np.ones((n, n), dtype=bool))
    assert np.array_equal(Gh[lower], g_ref[lower])
    assert np.array_equal(c.cpu().numpy(), c_ref)
    G32, _, _ = ctx.gram(A, b, precision=ts.MIXED)
    assert np.array_equal(G32.cpu().numpy()[:, :n].T[lower], g_ref.astype(np.float32)[lower])


def test_gather_exact(ts, ctx, torch_cuda):
    torch = torch_cuda
    rng = np.random.default_rng(3)
    n = 300
    g = rng.standard_normal((n, n))
    ldg = 320
    G = torch.zeros((n, ldg), dtype=torch.float64, device="cuda")
    G[:, :n] = torch.as_tensor(g.T, device="cuda")  # column j of g in row j
    F = np.sort(rng.choice(n, 137, replace=False)).astype(np.int32)
    S = ctx.gather(G, ldg, torch.as_tensor(F, device="cuda"), precision=ts.FP64)
    got = S.cpu().numpy().T  # got[a, b] = S(a, b)
    want = g[np.ix_(F, F)]
    lower = np.tril(np.ones((137, 137), dtype=bool))
    assert np.array_equal(got[lower], want[lower])


@pytest.mark.parametrize("k", [1, 31, 32, 33, 63, 64, 65, 130, 257, 700])
def test_cholesky_and_solve(ts, ctx, torch_cuda, oracle_mod, k):
    torch = torch_cuda
    rng = np.random.default_rng(k)
    a = rng.standard_normal((k + 40, k))
    s = a.T @ a
    L_ref = oracle_mod.cholesky(s)
    rhs = rng.standard_normal(k)
    x_ref = oracle_mod.cholesky_solve(L_ref, rhs)
    lower = np.tril(np.ones((k, k), dtype=bool))
    # forward error of L (FP64 only: the FP32 factor's forward error grows
    # like cond(S) u) and backward error ||L L^T - S|| / ||S|| (both)
    for prec, dt, tol_l, tol_back, tol_x in ((ts.FP64, torch.float64, 1e-11, 1e-13, 1e-9),
                                             (ts.MIXED, torch.float32, None, 2e-5, 1e-2)):
        S = torch.as_tensor(s.T.copy(), dtype=dt, device="cuda")  # column-major, lds = k
        st, info = ctx.cholesky(S, k, k, precision=prec)
        assert st == ts.OK and info == 0
        L = np.tril(S.cpu().numpy().astype(np.float64).T)
        if tol_l is not None:
            assert np.abs(L[lower] - L_ref[lower]).max() <= tol_l * np.abs(L_ref).max()
        assert np.abs(L @ L.T - s).max() <= tol_back * np.abs(s).max()
        r = torch.as_tensor(rhs, dtype=dt, device="cuda")
        ctx.chol_solve(S, k, k, r, precision=prec)
        x = r.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(x - x_ref) <= tol_x * np.linalg.norm(x_ref)


def test_cholesky_reports_not_pd(ts, ctx, torch_cuda):
    torch = torch_cuda
    s = np.eye(80)
    s[50, 50] = -1.0
    S = torch.as_tensor(s, device="cuda")
    st, info = ctx.cholesky(S, 80, 80, precision=ts.FP64)
    assert st == ts.ENOTPD and info == 51


@pytest.mark.parametrize("trans", [0, 1])
def test_spmv(ts, ctx, torch_cuda, trans):
    torch = torch_cuda
    p = workloads.random_sparse(500, 300, 0.03, seed=11)
    A = ts.DeviceCSR.from_problem(p)
    a = p.dense()
    rng = np.random.default_rng(5)
    x = rng.standard_normal(500 if trans else 300)
    z = rng.standard_normal(300 if trans else 500)
    out = ctx.spmv(A, trans, -1.5, torch.as_tensor(x, device="cuda"), 0.5,
                   torch.as_tensor(z, device="cuda")).cpu().numpy()
    want = -1.5 * ((a.T if trans else a) @ x) + 0.5 * z
    np.testing.assert_allclose(out, want, rtol=1e-13, atol=1e-13)


# ---------------------------------------------------------------------------
# whole solves


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_plain_single_600x400(ts, ctx, oracle_mod, precision):
    p = workloads.plain_single()
    ref = oracle_mod.bpp_solve(p)
    x, y, inF, trace, info = ctx.solve_ex(ts.HostCSR.from_problem(p), p.b, precision=precision)
    _check_solution(p, ref, x, inF)
    # the pivot path (integer decisions of the exchange rule) matches the oracle
    assert np.array_equal(trace, ref.trace)
    assert info.iters == ref.iters


@pytest.mark.parametrize("m,n,density,seed", [(1500, 1000, 0.02, 1), (900, 700, 0.05, 2),
                                              (2600, 1300, 0.004, 3), (130, 97, 0.2, 4)])
def test_random_sparse_tiles_and_tails(ts, ctx, oracle_mod, m, n, density, seed):
    """Sizes that span several factor / solve tiles and a ragged tail."""
    p = workloads.random_sparse(m, n, density, seed=seed, zero_frac=0.4, noise=0.05)
    ref = oracle_mod.bpp_solve(p)
    for precision in ("mixed", "fp64"):
        x, y, inF, trace, info = ctx.solve_ex(ts.HostCSR.from_problem(p), p.b, precision=precision)
        _check_solution(p, ref, x, inF)
        assert np.array_equal(trace, ref.trace), precision


def _worked_fallback_problem():
    """The 4 x 3 example worked by hand in tests/test_oracle.py: with no
    backup exchanges the second and third pivots are single exchanges that
    move index 2 (the larger of the tied infeasible {1, 2}) and then 1."""
    a = np.array([[1.0, -1.0, -1.0], [0.0, 1.0, 1.0], [0.0, 1.0, -1.0], [0.0, 0.0, 0.0]])
    b = np.array([2.0, 1.0, 0.0, 5.0])
    return workloads.dense_to_csr(a, b)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_single_exchange_worked_example(ts, ctx, oracle_mod, precision):
    """Section 2, algorithm box: once the backup counter is spent, only the
    infeasible variable with the largest index changes sides."""
    p = _worked_fallback_problem()
    big = np.iinfo(np.int64).max
    expect = np.array([[1, big, 0, 0, 1, -1], [2, 1, 0, 2, 2, 2], [1, 1, 0, 2, 3, 1]])
    ref = oracle_mod.bpp_solve(p, p_max=0)
    assert np.array_equal(ref.trace, expect)
    x, y, inF, trace, info = ctx.solve_ex(ts.HostCSR.from_problem(p), p.b, precision=precision,
                                          p_max=0)
    assert np.array_equal(trace, expect)
    np.testing.assert_allclose(x, [3.0, 0.5, 0.5], rtol=1e-13)
    assert inF.all()


def _fallback_cases():
    prob, _, _ = workloads.conditioned_dense(400, 300, 3e3, seed=4, active_frac=1.0)
    return [("plain_single_600x400", workloads.plain_single()),
            ("conditioned_400x300", workloads.dense_to_csr(prob.a, prob.b))]


@pytest.mark.parametrize("case", [0, 1])
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_single_exchange_trace_matches_oracle(ts, ctx, oracle_mod, case, precision):
    """p_max = 0 makes every pivot whose infeasible count does not drop a
    single exchange.  On the 600 x 400 config (3 such pivots) and on a
    conditioned 400 x 300 problem whose final F spans two 128-column blocks
    and a ragged tail (15 of 31 pivots), the GPU's pivot trace, including the
    index each single exchange moved, equals the oracle's."""
    name, p = _fallback_cases()[case]
    ref = oracle_mod.bpp_solve(p, p_max=0)
    singles = ref.trace[:, 3] == 2
    assert singles.sum() >= 3
    x, y, inF, trace, info = ctx.solve_ex(ts.HostCSR.from_problem(p), p.b, precision=precision,
                                          p_max=0)
    _check_solution(p, ref, x, inF)
    assert np.array_equal(trace, ref.trace), name
    assert np.array_equal(trace[singles, 5], ref.trace[singles, 5])


@pytest.mark.parametrize("kw", [{}, {"precision": "fp64"}, {"path": "lsqr"}])
def test_info_quality_fields(ts, ctx, kw):
    """info.kkt_viol is the violation of Eq. 3 at the returned x over
    ||A^T b||, computed on the device; it must agree with the CPU
    certificate (scipy products) to rounding.  info.rel_resid_change is the
    residual change of the last refinement correction: small once the
    refinement has converged, 0 on the plain FP64 path, which takes none."""
    p = workloads.plain_single()
    x, info = ctx.solve(ts.HostCSR.from_problem(p), p.b, **kw)
    want = kkt.violation(p, x) / kkt.atb_norm(p)
    assert want <= KKT_FACTOR
    assert info.kkt_viol <= KKT_FACTOR
    assert abs(info.kkt_viol - want) <= 1e-14
    if kw.get("precision") == "fp64":
        assert info.rel_resid_change == 0.0
    else:
        assert 0.0 < info.rel_resid_change <= 1e-8


def test_info_quality_fields_zero_pivots(ts, ctx):
    """A^T b <= 0: x = 0 after no pivot; the certificate is then that of x = 0."""
    rng = np.random.default_rng(40)
    a = np.abs(rng.standard_normal((20, 6)))
    b = -np.abs(rng.standard_normal(20))
    p = workloads.dense_to_csr(a, b)
    x, info = ctx.solve(ts.HostCSR.from_problem(p), p.b)
    assert info.iters == 0 and info.rel_resid_change == 0.0
    assert abs(info.kkt_viol - kkt.violation(p, x) / kkt.atb_norm(p)) <= 1e-15


def test_device_input_matches_host_input(ts, ctx, torch_cuda):
    torch = torch_cuda
    p = workloads.random_sparse(800, 500, 0.02, seed=9)
    xh, _ = ctx.solve(ts.HostCSR.from_problem(p), p.b)
    xd, _ = ctx.solve(ts.DeviceCSR.from_problem(p), torch.as_tensor(p.b, device="cuda"))
    assert np.array_equal(xh, xd.cpu().numpy())


def test_solve_is_deterministic(ts, ctx):
    p = workloads.random_sparse(800, 500, 0.02, seed=10)
    A = ts.HostCSR.from_problem(p)
    x1, _ = ctx.solve(A, p.b)
    x2, _ = ctx.solve(A, p.b)
    assert np.array_equal(x1, x2)


def test_factor_graph_replay_is_bitwise_equal(ts, ctx, oracle_mod):
    """A lane launches a look-ahead factorisation directly the first time it
    meets its key, captures it into a graph the second time and replays the
    graph after that: every solve must be bitwise the one launched directly
    and meet the oracle bar, also with a solve of another size in between."""
    p = workloads.random_sparse(2600, 1300, 0.004, seed=3, zero_frac=0.4, noise=0.05)
    q = workloads.random_sparse(900, 700, 0.01, seed=31)
    ref = oracle_mod.bpp_solve(p)
    A, B = ts.HostCSR.from_problem(p), ts.HostCSR.from_problem(q)
    runs = [ctx.solve_ex(A, p.b) for _ in range(3)]
    xq, _ = ctx.solve(B, q.b)
    runs.append(ctx.solve_ex(A, p.b))
    x0, _, inF0, tr0, _ = runs[0]
    _check_solution(p, ref, x0, inF0)
    assert np.array_equal(tr0, ref.trace)
    for x, _, inF, tr, _ in runs[1:]:
        assert np.array_equal(x, x0) and np.array_equal(inF, inF0) and np.array_equal(tr, tr0)
    xq2, _ = ctx.solve(B, q.b)
    assert np.array_equal(xq, xq2)


def test_in_order_factor_matches_look_ahead(ts, ctx, oracle_mod):
    """Kernel-by-kernel timing runs the factorisation in order, without the
    look-ahead side stream: both schedules must meet the oracle bar and give
    the same pivot trace, and the timing must see all three factor kernels."""
    p = workloads.random_sparse(2600, 1300, 0.004, seed=3, zero_frac=0.4, noise=0.05)
    ref = oracle_mod.bpp_solve(p)
    A = ts.HostCSR.from_problem(p)
    for precision in ("mixed", "fp64"):
        x1, _, inF1, tr1, _ = ctx.solve_ex(A, p.b, precision=precision)
        ctx.profile(True, kernels=True)
        try:
            x2, _, inF2, tr2, _ = ctx.solve_ex(A, p.b, precision=precision)
            stats = ctx.profile_read()
        finally:
            ctx.profile(False)
        for x, inF in ((x1, inF1), (x2, inF2)):
            _check_solution(p, ref, x, inF)
        assert np.array_equal(tr1, tr2) and np.array_equal(tr1, ref.trace)
        for ph in ("factor_diag", "factor_panel", "factor_update"):
            assert stats[ph]["launches"] > 0, ph
        assert stats["factor"]["launches"] == 0


def test_settle_stop_matches_full_refinement(ts, ctx, oracle_mod):
    """Before the last pivot only the signs of x_F and y_G matter (Section 3):
    a pivot's refinement may stop once no decision of the next exchange can
    change.  The pivots, the split and x must be those of refinement to
    rel_tol at every pivot, and the oracle's."""
    p = workloads.random_sparse(2600, 1300, 0.004, seed=3, zero_frac=0.4, noise=0.05)
    ref = oracle_mod.bpp_solve(p)
    A = ts.HostCSR.from_problem(p)
    x1, _, inF1, tr1, i1 = ctx.solve_ex(A, p.b, full_refine=1)
    x2, _, inF2, tr2, i2 = ctx.solve_ex(A, p.b, full_refine=0)
    for x, inF in ((x1, inF1), (x2, inF2)):
        _check_solution(p, ref, x, inF)
    assert np.array_equal(tr1, tr2) and np.array_equal(tr1, ref.trace)
    assert np.array_equal(inF1, inF2)
    assert i2.refine_steps <= i1.refine_steps
    assert np.linalg.norm(x1 - x2) <= 1e-12 * np.linalg.norm(x1)


def test_factor_reuse_matches_refactoring(ts, ctx, oracle_mod):
    """A pivot that moves only a few variables since the last factorisation is
    solved on that factor, bordered by the added columns and with the removed
    ones held at zero by a capacitance correction: the pivots, the split and x
    must equal those of refactoring every pivot (as the paper does), and the
    oracle's."""
    p = workloads.random_sparse(5000, 2500, 0.004, seed=7, zero_frac=0.4, noise=0.05)
    ref = oracle_mod.bpp_solve(p)
    A = ts.HostCSR.from_problem(p)
    x1, _, inF1, tr1, i1 = ctx.solve_ex(A, p.b)
    x2, _, inF2, tr2, i2 = ctx.solve_ex(A, p.b, no_reuse=1)
    assert i1.factor_reuses >= 1 and i2.factor_reuses == 0
    for x, inF in ((x1, inF1), (x2, inF2)):
        _check_solution(p, ref, x, inF)
    assert np.array_equal(tr1, tr2) and np.array_equal(tr1, ref.trace)
    assert np.array_equal(inF1, inF2)
    assert np.linalg.norm(x1 - x2) <= 1e-12 * np.linalg.norm(x2)


def test_fallback_to_fp64_when_the_fp32_factor_fails(ts, ctx):
    """kappa(A) = 1e5 puts kappa(A^T A) = 1e10 beyond an FP32 factor: the
    mixed solve either loses positive definiteness or its refinement
    stagnates, and is redone with the FP64 factor and the same FP64
    refinement, whose error stays near kappa eps (the normal equations alone
    give up to kappa^2 eps, Section 2)."""
    kappa = 1e5
    prob, xs, _ = workloads.conditioned_dense(300, 200, kappa, seed=51)
    p = workloads.dense_to_csr(prob.a, prob.b)
    A = ts.HostCSR.from_problem(p)
    with pytest.raises(ts.TsnnlsError) as err:
        ctx.solve_ex(A, p.b, no_fallback=1)
    assert err.value.status in (ts.ENOCONV, ts.ENOTPD)
    x, _, _, _, info = ctx.solve_ex(A, p.b)
    assert info.fallback_used == 1 and info.precision_used == ts.FP64
    eps = np.finfo(float).eps
    assert np.linalg.norm(x - xs) <= 1e3 * kappa * eps * np.linalg.norm(xs)


@pytest.mark.parametrize("kappa", [1e1, 1e3, 1e5])
def test_accuracy_vs_condition(ts, ctx, kappa):
    """Fig. 1's experiment on the known-solution generator: the plain FP64
    normal equations stay within the paper's c kappa^2 eps (c = 1 here), the
    refined mixed path (FP64 fallback at kappa = 1e5) near kappa eps."""
    eps = np.finfo(float).eps
    prob, xs, _ = workloads.conditioned_dense(240, 160, kappa, seed=53)
    p = workloads.dense_to_csr(prob.a, prob.b)
    A = ts.HostCSR.from_problem(p)
    paths = (("mixed", {}), ("fp64", {"precision": "fp64"}))
    if kappa <= 1e1:  # restarted LSQR needs O(kappa) iterations: past its limits on these dense cases
        paths += (("lsqr", {"path": "lsqr"}),)
    err = {}
    for name, kw in paths:
        x, _ = ctx.solve(A, p.b, **kw)
        err[name] = np.linalg.norm(x - xs) / np.linalg.norm(xs)
    assert err["fp64"] <= kappa ** 2 * eps + 1e-14
    assert err["mixed"] <= 1e3 * kappa * eps
    if "lsqr" in err:
        assert err["lsqr"] <= 1e3 * kappa * eps


@pytest.mark.parametrize("kappa", [1e2, 1e4])
def test_condition_estimate(ts, ctx, kappa):
    """The 1-norm condition estimate of (A^T A)_FF at the last pivot is a
    lower bound of the exact kappa_1 (to rounding) within the usual factor
    of the estimator."""
    prob, _, _ = workloads.conditioned_dense(300, 200, kappa, seed=52)
    p = workloads.dense_to_csr(prob.a, prob.b)
    A = ts.HostCSR.from_problem(p)
    _, _, inF, _, info = ctx.solve_ex(A, p.b, cond_est=1)
    af = prob.a[:, inF]
    g = af.T @ af
    exact = np.linalg.norm(g, 1) * np.linalg.norm(np.linalg.inv(g), 1)
    assert exact / 10 <= info.cond_est <= 1.05 * exact, (info.cond_est, exact)
    _, _, _, _, info0 = ctx.solve_ex(A, p.b)
    assert info0.cond_est == 0.0


# ---------------------------------------------------------------------------
# degenerate and special cases


def test_nonpositive_atb_zero_iterations(ts, ctx):
    rng = np.random.default_rng(40)
    a = np.abs(rng.standard_normal((20, 6)))
    b = -np.abs(rng.standard_normal(20))
    p = workloads.dense_to_csr(a, b)
    x, y, inF, trace, info = ctx.solve_ex(ts.HostCSR.from_problem(p), p.b)
    assert info.iters == 0 and np.all(x == 0) and not inF.any()
    np.testing.assert_allclose(y, -(a.T @ b), rtol=1e-14)


def test_single_column(ts, ctx):
    rng = np.random.default_rng(43)
    a = rng.standard_normal((7, 1))
    b = a[:, 0] * 2.5 + 0.1 * rng.standard_normal(7)
    p = workloads.dense_to_csr(a, b)
    x, _ = ctx.solve(ts.HostCSR.from_problem(p), p.b, precision="fp64")
    np.testing.assert_allclose(x, [float(a[:, 0] @ b) / float(a[:, 0] @ a[:, 0])], rtol=1e-13)


def test_orthogonal_columns(ts, ctx):
    rng = np.random.default_rng(42)
    q, _ = np.linalg.qr(rng.standard_normal((30, 10)))
    a = q * rng.uniform(0.5, 3.0, 10)
    b = rng.standard_normal(30)
    p = workloads.dense_to_csr(a, b)
    expect = np.maximum(0.0, a.T @ b) / np.sum(a * a, axis=0)
    x, _ = ctx.solve(ts.HostCSR.from_problem(p), p.b)
    np.testing.assert_allclose(x, expect, rtol=1e-10, atol=1e-13)


def test_empty_rows_and_degenerate(ts, ctx, oracle_mod):
    prob, xs, ys = workloads.conditioned_dense(50, 30, 5.0, seed=45, zero_frac=0.5,
                                               active_frac=0.4)
    a = np.vstack([prob.a, np.zeros((5, 30))])  # empty rows
    b = np.concatenate([prob.b, np.zeros(5)])
    p = workloads.dense_to_csr(a, b)
    x, _ = ctx.solve(ts.HostCSR.from_problem(p), p.b)
    np.testing.assert_allclose(x, xs, rtol=0, atol=1e-10)


def test_bounded_wait_reports_timeout(ts, ctx):
    """A device wait on a flag that nothing sets gives up after its bound and
    reports TSNNLS_ETIMEOUT; the device stays usable for the next solve."""
    assert ts.wait_probe(1 << 16) == ts.ETIMEOUT
    assert ts.wait_probe(-1) == ts.EINVAL
    assert ts.wait_probe(ts.WAIT_PROBE_MAX_POLLS + 1) == ts.EINVAL  # no unbounded waits
    p = workloads.plain_single()
    x, info = ctx.solve(ts.HostCSR.from_problem(p), p.b)
    assert info.status == ts.OK and np.all(np.isfinite(x))


def test_invalid_inputs(ts, ctx):
    p = workloads.random_sparse(40, 20, 0.2, seed=3)
    A = ts.HostCSR.from_problem(p)
    bad = ts.HostCSR(p.m, p.n, p.row_ptr, p.col_idx.copy(), p.val)
    r0, r1 = int(p.row_ptr[0]), int(p.row_ptr[1])
    assert r1 - r0 >= 2
    bad.col_idx[r0], bad.col_idx[r0 + 1] = bad.col_idx[r0 + 1], bad.col_idx[r0]  # unsorted
    _, info = ctx.solve(bad, p.b, raise_on_error=False)
    assert info.status == ts.EINVAL
    oob = ts.HostCSR(p.m, p.n, p.row_ptr, p.col_idx.copy(), p.val)
    oob.col_idx[-1] = p.n  # out of range
    _, info = ctx.solve(oob, p.b, raise_on_error=False)
    assert info.status == ts.EINVAL
    sq = ts.HostCSR(20, 20, p.row_ptr[:21], p.col_idx, p.val)  # m == n
    _, info = ctx.solve(sq, p.b[:20], raise_on_error=False)
    assert info.status == ts.EINVAL
    nan_b = p.b.copy()
    nan_b[3] = np.nan
    _, info = ctx.solve(A, nan_b, raise_on_error=False)
    assert info.status == ts.EINVAL
    # the context stays usable
    x, _ = ctx.solve(A, p.b)
    assert np.isfinite(x).all()


def test_admission_budget(ts):
    p = workloads.random_sparse(300, 200, 0.05, seed=7)
    with ts.Context(0, hbm_budget=1 << 16) as small:
        _, info = small.solve(ts.HostCSR.from_problem(p), p.b, raise_on_error=False)
        assert info.status == ts.EADMIT
