"""Pins for the CPU oracle (no GPU).

Each test checks the oracle against something other than itself: the
brute-force definition of the LCP solution (Eq. 3), scipy's Lawson-Hanson
NNLS, numpy/LAPACK factorisations, closed forms, constructed solutions with a
known answer, and invariances of Eq. 1.  A plausible slip in the oracle (a
dropped term, a sign, an index, a transposed operand, a wrong exchange rule)
fails at least one of them.
"""
import numpy as np
import pytest
import scipy.optimize

import workloads
from oracle import kkt, lcp_enumerate


def _dense_prob(a, b):
    return workloads.dense_to_csr(a, b)


def _rand_dense(seed, m, n, shift=0.0):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((m, n))
    b = rng.standard_normal(m) + shift
    return a, b


# --------------------------------------------------------------------------
# building blocks against library routines


def test_gram_matches_dense_product(oracle_mod):
    p = workloads.random_sparse(70, 40, 0.1, seed=1)
    a = p.dense()
    np.testing.assert_allclose(oracle_mod.gram(p), a.T @ a, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(oracle_mod.atb(p), a.T @ p.b, rtol=1e-13, atol=1e-13)


def test_gram_handles_empty_rows_and_columns(oracle_mod):
    a = np.zeros((6, 4))
    a[0, 0] = 2.0
    a[3, 2] = -1.0
    a[3, 0] = 0.5
    p = _dense_prob(a, np.arange(6.0))
    np.testing.assert_allclose(oracle_mod.gram(p), a.T @ a)
    np.testing.assert_allclose(oracle_mod.atb(p), a.T @ np.arange(6.0))


def test_cholesky_matches_lapack(oracle_mod):
    rng = np.random.default_rng(2)
    m = rng.standard_normal((50, 30))
    s = m.T @ m
    L = oracle_mod.cholesky(s)
    np.testing.assert_allclose(L, np.linalg.cholesky(s), rtol=1e-11, atol=1e-11)
    rhs = rng.standard_normal(30)
    np.testing.assert_allclose(oracle_mod.cholesky_solve(L, rhs), np.linalg.solve(s, rhs),
                               rtol=1e-10)


def test_cholesky_reports_not_pd(oracle_mod):
    s = np.array([[1.0, 2.0], [2.0, 1.0]])
    with pytest.raises(oracle_mod.OracleError) as e:
        oracle_mod.cholesky(s)
    assert e.value.status == oracle_mod.ENOTPD


def test_qr_lstsq_matches_lapack(oracle_mod):
    a, b = _rand_dense(3, 40, 17)
    np.testing.assert_allclose(oracle_mod.qr_lstsq(a, b), np.linalg.lstsq(a, b, rcond=None)[0],
                               rtol=1e-11, atol=1e-12)


# --------------------------------------------------------------------------
# the BPP solution against the plain definition (enumeration of all splits)


@pytest.mark.parametrize("seed,m,n", [(10, 14, 12), (11, 12, 11), (12, 9, 8), (13, 30, 10),
                                      (14, 13, 12), (15, 6, 5)])
def test_bpp_equals_enumeration(oracle_mod, seed, m, n):
    a, b = _rand_dense(seed, m, n, shift=0.3)
    x_e, y_e, f_e = lcp_enumerate.enumerate_solution(a, b)
    r = oracle_mod.bpp_solve(_dense_prob(a, b))
    np.testing.assert_allclose(r.x, x_e, rtol=1e-10, atol=1e-12)
    band = 1e-10 * np.linalg.norm(a.T @ b)
    clear = (np.abs(x_e) > band) | (np.abs(y_e) > band)
    assert np.array_equal(r.inF[clear], f_e[clear])


def test_bpp_equals_enumeration_sparse(oracle_mod):
    p = workloads.random_sparse(16, 12, 0.3, seed=21)
    x_e, _, _ = lcp_enumerate.enumerate_solution(p.dense(), p.b)
    r = oracle_mod.bpp_solve(p)
    np.testing.assert_allclose(r.x, x_e, rtol=1e-10, atol=1e-12)


def test_enumeration_many_small(oracle_mod):
    for seed in range(100, 140):
        rng = np.random.default_rng(seed)
        n = int(rng.integers(1, 9))
        m = n + int(rng.integers(1, 6))
        a, b = _rand_dense(seed, m, n, shift=float(rng.uniform(-1, 1)))
        x_e, _, _ = lcp_enumerate.enumerate_solution(a, b)
        r = oracle_mod.bpp_solve(_dense_prob(a, b))
        np.testing.assert_allclose(r.x, x_e, rtol=1e-9, atol=1e-11, err_msg=f"seed {seed}")


# --------------------------------------------------------------------------
# against an independent active-set NNLS (Lawson-Hanson, scipy)


@pytest.mark.parametrize("seed,m,n", [(30, 120, 80), (31, 300, 200), (32, 81, 80)])
def test_bpp_matches_lawson_hanson_dense(oracle_mod, seed, m, n):
    a, b = _rand_dense(seed, m, n, shift=0.2)
    x_s, _ = scipy.optimize.nnls(a, b, maxiter=50 * n)
    r = oracle_mod.bpp_solve(_dense_prob(a, b))
    assert np.linalg.norm(r.x - x_s) <= 1e-9 * np.linalg.norm(x_s)


def test_bpp_plain_single_config(oracle_mod):
    """600 x 400, 2 % density: Lawson-Hanson and the KKT certificate agree."""
    p = workloads.plain_single()
    r = oracle_mod.bpp_solve(p)
    x_s, _ = scipy.optimize.nnls(p.dense(), p.b, maxiter=20000)
    assert np.linalg.norm(r.x - x_s) <= 1e-10 * np.linalg.norm(x_s)
    assert kkt.violation(p, r.x) <= 1e-10 * kkt.atb_norm(p)
    assert r.iters > 1
    # the perturbation made a good share of the constraints strictly active
    assert ((r.x == 0) & (r.y > 0)).sum() >= 0.2 * p.n


# --------------------------------------------------------------------------
# closed forms and special cases


def test_nonpositive_atb_gives_zero(oracle_mod):
    rng = np.random.default_rng(40)
    a = np.abs(rng.standard_normal((20, 6)))
    b = -np.abs(rng.standard_normal(20))  # A^T b <= 0 entrywise
    r = oracle_mod.bpp_solve(_dense_prob(a, b))
    assert r.iters == 0
    assert np.all(r.x == 0.0)
    np.testing.assert_allclose(r.y, -(a.T @ b))


def test_unconstrained_nonnegative_equals_lstsq(oracle_mod):
    rng = np.random.default_rng(41)
    a = rng.standard_normal((50, 20))
    xt = rng.uniform(0.5, 1.0, 20)
    b = a @ xt + 1e-3 * rng.standard_normal(50)
    x_ls = np.linalg.lstsq(a, b, rcond=None)[0]
    assert (x_ls > 0).all()
    r = oracle_mod.bpp_solve(_dense_prob(a, b))
    np.testing.assert_allclose(r.x, x_ls, rtol=1e-11)
    assert r.inF.all()


def test_orthogonal_columns_closed_form(oracle_mod):
    rng = np.random.default_rng(42)
    q, _ = np.linalg.qr(rng.standard_normal((30, 10)))
    a = q * rng.uniform(0.5, 3.0, 10)  # orthogonal, not orthonormal, columns
    b = rng.standard_normal(30)
    expect = np.maximum(0.0, a.T @ b) / np.sum(a * a, axis=0)
    r = oracle_mod.bpp_solve(_dense_prob(a, b))
    np.testing.assert_allclose(r.x, expect, rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_single_column(oracle_mod, sign):
    rng = np.random.default_rng(43)
    a = rng.standard_normal((7, 1))
    b = sign * a[:, 0] * 2.5 + 0.1 * rng.standard_normal(7)
    expect = max(0.0, float(a[:, 0] @ b) / float(a[:, 0] @ a[:, 0]))
    r = oracle_mod.bpp_solve(_dense_prob(a, b))
    np.testing.assert_allclose(r.x, [expect], rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("kappa", [10.0, 1e3])
def test_known_solution_construction(oracle_mod, kappa):
    prob, xs, ys = workloads.conditioned_dense(60, 40, kappa, seed=44)
    r = oracle_mod.bpp_solve(_dense_prob(prob.a, prob.b))
    assert np.linalg.norm(r.x - xs) <= 1e-12 * kappa * np.linalg.norm(xs)
    on = ys > 0
    assert np.all(r.x[on] == 0.0) and np.all(~r.inF[on])


def test_degenerate_indices_converge(oracle_mod):
    """x*_i = y*_i = 0 on part of the zero set: the 1e-12 zeroing of Section 2
    keeps the method from passing those indices back and forth."""
    prob, xs, ys = workloads.conditioned_dense(50, 30, 5.0, seed=45, zero_frac=0.5,
                                               active_frac=0.4)
    assert ((xs == 0) & (ys == 0)).sum() >= 5
    r = oracle_mod.bpp_solve(_dense_prob(prob.a, prob.b))
    np.testing.assert_allclose(r.x, xs, rtol=0, atol=1e-11)


@pytest.mark.parametrize("kappa", [1e1, 1e3, 1e5, 1e7])
def test_error_model_normal_equations_vs_final_qr(oracle_mod, kappa):
    """Section 2: the normal-equations error is bounded by about kappa^2 eps
    (c kappa^2 eps with c not large; Fig. 1 fits kappa^2 eps / 10).  The final
    recomputation by QR must not be worse and stays near kappa * eps."""
    eps = np.finfo(float).eps
    prob, xs, _ = workloads.conditioned_dense(80, 70, kappa, seed=46)
    p = _dense_prob(prob.a, prob.b)
    ne = oracle_mod.bpp_solve(p, final_step=oracle_mod.FINAL_NONE)
    qr = oracle_mod.bpp_solve(p, final_step=oracle_mod.FINAL_QR)
    e_ne = np.linalg.norm(ne.x - xs) / np.linalg.norm(xs)
    e_qr = np.linalg.norm(qr.x - xs) / np.linalg.norm(xs)
    assert e_ne <= kappa ** 2 * eps
    assert e_qr <= 1e3 * kappa * eps
    assert e_qr <= 1.5 * e_ne + 1e-14


def test_final_lsqr_agrees_with_final_qr(oracle_mod):
    p = workloads.plain_single()
    a = oracle_mod.bpp_solve(p, final_step=oracle_mod.FINAL_QR)
    b = oracle_mod.bpp_solve(p, final_step=oracle_mod.FINAL_LSQR)
    assert np.linalg.norm(a.x - b.x) <= 1e-12 * np.linalg.norm(a.x)


def test_inner_lsqr_agrees_with_inner_cholesky(oracle_mod):
    p = workloads.random_sparse(300, 120, 0.05, seed=47)
    a = oracle_mod.bpp_solve(p)
    b = oracle_mod.bpp_solve(p, inner=oracle_mod.INNER_LSQR, final_step=oracle_mod.FINAL_LSQR)
    assert np.linalg.norm(a.x - b.x) <= 1e-11 * np.linalg.norm(a.x)
    assert b.lsqr_steps > 0


# --------------------------------------------------------------------------
# invariances of Eq. 1


def test_invariances(oracle_mod):
    rng = np.random.default_rng(50)
    a, b = _rand_dense(50, 90, 60, shift=0.1)
    base = oracle_mod.bpp_solve(_dense_prob(a, b)).x
    scale = oracle_mod.bpp_solve(_dense_prob(a, 3.5 * b)).x
    np.testing.assert_allclose(scale, 3.5 * base, rtol=1e-10, atol=1e-13)
    d = rng.uniform(0.2, 5.0, 60)
    col = oracle_mod.bpp_solve(_dense_prob(a * d, b)).x
    np.testing.assert_allclose(col, base / d, rtol=1e-9, atol=1e-13)
    perm = rng.permutation(60)
    pm = oracle_mod.bpp_solve(_dense_prob(a[:, perm], b)).x
    np.testing.assert_allclose(pm, base[perm], rtol=1e-10, atol=1e-13)
    q, _ = np.linalg.qr(rng.standard_normal((90, 90)))
    rot = oracle_mod.bpp_solve(_dense_prob(q @ a, q @ b)).x
    np.testing.assert_allclose(rot, base, rtol=1e-9, atol=1e-12)
    # appending a column that points uphill leaves x unchanged (its entry is 0)
    r = a @ base - b
    new = r / np.linalg.norm(r) + 0.01 * rng.standard_normal(90)
    assert new @ r > 0
    ext = oracle_mod.bpp_solve(_dense_prob(np.column_stack([a, new]), b)).x
    np.testing.assert_allclose(ext[:60], base, rtol=1e-10, atol=1e-13)
    assert ext[60] == 0.0


# --------------------------------------------------------------------------
# the exchange rule of the algorithm box, read off the trace


def _check_trace(trace, p_max=3):
    p_prev, n_best = p_max, None
    for n_inf, n_before, p_after, branch, _, moved in trace:
        assert (moved >= 0) == (branch == 2)
        if n_best is None:
            assert n_before == np.iinfo(np.int64).max  # N = infinity at the start
        else:
            assert n_before == n_best
        if n_best is None or n_inf < n_best:
            assert branch == 0 and p_after == p_max
            n_best = n_inf
        elif p_prev > 0:
            assert branch == 1 and p_after == p_prev - 1
        else:
            assert branch == 2 and p_after == 0
        p_prev = p_after


def test_exchange_rule_trace(oracle_mod):
    seen = set()
    for seed in range(60, 90):
        p = workloads.random_sparse(150, 120, 0.08, seed=seed, zero_frac=0.5, noise=0.3)
        r = oracle_mod.bpp_solve(p)
        _check_trace(r.trace)
        seen.update(int(t[3]) for t in r.trace)
        # a single exchange moves exactly one variable
        ks = [0] + [int(t[4]) for t in r.trace]
        for i, t in enumerate(r.trace):
            if t[3] == 2:
                assert abs(ks[i + 1] - ks[i]) == 1
        assert kkt.violation(p, r.x) <= 1e-10 * kkt.atb_norm(p)
    assert 0 in seen and 1 in seen


def test_single_exchange_fallback_reaches_solution(oracle_mod):
    """With p_max = 0 every non-decreasing step uses the single-variable
    fallback; the answer must still be the unique solution."""
    p = workloads.random_sparse(150, 120, 0.08, seed=61, zero_frac=0.5, noise=0.3)
    ref = oracle_mod.bpp_solve(p)
    r = oracle_mod.bpp_solve(p, p_max=0)
    _check_trace(r.trace, p_max=0)
    np.testing.assert_allclose(r.x, ref.x, rtol=1e-10, atol=1e-13)


def _worked_fallback_problem():
    """A 4 x 3 problem worked by hand for the single-variable rule.

    Columns a0 = (1,0,0,0), a1 = (-1,1,1,0), a2 = (-1,1,-1,0) give
    A^T A = [[1,-1,-1],[-1,3,1],[-1,1,3]]; b = (2,1,0,5) gives
    c = A^T b = (2,-1,-1).  With p = 0 backup exchanges allowed:

    pivot 1: y = -c = (-2,1,1); infeasible {0}, count 1 < N = inf, so N = 1
             and the full exchange gives F = {0}; x_0 = c_0 / 1 = 2,
             y_1 = y_2 = -1*2 - (-1) = -1.
    pivot 2: infeasible {1, 2}, count 2 >= N = 1 and p = 0, so only the
             largest infeasible index moves: F = {0, 2}.  Then
             [[1,-1],[-1,3]] x_F = (2,-1) gives x_0 = 5/2, x_2 = 1/2, and
             y_1 = -5/2 + 1/2 + 1 = -1.
    pivot 3: infeasible {1}, count 1 >= N: the single exchange moves 1,
             F = {0,1,2}, x = (A^T A)^{-1} c = (3, 1/2, 1/2) > 0: done.

    Every value is a small dyadic rational, so no rounding enters.  Moving
    the smallest infeasible index instead would move 1 at pivot 2 (and
    reach the same x), which only the moved-index column tells apart."""
    a = np.array([[1.0, -1.0, -1.0], [0.0, 1.0, 1.0], [0.0, 1.0, -1.0], [0.0, 0.0, 0.0]])
    b = np.array([2.0, 1.0, 0.0, 5.0])
    return a, b


def test_single_exchange_moves_largest_index_worked_example(oracle_mod):
    a, b = _worked_fallback_problem()
    big = np.iinfo(np.int64).max
    r = oracle_mod.bpp_solve(_dense_prob(a, b), p_max=0, final_step=oracle_mod.FINAL_NONE)
    expect = np.array([[1, big, 0, 0, 1, -1],
                       [2, 1, 0, 2, 2, 2],
                       [1, 1, 0, 2, 3, 1]])
    assert np.array_equal(r.trace, expect)
    np.testing.assert_allclose(r.x, [3.0, 0.5, 0.5], rtol=1e-14)  # square roots round
    # with the backup counter at its default the second pivot is a full exchange
    r3 = oracle_mod.bpp_solve(_dense_prob(a, b), p_max=3, final_step=oracle_mod.FINAL_NONE)
    assert [tuple(t[3:]) for t in r3.trace] == [(0, 1, -1), (1, 3, -1)]
    np.testing.assert_allclose(r3.x, [3.0, 0.5, 0.5], rtol=1e-14)


def _replay_exchange_rule(a, b, trace, p_max, zero_tol=1e-12):
    """Replay the algorithm box of Section 2 from the trace's own decisions,
    recomputing every pivot's x_F (numpy least squares on A_F) and
    y_G = A_G^T (A_F x_F - b) (Eq. 5) without the oracle, and check each row:
    the infeasible count, N and p, the branch, |F| and, for a single
    exchange, that the moved index is the largest infeasible one."""
    n = a.shape[1]
    inF = np.zeros(n, dtype=bool)
    x = np.zeros(n)
    y = -(a.T @ b)
    n_best, p = None, p_max
    for i, (n_inf, n_before, p_after, branch, k, moved) in enumerate(trace):
        infeas = np.nonzero(np.where(inF, x < 0, y < 0))[0]
        assert n_inf == infeas.size, i
        assert n_before == (np.iinfo(np.int64).max if n_best is None else n_best), i
        if n_best is None or infeas.size < n_best:
            n_best, p, want = infeas.size, p_max, 0
        elif p > 0:
            p, want = p - 1, 1
        else:
            want = 2
        assert branch == want and p_after == p, i
        if want == 2:
            assert moved == infeas.max(), i
            inF[infeas.max()] ^= True
        else:
            assert moved == -1, i
            inF[infeas] ^= True
        assert k == inF.sum(), i
        x = np.zeros(n)
        if inF.any():
            x[inF] = np.linalg.lstsq(a[:, inF], b, rcond=None)[0]
        y = a.T @ (a @ x - b)
        y[inF] = 0.0
        x[np.abs(x) < zero_tol] = 0.0
        y[np.abs(y) < zero_tol] = 0.0
    assert not np.where(inF, x < 0, y < 0).any()  # the last pivot is feasible


@pytest.mark.parametrize("m,n,kappa,seed", [(60, 40, 1e3, 2), (30, 20, 3e2, 2),
                                            (200, 150, 1e3, 3), (400, 300, 3e3, 4)])
@pytest.mark.parametrize("p_max", [0, 3])
def test_trace_replays_exchange_rule(oracle_mod, m, n, kappa, seed, p_max):
    """The oracle's trace follows the exchange rule step by step, against x
    and y recomputed in numpy from each pivot's F; with p_max = 0 these
    conditioned problems take the single-variable fallback many times."""
    prob, _, _ = workloads.conditioned_dense(m, n, kappa, seed=seed, active_frac=1.0)
    r = oracle_mod.bpp_solve(_dense_prob(prob.a, prob.b), p_max=p_max)
    _replay_exchange_rule(prob.a, prob.b, r.trace, p_max)
    if p_max == 0:
        assert (r.trace[:, 3] == 2).sum() >= 2


def test_invalid_inputs_rejected(oracle_mod):
    a, b = _rand_dense(70, 5, 5)  # m == n
    with pytest.raises(oracle_mod.OracleError) as e:
        oracle_mod.bpp_solve(_dense_prob(a, b))
    assert e.value.status == oracle_mod.EINVAL
