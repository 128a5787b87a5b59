"""The early stop of a pivot's refinement (no GPU).

Before the last pivot only the signs of x_F and y_G after the 1e-12 zeroing
enter the method (Section 3).  The solver stops a pivot's refinement once the
observed contraction rho = ||dx||_inf / ||dx_prev||_inf is <= 0.1 and no entry
lies within its error bound of 0 or +-1e-12:
E = min(0.5, 20 rho) ||dx||_inf + 1e-15 ||x_F||_inf for x_F (the error left
after the step is about rho ||dx|| / (1 - rho) while the contraction holds;
the bound allows 20 times that, at most 0.5 ||dx||_inf), and
c_i E for s_i = a_i^T (b - A x), c = |A|^T |A| 1.  These tests restate that rule on top
of an FP32 factor and FP64 residuals in numpy and check that whenever it
fires, every decision equals the one of the exact FP64 solution, and that it
does fire well before full accuracy on ordinary problems.
"""
import numpy as np
import pytest
import scipy.linalg

import workloads

TOL = 1e-12


def _categories(v):
    return np.where(np.abs(v) < TOL, 0, np.sign(v)).astype(int)


def _refine_until_settled(a, b, F, max_steps=30):
    """Refinement of min ||A_F x - b|| on an FP32 Cholesky factor with FP64
    residuals; returns (x on all columns, s = A^T (b - A x), steps) at the
    first step the rule fires, or None."""
    n = a.shape[1]
    af = a[:, F]
    g32 = (af.T @ af).astype(np.float32)
    l32 = scipy.linalg.cholesky(g32, lower=True)

    def solve32(v):
        y = scipy.linalg.solve_triangular(l32, v.astype(np.float32), lower=True)
        return scipy.linalg.solve_triangular(l32.T, y, lower=False).astype(np.float64)

    cbound = np.abs(a).T @ (np.abs(a) @ np.ones(n))
    x = np.zeros(n)
    s = a.T @ b
    prev = None
    for step in range(1, max_steps + 1):
        dx = solve32(s[F])
        x[F] += dx
        s = a.T @ (b - a @ x)
        d = np.max(np.abs(dx))
        xn = np.max(np.abs(x[F]))
        if prev is not None and d <= 0.1 * prev:
            E = min(0.5, 20.0 * d / prev) * d + 1e-15 * xn
            inF = np.zeros(n, dtype=bool)
            inF[F] = True
            v = np.where(inF, np.abs(x), np.abs(s))
            e = np.where(inF, E, cbound * E)
            if np.all((v >= TOL + e) | (v + e < TOL)):
                return x, s, step
        prev = d
    return None


def _exact(a, b, F):
    n = a.shape[1]
    x = np.zeros(n)
    x[F] = np.linalg.lstsq(a[:, F], b, rcond=None)[0]
    return x, a.T @ (b - a @ x)


@pytest.mark.parametrize("seed", range(6))
def test_settled_decisions_equal_exact_ones(seed):
    rng = np.random.default_rng(100 + seed)
    p = workloads.random_sparse(400, 160, 0.05, seed=200 + seed, zero_frac=0.4, noise=0.05)
    a = p.dense()
    # an intermediate pivot: a random F of half the columns
    F = np.sort(rng.permutation(p.n)[: p.n // 2])
    got = _refine_until_settled(a, p.b, F)
    assert got is not None, "the rule never fired"
    x, s, steps = got
    assert steps < 30
    xe, se = _exact(a, p.b, F)
    inF = np.zeros(p.n, dtype=bool)
    inF[F] = True
    assert np.array_equal(_categories(x[inF]), _categories(xe[inF]))
    assert np.array_equal(_categories(-s[~inF]), _categories(-se[~inF]))


def test_rule_fires_after_one_correction_on_a_wide_sweep():
    """Random intermediate pivots of well-conditioned sparse problems (an FP32
    factor leaves about 1e-6 relative error): the rule fires after the first
    correction, and every decision equals the exact solution's."""
    fired_early = 0
    for seed in range(30):
        rng = np.random.default_rng(300 + seed)
        p = workloads.random_sparse(300, 140, 0.06, seed=400 + seed, zero_frac=0.4, noise=0.05)
        a = p.dense()
        F = np.sort(rng.permutation(p.n)[: int(rng.integers(20, p.n))])
        got = _refine_until_settled(a, p.b, F)
        assert got is not None, seed
        x, s, steps = got
        fired_early += steps <= 2
        xe, se = _exact(a, p.b, F)
        inF = np.zeros(p.n, dtype=bool)
        inF[F] = True
        assert np.array_equal(_categories(x[inF]), _categories(xe[inF])), seed
        assert np.array_equal(_categories(-s[~inF]), _categories(-se[~inF])), seed
    assert fired_early >= 25


@pytest.mark.parametrize("kappa", [1e1, 1e2, 1e3])
def test_rule_on_conditioned_problems(kappa):
    """Harder conditioning slows the contraction; when the rule fires the
    decisions still match, and it fires before the refinement would reach
    1e-14 of x (the solver's full-accuracy target)."""
    prob, _, _ = workloads.conditioned_dense(240, 120, kappa, seed=61)
    a, b = prob.a, prob.b
    F = np.arange(0, 120, 2)
    got = _refine_until_settled(a, b, F)
    assert got is not None
    x, s, steps = got
    xe, se = _exact(a, b, F)
    inF = np.zeros(120, dtype=bool)
    inF[F] = True
    assert np.array_equal(_categories(x[inF]), _categories(xe[inF]))
    assert np.array_equal(_categories(-s[~inF]), _categories(-se[~inF]))
    assert np.max(np.abs(x[F] - xe[F])) > 1e-14 * np.max(np.abs(xe[F])) or steps <= 3


def test_rule_does_not_fire_on_a_tie_with_the_threshold():
    """An entry of x_F sitting at 1e-12 (the zeroing threshold) can never be
    settled, so the pivot refines on (to rel_tol in the solver)."""
    rng = np.random.default_rng(7)
    a = rng.standard_normal((60, 20))
    x_true = rng.uniform(0.5, 1.0, 20)
    x_true[3] = TOL  # exactly at the threshold
    b = a @ x_true
    F = np.arange(20)
    assert _refine_until_settled(a, b, F) is None
