"""The algebra of reusing a factor across pivots (no GPU).

The solver keeps the Cholesky factor L of G_BB for an earlier set B and
solves the system of a new set F' = (B \\ R) + A with a bordered factor for
the added columns and a capacitance correction that holds the removed ones
at zero.  Restated here in numpy (FP64), it must give the solution of
G_F'F' x = w_F' computed directly, for additions only, removals only, both,
and neither.
"""
import numpy as np
import pytest
import scipy.linalg


def _bordered_solver(G, B, A, R_pos):
    """Return solve(w) for w over U = B + A (R entries ignored) following the
    solver's steps; B, A index lists into G, R_pos positions within B."""
    L = np.linalg.cholesky(G[np.ix_(B, B)])
    a, kb = len(A), len(B)
    if a:
        Pt = scipy.linalg.solve_triangular(L, G[np.ix_(B, A)], lower=True)  # P^T = L^-1 G_BA
        Q = np.linalg.cholesky(G[np.ix_(A, A)] - Pt.T @ Pt)
    u = kb + a

    def h_solve(w):
        yB = scipy.linalg.solve_triangular(L, w[:kb], lower=True)
        z = np.zeros(u)
        if a:
            t = w[kb:] - Pt.T @ yB
            zA = scipy.linalg.cho_solve((Q, True), t)
            yB = yB - Pt @ zA
            z[kb:] = zA
        z[:kb] = scipy.linalg.solve_triangular(L.T, yB, lower=False)
        return z

    r = len(R_pos)
    if r:
        Z = np.column_stack([h_solve(np.eye(u)[:, p]) for p in R_pos])
        C = 0.5 * (Z[R_pos, :] + Z[R_pos, :].T)
        Lc = np.linalg.cholesky(C)

    def solve(w):
        w = w.copy()
        w[R_pos] = 0.0
        z = h_solve(w)
        if r:
            z -= Z @ scipy.linalg.cho_solve((Lc, True), z[R_pos])
        return z

    return solve


@pytest.mark.parametrize("na,nr", [(0, 0), (3, 0), (0, 4), (5, 2), (1, 5)])
def test_bordered_solve_equals_direct(na, nr):
    rng = np.random.default_rng(10 * na + nr)
    n = 60
    M = rng.standard_normal((120, n))
    G = M.T @ M
    perm = rng.permutation(n)
    B = np.sort(perm[:40])
    outside = np.sort(perm[40:])
    A = np.sort(outside[:na])
    R_pos = np.sort(rng.permutation(len(B))[:nr])
    Fp = np.array(sorted(set(B) - set(B[R_pos]) | set(A)))
    U = np.concatenate([B, A])
    w = rng.standard_normal(len(U))
    z = _bordered_solver(G, B, A, list(R_pos))(w)
    # z holds zeros on R and the solution of G_F'F' x = w_F' elsewhere
    np.testing.assert_allclose(z[R_pos], 0.0, atol=1e-10)
    keep = np.setdiff1d(np.arange(len(U)), R_pos)
    x_direct = np.linalg.solve(G[np.ix_(U[keep], U[keep])], w[keep])
    np.testing.assert_allclose(z[keep], x_direct, rtol=1e-9, atol=1e-12)
    assert set(U[keep]) == set(Fp)


def test_capacitance_block_is_the_inverse_block():
    """C = Z_R equals (H^-1)_RR, so it is symmetric positive definite."""
    rng = np.random.default_rng(3)
    M = rng.standard_normal((50, 20))
    G = M.T @ M
    B = np.arange(20)
    R_pos = [2, 7, 11]
    Hinv = np.linalg.inv(G)
    L = np.linalg.cholesky(G)
    Z = np.column_stack([scipy.linalg.cho_solve((L, True), np.eye(20)[:, p]) for p in R_pos])
    np.testing.assert_allclose(Z[R_pos, :], Hinv[np.ix_(R_pos, R_pos)], rtol=1e-10)
    assert np.all(np.linalg.eigvalsh(Z[R_pos, :]) > 0)
