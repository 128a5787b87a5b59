"""Plain definition of the NNLS solution by enumeration -- TEST INFRASTRUCTURE ONLY.

Eq. 3 (the LCP form of Eq. 1) has exactly one solution when A has full column
rank (A^T A is positive definite, Section 2).  For every complementary split
(F, G) of {0..n-1} the complementary basic solution is x_F from the
unconstrained least-squares problem of Eq. 4 and y_G from Eq. 5; the split is
the answer when x_F >= 0 and y_G >= 0.  This module tries all 2^n splits, so
it is usable for n <= 12 only.  It uses numpy's lstsq as the unconstrained
solver and has no code in common with the C oracle or the CUDA library.
"""
from __future__ import annotations

import itertools

import numpy as np


def enumerate_solution(a: np.ndarray, b: np.ndarray, tol: float = 1e-10):
    """Return (x, y, F-mask) of the feasible complementary basic solution.

    ``tol`` absorbs rounding in the sign tests.  Raises if no split or more
    than one *different* x is feasible (that would contradict uniqueness)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    m, n = a.shape
    if n > 12:
        raise ValueError("enumeration is exponential; n <= 12 only")
    found = []
    for bits in itertools.product((False, True), repeat=n):
        f = np.array(bits, dtype=bool)
        x = np.zeros(n)
        if f.any():
            x[f] = np.linalg.lstsq(a[:, f], b, rcond=None)[0]
        r = a @ x - b
        y = a.T @ r
        y[f] = 0.0
        if (x[f] >= -tol).all() and (y[~f] >= -tol).all():
            found.append((x, y, f))
    if not found:
        raise RuntimeError("no feasible complementary basic solution found")
    x0 = found[0][0]
    for x, _, _ in found[1:]:
        if np.max(np.abs(x - x0)) > 1e3 * tol * max(1.0, np.max(np.abs(x0))):
            raise RuntimeError("two different feasible solutions: uniqueness violated")
    return found[0]
