"""Optimality certificate for NNLS -- TEST INFRASTRUCTURE ONLY.

x solves Eq. 1 exactly when the LCP conditions of Eq. 3 hold:
    y = A^T A x - A^T b = A^T (A x - b),  x >= 0,  y >= 0,  <x, y> = 0.
Because A^T A is positive definite the solution is unique (Section 2), so a
small violation certifies x at any size.  The residual products here are
plain FP64 sparse products (scipy), independent of both the oracle's C code
and the CUDA library.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def csr_matrix(prob):
    return sp.csr_matrix((prob.val, prob.col_idx, prob.row_ptr), shape=(prob.m, prob.n))


def dual(prob, x):
    """y = A^T (A x - b) in FP64."""
    a = csr_matrix(prob)
    return a.T @ (a @ x - prob.b)


def violation(prob, x):
    """Largest violation of Eq. 3 at x, as absolute numbers:
    max(-min x, -min y, max |x_i y_i| / max(1,|x_i|)) with y = A^T (A x - b).

    The complementarity term is scaled per entry so that it is measured in
    the units of y (a violation of y_i >= 0 on the support of x)."""
    y = dual(prob, x)
    neg_x = max(0.0, -float(np.min(x)))
    neg_y = max(0.0, -float(np.min(y)))
    comp = float(np.max(np.abs(x * y) / np.maximum(1.0, np.abs(x))))
    return max(neg_x, neg_y, comp)


def atb_norm(prob):
    a = csr_matrix(prob)
    return float(np.linalg.norm(a.T @ prob.b))
