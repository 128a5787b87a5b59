"""Seeded synthetic NNLS problems (inputs only).

This module builds the inputs that both the CUDA library and the CPU oracle
consume, so that both read identical bytes.  It holds none of the block
principal pivoting arithmetic: it only draws random sparse/dense matrices, a
planted non-negative x*, and a right-hand side b.  Every generator is a pure
function of its seed (numpy ``default_rng``, PCG64), so the bytes are the same
on x86_64 and aarch64.

Problem shape follows Eq. 1 of the paper: A is m x n with m > n and full
column rank.  The workloads stand in for the paper's ``sprandn`` test matrices
(Section 4, Fig. 2) and its condition-controlled LSQR generator (Fig. 1), which
are not available here.

Recipes (each docstring restates its own):
  * plain_single      600 x 400, 2 % density, unit diagonal, 50 % zeros in x*,
                      noise 1e-3, then a perturbation making ~20 % of the
                      constraints strictly active.
  * larger_sparse     20000 x 8000, 20 nnz/row + unit diagonal, 40 % zeros,
                      noise 1e-2.
  * batched_uneven    512 dense FP32 problems, n log-uniform in [32, 1024],
                      m = round(1.5 n), 30 % zeros, noise 1e-3.
  * lsqr_large        2e6 x 2e5, 8 nnz/row, columns scaled by 10^U(-2,2),
                      60 % zeros, noise 1e-3.
  * serving_request   one request of the serving mix: n log-uniform in
                      [64, 8192], m = 2n, density U(1 %, 5 %), 40 % zeros.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 20040810


@dataclasses.dataclass
class CSRProblem:
    """A sparse NNLS instance: CSR matrix (sorted, duplicate-free rows) and b."""

    m: int
    n: int
    row_ptr: np.ndarray  # int64 [m+1]
    col_idx: np.ndarray  # int32 [nnz], ascending within each row
    val: np.ndarray      # float64 [nnz]
    b: np.ndarray        # float64 [m]
    x_planted: np.ndarray  # float64 [n], the x* used to build b (not the NNLS solution)
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def dense(self) -> np.ndarray:
        a = np.zeros((self.m, self.n))
        rows = np.repeat(np.arange(self.m), np.diff(self.row_ptr))
        a[rows, self.col_idx] = self.val
        return a


@dataclasses.dataclass
class DenseProblem:
    """A dense NNLS instance.  ``a`` is row-major m x n in the stated dtype."""

    m: int
    n: int
    a: np.ndarray  # [m, n]
    b: np.ndarray  # float64 [m]
    x_planted: np.ndarray
    name: str = ""


def _csr_from_rows(m, n, rows, cols, vals):
    """Assemble CSR from COO triples that are already duplicate-free."""
    order = np.lexsort((cols, rows))
    rows = rows[order]
    cols = cols[order].astype(np.int32)
    vals = vals[order].astype(np.float64)
    counts = np.bincount(rows, minlength=m)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return row_ptr, cols, vals


def _distinct_cols_per_row(rng, m, n, per_row):
    """m x per_row column indices, distinct within each row, uniform."""
    cols = rng.integers(0, n, size=(m, per_row))
    s = np.sort(cols, axis=1)
    bad = np.nonzero((s[:, 1:] == s[:, :-1]).any(axis=1))[0]
    for r in bad:
        cols[r] = rng.choice(n, size=per_row, replace=False)
    return cols


def _set_unit_diagonal(m, n, rows, cols, vals):
    """A[i, i] = 1 for i < n: overwrite the entry if present, else insert it."""
    on_diag = (rows == cols) & (rows < n)
    vals = vals.copy()
    vals[on_diag] = 1.0
    present = np.zeros(n, dtype=bool)
    present[rows[on_diag]] = True
    missing = np.nonzero(~present)[0]
    rows = np.concatenate([rows, missing])
    cols = np.concatenate([cols, missing])
    vals = np.concatenate([vals, np.ones(missing.size)])
    return rows, cols, vals


def _planted_x(rng, n, zero_frac):
    """x* with round(zero_frac*n) entries exactly 0 and the rest U(0.1, 1)."""
    x = rng.uniform(0.1, 1.0, size=n)
    zeros = rng.permutation(n)[: int(round(zero_frac * n))]
    x[zeros] = 0.0
    return x, np.sort(zeros)


def _csr_matvec(row_ptr, col_idx, val, x):
    rows = np.repeat(np.arange(row_ptr.size - 1), np.diff(row_ptr))
    return np.bincount(rows, weights=val * x[col_idx], minlength=row_ptr.size - 1)


def random_sparse(m, n, density, seed, *, unit_diagonal=True, zero_frac=0.5,
                  noise=1e-3, name="random_sparse") -> CSRProblem:
    """Entries nonzero independently with probability ``density`` (uniform
    positions), values N(0,1); optional A[i,i] = 1 for i < n; b = A x* + noise."""
    rng = np.random.default_rng(seed)
    mask = rng.random((m, n)) < density
    rows, cols = np.nonzero(mask)
    vals = rng.standard_normal(rows.size)
    if unit_diagonal:
        rows, cols, vals = _set_unit_diagonal(m, n, rows, cols, vals)
    row_ptr, col_idx, val = _csr_from_rows(m, n, rows, cols, vals)
    x, _ = _planted_x(rng, n, zero_frac)
    b = _csr_matvec(row_ptr, col_idx, val, x) + rng.normal(0.0, noise, size=m)
    return CSRProblem(m, n, row_ptr, col_idx, val, b, x, name)


def plain_single(seed=SEED_BASE + 0) -> CSRProblem:
    """A 600 x 400, each entry nonzero with p = 0.02 at uniform positions, N(0,1)
    values, A[i,i] = 1 for i < 400.  x*: 200 entries exactly 0, the rest
    U(0.1, 1).  b = A x* + N(0, (1e-3)^2).  Then a perturbation: on a random
    80-element (20 % of n) subset S of x*'s zeros draw y*_S ~ U(0.1,1) *
    ||A^T b||_2 / n and subtract w = A (A^T A)^{-1} y* from b, which makes
    A^T (A x* - b) = y* - A^T noise, i.e. those 80 constraints strictly active.
    """
    m, n = 600, 400
    rng = np.random.default_rng(seed)
    mask = rng.random((m, n)) < 0.02
    rows, cols = np.nonzero(mask)
    vals = rng.standard_normal(rows.size)
    rows, cols, vals = _set_unit_diagonal(m, n, rows, cols, vals)
    row_ptr, col_idx, val = _csr_from_rows(m, n, rows, cols, vals)
    x, zeros = _planted_x(rng, n, 0.5)
    b = _csr_matvec(row_ptr, col_idx, val, x) + rng.normal(0.0, 1e-3, size=m)
    prob = CSRProblem(m, n, row_ptr, col_idx, val, b, x, "plain_single_600x400")
    a = prob.dense()
    scale = np.linalg.norm(a.T @ b) / n
    subset = rng.permutation(zeros)[: int(round(0.2 * n))]
    ystar = np.zeros(n)
    ystar[subset] = rng.uniform(0.1, 1.0, size=subset.size) * scale
    w = a @ np.linalg.solve(a.T @ a, ystar)
    prob.b = b - w
    return prob


def larger_sparse(seed=SEED_BASE + 1, m=20000, n=8000, per_row=20,
                  zero_frac=0.4, noise=1e-2) -> CSRProblem:
    """A 20000 x 8000: 20 nonzeros per row at distinct uniform columns, N(0,1)
    values, plus A[i,i] = 1 for i < 8000 (the identity-diagonal block, written
    over the top n x n block).  x*: 40 % exactly 0, the rest U(0.1,1).
    b = A x* + N(0, (1e-2)^2).  ``m``, ``n`` and ``per_row`` may be reduced to
    build the same recipe at a smaller size."""
    rng = np.random.default_rng(seed)
    cols = _distinct_cols_per_row(rng, m, n, per_row)
    rows = np.repeat(np.arange(m), per_row)
    cols = cols.reshape(-1)
    vals = rng.standard_normal(rows.size)
    rows, cols, vals = _set_unit_diagonal(m, n, rows, cols, vals)
    row_ptr, col_idx, val = _csr_from_rows(m, n, rows, cols, vals)
    x, _ = _planted_x(rng, n, zero_frac)
    b = _csr_matvec(row_ptr, col_idx, val, x) + rng.normal(0.0, noise, size=m)
    return CSRProblem(m, n, row_ptr, col_idx, val, b, x, f"larger_sparse_{m}x{n}")


def batched_uneven(seed=SEED_BASE + 2, count=512, n_lo=32, n_hi=1024,
                   zero_frac=0.3, noise=1e-3):
    """``count`` independent dense problems: n = round(exp(U(ln 32, ln 1024))),
    m = round(1.5 n), A dense FP32 with N(0,1) values (row-major), x* with 30 %
    exact zeros and the rest U(0.1,1), b = float64(A) x* + N(0, (1e-3)^2)."""
    rng = np.random.default_rng(seed)
    ns = np.rint(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=count))).astype(int)
    out = []
    for i, n in enumerate(ns):
        m = int(round(1.5 * n))
        a = rng.standard_normal((m, n)).astype(np.float32)
        x, _ = _planted_x(rng, n, zero_frac)
        b = a.astype(np.float64) @ x + rng.normal(0.0, noise, size=m)
        out.append(DenseProblem(m, int(n), a, b, x, f"batched_{i}_{m}x{n}"))
    return out


def lsqr_large(seed=SEED_BASE + 3, m=2_000_000, n=200_000, per_row=8,
               zero_frac=0.6, noise=1e-3, col_spread=2.0) -> CSRProblem:
    """A 2e6 x 2e5: 8 nonzeros per row at distinct uniform columns, N(0,1), then
    column j scaled by s_j = 10^U(-2, 2) (condition number ~1e4; ``col_spread``
    sets the exponent range).  x*: 60 % exact zeros, rest U(0.1,1).
    b = A x* + N(0, (1e-3)^2)."""
    rng = np.random.default_rng(seed)
    cols = _distinct_cols_per_row(rng, m, n, per_row).reshape(-1)
    rows = np.repeat(np.arange(m), per_row)
    vals = rng.standard_normal(rows.size)
    s = 10.0 ** rng.uniform(-col_spread, col_spread, size=n)
    vals = vals * s[cols]
    row_ptr, col_idx, val = _csr_from_rows(m, n, rows, cols, vals)
    x, _ = _planted_x(rng, n, zero_frac)
    b = _csr_matvec(row_ptr, col_idx, val, x) + rng.normal(0.0, noise, size=m)
    return CSRProblem(m, n, row_ptr, col_idx, val, b, x, f"lsqr_large_{m}x{n}")


def grid_sparse(g, seed=SEED_BASE + 6, m_factor=2, per_row=4, zero_frac=0.4, noise=1e-2,
                name=None) -> CSRProblem:
    """A sparse problem whose A^T A keeps a small-separator pattern (the
    sparse-Gram workload of the supernodal factor): n = g * g unknowns on a
    g x g grid.  Rows 0 .. n-1 hold the unit diagonal (A[i, i] = 1); each of
    the other m - n rows (m = m_factor * n) holds per_row distinct unknowns
    drawn from the 3 x 3 grid neighbourhood of a uniformly chosen point, with
    N(0,1) values.  Columns meet in A^T A only within grid distance 2.
    x* has zero_frac exact zeros, the rest U(0.1, 1); b = A x* + N(0, noise^2)."""
    rng = np.random.default_rng(seed)
    n = g * g
    m = int(m_factor * n)
    extra = m - n
    cx = rng.integers(0, g, size=extra)
    cy = rng.integers(0, g, size=extra)
    offs = np.array([(dx, dy) for dx in (-1, 0, 1) for dy in (-1, 0, 1)])
    keys = rng.random((extra, 9))
    nx = cx[:, None] + offs[None, :, 0]
    ny = cy[:, None] + offs[None, :, 1]
    inside = (nx >= 0) & (nx < g) & (ny >= 0) & (ny < g)
    keys[~inside] = 2.0  # never chosen before an inside neighbour
    pick = np.argsort(keys, axis=1)[:, :per_row]
    ok = np.take_along_axis(inside, pick, axis=1)
    cols = (np.take_along_axis(nx, pick, axis=1) * g + np.take_along_axis(ny, pick, axis=1))
    rows = np.repeat(np.arange(n, m), per_row).reshape(extra, per_row)
    vals = rng.standard_normal((extra, per_row))
    rows, cols, vals = rows[ok], cols[ok], vals[ok]
    rows = np.concatenate([np.arange(n), rows])
    cols = np.concatenate([np.arange(n), cols])
    vals = np.concatenate([np.ones(n), vals])
    row_ptr, col_idx, val = _csr_from_rows(m, n, rows, cols, vals)
    x, _ = _planted_x(rng, n, zero_frac)
    b = _csr_matvec(row_ptr, col_idx, val, x) + rng.normal(0.0, noise, size=m)
    return CSRProblem(m, n, row_ptr, col_idx, val, b, x, name or f"grid_sparse_{g}x{g}")


def serving_request(index, seed=SEED_BASE + 4, n_lo=64, n_hi=8192) -> CSRProblem:
    """Request ``index`` of the serving mix: n = round(exp(U(ln 64, ln 8192))),
    m = 2n, density d ~ U(0.01, 0.05) at uniform positions, N(0,1) values,
    A[i,i] = 1 for i < n, x* 40 % zeros, b = A x* + N(0, (1e-3)^2)."""
    rng = np.random.default_rng([seed, index])
    n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
    m = 2 * n
    d = rng.uniform(0.01, 0.05)
    nnz_row = max(1, int(round(d * n)))
    cols = _distinct_cols_per_row(rng, m, n, nnz_row).reshape(-1)
    rows = np.repeat(np.arange(m), nnz_row)
    vals = rng.standard_normal(rows.size)
    rows, cols, vals = _set_unit_diagonal(m, n, rows, cols, vals)
    row_ptr, col_idx, val = _csr_from_rows(m, n, rows, cols, vals)
    x, _ = _planted_x(rng, n, 0.4)
    b = _csr_matvec(row_ptr, col_idx, val, x) + rng.normal(0.0, 1e-3, size=m)
    return CSRProblem(m, n, row_ptr, col_idx, val, b, x, f"serving_{index}_{m}x{n}")


def serving_arrivals(count, rate_per_s, seed=SEED_BASE + 5):
    """Poisson arrival times (seconds from 0) for ``count`` requests."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))


def conditioned_dense(m, n, kappa, seed, repeat=4, zero_frac=0.3, active_frac=0.5,
                      y_scale=None):
    """Condition-controlled dense problem with a known NNLS solution (stands
    in for the LSQR test generator P(m, n, d, x) of Section 4, Fig. 1, which
    is not available): A = U diag(sigma) V^T with U (m x n, orthonormal
    columns) and V (n x n, orthogonal) from QR of Gaussian matrices, sigma
    geometric from 1 to 1/kappa with each value repeated ``repeat`` times.

    x* has round(zero_frac*n) exact zeros, the rest U(0.1, 1); on a fraction
    ``active_frac`` of those zeros y*_i ~ U(0.1, 1) * y_scale (default
    1/kappa, which keeps ||A x* - b|| of order one), elsewhere y* = 0.  Then
    b = A x* - A (A^T A)^{-1} y* = U (sigma * V^T x* - V^T y* / sigma), so
    A^T (A x* - b) = y* and (x*, y*) satisfy Eq. 3: x* is the solution.
    Returns (DenseProblem with float64 A, x*, y*)."""
    rng = np.random.default_rng(seed)
    u, _ = np.linalg.qr(rng.standard_normal((m, n)))
    v, _ = np.linalg.qr(rng.standard_normal((n, n)))
    groups = -(-n // repeat)
    levels = kappa ** (-np.arange(groups) / max(groups - 1, 1))
    sigma = np.repeat(levels, repeat)[:n]
    a = u @ (sigma[:, None] * v.T)
    x, zeros = _planted_x(rng, n, zero_frac)
    y = np.zeros(n)
    act = rng.permutation(zeros)[: int(round(active_frac * zeros.size))]
    y[act] = rng.uniform(0.1, 1.0, size=act.size) * (1.0 / kappa if y_scale is None else y_scale)
    b = u @ (sigma * (v.T @ x) - (v.T @ y) / sigma)
    return DenseProblem(m, n, a, b, x, f"conditioned_{m}x{n}_k{kappa:g}"), x, y


def dense_to_csr(a: np.ndarray, b: np.ndarray, name="dense") -> CSRProblem:
    """Wrap a dense float64 matrix (explicit zeros dropped) as a CSRProblem."""
    a = np.asarray(a, dtype=np.float64)
    m, n = a.shape
    rows, cols = np.nonzero(a)
    row_ptr, col_idx, val = _csr_from_rows(m, n, rows, cols, a[rows, cols])
    return CSRProblem(m, n, row_ptr, col_idx, val, np.asarray(b, dtype=np.float64),
                      np.zeros(n), name)
