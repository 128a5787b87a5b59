/*
 * tsnnls_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU statement of the block principal pivoting (BPP)
 * method for non-negative least squares,
 *     min_x 1/2 ||A x - b||^2  subject to  x >= 0            (Eq. 1)
 * with A an m x n sparse matrix of full column rank, m > n.
 *
 * It exists to check the CUDA library, never to serve it: only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg may load it,
 * and it shares no code, header, table or helper with the CUDA path.
 *
 * Everything is FP64, IEEE round-to-nearest; it is compiled with
 * -ffp-contract=off so that no multiply-add is fused behind our back.
 * Nothing is blocked, fused or reordered beyond what the paper states:
 *   - Section 3: A^T A is formed by column dot products, without forming A^T,
 *     once, and each pivot takes the F x F submatrix of it.
 *   - Section 2 (normal equations solver): (A^T A)_FF x_F = (A^T b)_F is solved
 *     by a textbook (unblocked) Cholesky factorisation.
 *   - Section 2, Eq. 5: y_G = A_G^T (A_F x_F - b) by sparse products with A.
 *   - Section 2, algorithm box: the exchange rule with the backup counter p = 3,
 *     the single-variable fallback on the largest infeasible index, and the
 *     zeroing of entries within 1e-12 of zero.
 *   - Section 3: the final x_F is recomputed by a more accurate least-squares
 *     solver; the paper uses LSQR (Paige and Saunders), this file offers LSQR
 *     and, for small dense cases, Householder QR.
 *
 * Readings of the paper taken here (each also listed in the design notes):
 *   - "Set variables in x_F < 1e-12 and y_G < 1e-12 to zero" is read as
 *     |v| < zero_tol (absolute), as the prose of Section 2 describes; read
 *     literally it would erase every negative entry and the loop could not see
 *     an infeasible variable.
 *   - The initial y = -A^T b is taken as printed, without zeroing.
 *   - "Infeasible" means strictly negative after zeroing.
 *   - The largest index is taken over the infeasible variables of both sets.
 *   - N changes only when the infeasible count drops; p is reset to p_max
 *     only then.
 *   - The paper gives no iteration limit; max_iter guards the loop.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum {
    ORACLE_OK = 0,
    ORACLE_EMAXITER = 1,
    ORACLE_ENOTPD = 2,
    ORACLE_EINVAL = 3,
    ORACLE_ENOMEM = 4,
};

enum { ORACLE_FINAL_NONE = 0, ORACLE_FINAL_QR = 1, ORACLE_FINAL_LSQR = 2 };
enum { ORACLE_INNER_CHOLESKY = 0, ORACLE_INNER_LSQR = 1 };

/* ------------------------------------------------------------------------ */
/* Compressed sparse column copy of a CSR matrix (rows ascending per column). */

typedef struct {
    int64_t m, n;
    int64_t *col_ptr; /* [n+1] */
    int64_t *row_idx; /* [nnz] */
    double *cval;     /* [nnz] */
} csc_t;

static void csc_free(csc_t *c) {
    free(c->col_ptr);
    free(c->row_idx);
    free(c->cval);
}

static int csc_from_csr(int64_t m, int64_t n, const int64_t *row_ptr, const int32_t *col,
                        const double *val, csc_t *out) {
    int64_t nnz = row_ptr[m];
    out->m = m;
    out->n = n;
    out->col_ptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    out->row_idx = (int64_t *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int64_t));
    out->cval = (double *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(double));
    int64_t *next = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!out->col_ptr || !out->row_idx || !out->cval || !next) {
        free(next);
        csc_free(out);
        return ORACLE_ENOMEM;
    }
    for (int64_t e = 0; e < nnz; ++e) out->col_ptr[col[e] + 1] += 1;
    for (int64_t j = 0; j < n; ++j) out->col_ptr[j + 1] += out->col_ptr[j];
    for (int64_t j = 0; j < n; ++j) next[j] = out->col_ptr[j];
    /* Rows are visited in ascending order, so each column's rows come out sorted. */
    for (int64_t r = 0; r < m; ++r) {
        for (int64_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e) {
            int64_t j = col[e];
            out->row_idx[next[j]] = r;
            out->cval[next[j]] = val[e];
            next[j] += 1;
        }
    }
    free(next);
    return ORACLE_OK;
}

/* <a_i, a_j>: merge of two sorted sparse columns. */
static double column_dot(const csc_t *c, int64_t i, int64_t j) {
    int64_t p = c->col_ptr[i], pe = c->col_ptr[i + 1];
    int64_t q = c->col_ptr[j], qe = c->col_ptr[j + 1];
    double s = 0.0;
    while (p < pe && q < qe) {
        if (c->row_idx[p] < c->row_idx[q]) {
            ++p;
        } else if (c->row_idx[p] > c->row_idx[q]) {
            ++q;
        } else {
            s += c->cval[p] * c->cval[q];
            ++p;
            ++q;
        }
    }
    return s;
}

/* <a_j, v> for a dense v of length m. */
static double column_dot_dense(const csc_t *c, int64_t j, const double *v) {
    double s = 0.0;
    for (int64_t p = c->col_ptr[j]; p < c->col_ptr[j + 1]; ++p) s += c->cval[p] * v[c->row_idx[p]];
    return s;
}

static int validate_csr(int64_t m, int64_t n, const int64_t *row_ptr, const int32_t *col) {
    if (m <= 0 || n <= 0 || !row_ptr) return ORACLE_EINVAL;
    if (row_ptr[0] != 0) return ORACLE_EINVAL;
    for (int64_t r = 0; r < m; ++r) {
        if (row_ptr[r + 1] < row_ptr[r]) return ORACLE_EINVAL;
        for (int64_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e) {
            if (col[e] < 0 || col[e] >= n) return ORACLE_EINVAL;
            if (e > row_ptr[r] && col[e] <= col[e - 1]) return ORACLE_EINVAL;
        }
    }
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* Section 3: A^T A by column dot products, A^T b by column dots with b.      */

/* G (n x n, row-major, both triangles) with G[i][j] = <a_i, a_j>. */
int oracle_gram(int64_t m, int64_t n, const int64_t *row_ptr, const int32_t *col,
                const double *val, double *G) {
    int st = validate_csr(m, n, row_ptr, col);
    if (st) return st;
    csc_t c;
    st = csc_from_csr(m, n, row_ptr, col, val, &c);
    if (st) return st;
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t i = 0; i <= j; ++i) {
            double d = column_dot(&c, i, j);
            G[i * n + j] = d;
            G[j * n + i] = d;
        }
    }
    csc_free(&c);
    return ORACLE_OK;
}

/* c = A^T b. */
int oracle_atb(int64_t m, int64_t n, const int64_t *row_ptr, const int32_t *col,
               const double *val, const double *b, double *c_out) {
    int st = validate_csr(m, n, row_ptr, col);
    if (st) return st;
    csc_t c;
    st = csc_from_csr(m, n, row_ptr, col, val, &c);
    if (st) return st;
    for (int64_t j = 0; j < n; ++j) c_out[j] = column_dot_dense(&c, j, b);
    csc_free(&c);
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* Section 2 (normal equations solver): textbook Cholesky, row by row.       */

/* In place on a k x k row-major symmetric matrix: on return the lower
 * triangle holds L with L L^T = S (the strict upper triangle is left as is).
 * Returns ORACLE_ENOTPD on a non-positive pivot. */
int oracle_cholesky(int64_t k, double *S) {
    for (int64_t i = 0; i < k; ++i) {
        for (int64_t j = 0; j <= i; ++j) {
            double s = S[i * k + j];
            for (int64_t p = 0; p < j; ++p) s -= S[i * k + p] * S[j * k + p];
            if (i == j) {
                if (!(s > 0.0)) return ORACLE_ENOTPD;
                S[i * k + i] = sqrt(s);
            } else {
                S[i * k + j] = s / S[j * k + j];
            }
        }
    }
    return ORACLE_OK;
}

/* Solve L L^T x = rhs with the lower triangle of L (row-major, k x k). */
void oracle_cholesky_solve(int64_t k, const double *L, const double *rhs, double *x) {
    for (int64_t i = 0; i < k; ++i) { /* L z = rhs */
        double s = rhs[i];
        for (int64_t p = 0; p < i; ++p) s -= L[i * k + p] * x[p];
        x[i] = s / L[i * k + i];
    }
    for (int64_t i = k - 1; i >= 0; --i) { /* L^T x = z */
        double s = x[i];
        for (int64_t p = i + 1; p < k; ++p) s -= L[p * k + i] * x[p];
        x[i] = s / L[i * k + i];
    }
}

/* ------------------------------------------------------------------------ */
/* Final-step least-squares solvers (Section 3).                             */

/* min ||M z - rhs|| by Householder QR.  M is m x k column-major and is
 * overwritten; rhs (length m) is overwritten with Q^T rhs. */
int oracle_qr_lstsq(int64_t m, int64_t k, double *M, double *rhs, double *z) {
    if (k > m) return ORACLE_EINVAL;
    for (int64_t j = 0; j < k; ++j) {
        double *cj = M + j * m;
        double norm = 0.0;
        for (int64_t i = j; i < m; ++i) norm += cj[i] * cj[i];
        norm = sqrt(norm);
        if (norm == 0.0) return ORACLE_ENOTPD;
        double alpha = cj[j] > 0.0 ? -norm : norm; /* R_jj, sign chosen against cancellation */
        /* reflector v = x - alpha e_1, stored over the column; H = I - 2 v v^T / (v^T v) */
        cj[j] -= alpha;
        double vtv = 0.0;
        for (int64_t i = j; i < m; ++i) vtv += cj[i] * cj[i];
        for (int64_t l = j + 1; l < k; ++l) {
            double *cl = M + l * m;
            double d = 0.0;
            for (int64_t i = j; i < m; ++i) d += cj[i] * cl[i];
            double f = 2.0 * d / vtv;
            for (int64_t i = j; i < m; ++i) cl[i] -= f * cj[i];
        }
        double d = 0.0;
        for (int64_t i = j; i < m; ++i) d += cj[i] * rhs[i];
        double f = 2.0 * d / vtv;
        for (int64_t i = j; i < m; ++i) rhs[i] -= f * cj[i];
        cj[j] = alpha; /* keep R_jj on the diagonal; the rest of the reflector is no longer needed */
    }
    for (int64_t i = k - 1; i >= 0; --i) { /* R z = (Q^T rhs)_{0..k-1} */
        double s = rhs[i];
        for (int64_t l = i + 1; l < k; ++l) s -= M[l * m + i] * z[l];
        z[i] = s / M[i * m + i];
    }
    return ORACLE_OK;
}

/* y = A_F v_F (m-vector) where v is indexed by the position in F. */
static void apply_AF(int64_t m, const int64_t *row_ptr, const int32_t *col, const double *val,
                     const int64_t *pos_in_F, const double *vF, double *y) {
    for (int64_t r = 0; r < m; ++r) {
        double s = 0.0;
        for (int64_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e) {
            int64_t p = pos_in_F[col[e]];
            if (p >= 0) s += val[e] * vF[p];
        }
        y[r] = s;
    }
}

/* w_F = A_F^T u via the CSC copy. */
static void apply_AFt(const csc_t *c, int64_t k, const int64_t *F, const double *u, double *wF) {
    for (int64_t a = 0; a < k; ++a) wF[a] = column_dot_dense(c, F[a], u);
}

/* LSQR of Paige and Saunders (1982) for min ||A_F z - rhs||, z in R^k, from
 * z = 0: Golub-Kahan bidiagonalisation with the QR update of the bidiagonal
 * by plane rotations.  Stops when the estimate of ||A_F^T r|| falls below
 * atol * ||A_F||_F * ||r||, or after max_it steps.  Returns the step count. */
static int64_t lsqr_on_AF(int64_t m, const int64_t *row_ptr, const int32_t *col,
                          const double *val, const csc_t *c, int64_t k, const int64_t *F,
                          const int64_t *pos_in_F, const double *rhs, double atol,
                          int64_t max_it, double *z, double *work) {
    double *u = work;          /* m */
    double *tmp_m = u + m;     /* m */
    double *v = tmp_m + m;     /* k */
    double *w = v + k;         /* k */
    double *tmp_k = w + k;     /* k */
    double anorm = 0.0;
    for (int64_t a = 0; a < k; ++a)
        for (int64_t p = c->col_ptr[F[a]]; p < c->col_ptr[F[a] + 1]; ++p) anorm += c->cval[p] * c->cval[p];
    anorm = sqrt(anorm);
    for (int64_t a = 0; a < k; ++a) z[a] = 0.0;

    double beta = 0.0;
    for (int64_t r = 0; r < m; ++r) beta += rhs[r] * rhs[r];
    beta = sqrt(beta);
    if (beta == 0.0) return 0;
    for (int64_t r = 0; r < m; ++r) u[r] = rhs[r] / beta;
    apply_AFt(c, k, F, u, v);
    double alpha = 0.0;
    for (int64_t a = 0; a < k; ++a) alpha += v[a] * v[a];
    alpha = sqrt(alpha);
    if (alpha == 0.0) return 0;
    for (int64_t a = 0; a < k; ++a) { v[a] /= alpha; w[a] = v[a]; }
    double phibar = beta, rhobar = alpha;
    int64_t it = 0;
    while (it < max_it) {
        ++it;
        /* beta u = A_F v - alpha u */
        apply_AF(m, row_ptr, col, val, pos_in_F, v, tmp_m);
        beta = 0.0;
        for (int64_t r = 0; r < m; ++r) { u[r] = tmp_m[r] - alpha * u[r]; beta += u[r] * u[r]; }
        beta = sqrt(beta);
        if (beta > 0.0) for (int64_t r = 0; r < m; ++r) u[r] /= beta;
        /* alpha v = A_F^T u - beta v */
        apply_AFt(c, k, F, u, tmp_k);
        alpha = 0.0;
        for (int64_t a = 0; a < k; ++a) { v[a] = tmp_k[a] - beta * v[a]; alpha += v[a] * v[a]; }
        alpha = sqrt(alpha);
        if (alpha > 0.0) for (int64_t a = 0; a < k; ++a) v[a] /= alpha;
        /* plane rotation eliminating the subdiagonal beta */
        double rho = sqrt(rhobar * rhobar + beta * beta);
        double cs = rhobar / rho, sn = beta / rho;
        double theta = sn * alpha;
        rhobar = -cs * alpha;
        double phi = cs * phibar;
        phibar = sn * phibar;
        for (int64_t a = 0; a < k; ++a) {
            z[a] += (phi / rho) * w[a];
            w[a] = v[a] - (theta / rho) * w[a];
        }
        /* ||A_F^T r|| = phibar * alpha * |cs|, ||r|| = phibar */
        if (phibar * alpha * fabs(cs) <= atol * anorm * phibar) break;
        if (alpha == 0.0 || beta == 0.0) break;
    }
    return it;
}

/* ------------------------------------------------------------------------ */
/* The BPP loop (Section 2, algorithm box).                                  */

typedef struct {
    double zero_tol;   /* 1e-12 in the paper */
    int64_t p_max;     /* 3 in the paper */
    int64_t max_iter;  /* guard; the paper gives none */
    int32_t inner;     /* ORACLE_INNER_* : how x_F of Eq. 4 is solved per pivot */
    int32_t final_step;/* ORACLE_FINAL_* : recomputation of the last x_F */
    double lsqr_atol;
    int64_t lsqr_max_it;
} oracle_opts;

typedef struct {
    int64_t iters;        /* pivots (exchanges + solves) performed */
    int64_t final_k;      /* |F| at the end */
    int64_t lsqr_steps;   /* total LSQR steps, inner and final */
} oracle_info;

static void zero_small(double *v, int64_t n, double tol) {
    for (int64_t i = 0; i < n; ++i)
        if (fabs(v[i]) < tol) v[i] = 0.0;
}

/* y_G = A_G^T (A_F x_F - b) for all G, y_F = 0 (Eq. 5); x_G is already 0. */
static void compute_y(int64_t m, int64_t n, const int64_t *row_ptr, const int32_t *col,
                      const double *val, const csc_t *c, const double *b, const double *x,
                      const uint8_t *inF, double *resid, double *y) {
    for (int64_t r = 0; r < m; ++r) {
        double s = 0.0;
        for (int64_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e) s += val[e] * x[col[e]];
        resid[r] = s - b[r];
    }
    for (int64_t j = 0; j < n; ++j) y[j] = inF[j] ? 0.0 : column_dot_dense(c, j, resid);
}

/*
 * Solve Eq. 1 by BPP.  x_out, y_out (length n) receive the final x and
 * y = A^T (A x - b) restricted to G (0 on F); inF_out (length n) the final
 * set F as 0/1.  trace, if non-NULL, receives up to trace_cap rows of six
 * int64 per pivot: {n_inf, N before the branch, p after the branch,
 * branch (0 = count dropped, 1 = backup full exchange, 2 = single), |F| after,
 * the index the single exchange moved (-1 for a full exchange)}.
 */
int oracle_bpp_solve(int64_t m, int64_t n, const int64_t *row_ptr, const int32_t *col,
                     const double *val, const double *b, const oracle_opts *opts,
                     double *x_out, double *y_out, uint8_t *inF_out, oracle_info *info,
                     int64_t *trace, int64_t trace_cap) {
    int st = validate_csr(m, n, row_ptr, col);
    if (st) return st;
    if (m <= n) return ORACLE_EINVAL;
    csc_t c;
    st = csc_from_csr(m, n, row_ptr, col, val, &c);
    if (st) return st;

    const int use_chol = opts->inner == ORACLE_INNER_CHOLESKY;
    double *G = NULL;
    double *cvec = (double *)malloc((size_t)n * sizeof(double));
    double *x = (double *)calloc((size_t)n, sizeof(double));
    double *y = (double *)malloc((size_t)n * sizeof(double));
    double *resid = (double *)malloc((size_t)m * sizeof(double));
    uint8_t *inF = (uint8_t *)calloc((size_t)n, 1);
    uint8_t *infeasible = (uint8_t *)calloc((size_t)n, 1);
    int64_t *F = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    int64_t *pos = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    double *xF = (double *)malloc((size_t)n * sizeof(double));
    double *rhs = (double *)malloc((size_t)(m > n ? m : n) * sizeof(double));
    double *work = (double *)malloc((size_t)(2 * m + 3 * n) * sizeof(double));
    double *S = NULL;
    if (use_chol) {
        G = (double *)malloc((size_t)n * (size_t)n * sizeof(double));
        S = (double *)malloc((size_t)n * (size_t)n * sizeof(double));
    }
    if (!cvec || !x || !y || !resid || !inF || !infeasible || !F || !pos || !xF || !rhs || !work ||
        (use_chol && (!G || !S))) {
        st = ORACLE_ENOMEM;
        goto done;
    }

    /* Precompute c = A^T b and, for the normal-equations path, G = A^T A (Section 3). */
    for (int64_t j = 0; j < n; ++j) cvec[j] = column_dot_dense(&c, j, b);
    if (use_chol) {
        for (int64_t j = 0; j < n; ++j)
            for (int64_t i = 0; i <= j; ++i) {
                double d = column_dot(&c, i, j);
                G[i * n + j] = d;
                G[j * n + i] = d;
            }
    }

    /* F = {}, G = all, x = 0, y = -A^T b, p = p_max, N = infinity. */
    for (int64_t j = 0; j < n; ++j) y[j] = -cvec[j];
    int64_t p = opts->p_max;
    int64_t Nbest = INT64_MAX;
    int64_t iters = 0, k = 0, lsqr_steps = 0;

    for (;;) {
        /* infeasible variables: negative entries of x_F and y_G */
        int64_t ninf = 0, largest = -1;
        for (int64_t j = 0; j < n; ++j) {
            int bad = inF[j] ? (x[j] < 0.0) : (y[j] < 0.0);
            infeasible[j] = (uint8_t)bad;
            if (bad) { ++ninf; largest = j; }
        }
        if (ninf == 0) break;
        if (iters >= opts->max_iter) { st = ORACLE_EMAXITER; goto done; }

        int64_t branch, Nprev = Nbest;
        if (ninf < Nbest) {
            Nbest = ninf;
            p = opts->p_max;
            branch = 0;
        } else if (p > 0) {
            p -= 1;
            branch = 1;
        } else {
            branch = 2;
        }
        if (branch == 2) {
            inF[largest] ^= 1;
        } else {
            for (int64_t j = 0; j < n; ++j)
                if (infeasible[j]) inF[j] ^= 1;
        }

        /* the new F, ascending */
        k = 0;
        for (int64_t j = 0; j < n; ++j) {
            pos[j] = -1;
            if (inF[j]) { pos[j] = k; F[k++] = j; }
        }

        /* Eq. 4: x_F = argmin ||A_F x_F - b||; x_G = 0 */
        for (int64_t j = 0; j < n; ++j) x[j] = 0.0;
        if (k > 0) {
            if (use_chol) {
                for (int64_t a = 0; a < k; ++a) {
                    for (int64_t bb = 0; bb < k; ++bb) S[a * k + bb] = G[F[a] * n + F[bb]];
                    rhs[a] = cvec[F[a]];
                }
                st = oracle_cholesky(k, S);
                if (st) goto done;
                oracle_cholesky_solve(k, S, rhs, xF);
            } else {
                lsqr_steps += lsqr_on_AF(m, row_ptr, col, val, &c, k, F, pos, b, opts->lsqr_atol,
                                         opts->lsqr_max_it, xF, work);
            }
            for (int64_t a = 0; a < k; ++a) x[F[a]] = xF[a];
        }
        /* Eq. 5 */
        compute_y(m, n, row_ptr, col, val, &c, b, x, inF, resid, y);
        /* zeroing of near-zero entries (Section 2) */
        zero_small(x, n, opts->zero_tol);
        zero_small(y, n, opts->zero_tol);

        if (trace && iters < trace_cap) {
            int64_t *t = trace + 6 * iters;
            t[0] = ninf;
            t[1] = Nprev;
            t[2] = p;
            t[3] = branch;
            t[4] = k;
            t[5] = branch == 2 ? largest : -1;
        }
        ++iters;
    }

    /* Section 3: recompute the final x_F with a more accurate solver. */
    if (k > 0 && opts->final_step != ORACLE_FINAL_NONE) {
        if (opts->final_step == ORACLE_FINAL_QR) {
            double *M = (double *)calloc((size_t)m * (size_t)k, sizeof(double));
            if (!M) { st = ORACLE_ENOMEM; goto done; }
            for (int64_t r = 0; r < m; ++r)
                for (int64_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e)
                    if (pos[col[e]] >= 0) M[pos[col[e]] * m + r] = val[e];
            for (int64_t r = 0; r < m; ++r) rhs[r] = b[r];
            st = oracle_qr_lstsq(m, k, M, rhs, xF);
            free(M);
            if (st) goto done;
        } else {
            /* LSQR on the correction: min ||A_F z - (b - A_F x_F)||, then x_F += z */
            for (int64_t a = 0; a < k; ++a) xF[a] = x[F[a]];
            apply_AF(m, row_ptr, col, val, pos, xF, resid);
            for (int64_t r = 0; r < m; ++r) rhs[r] = b[r] - resid[r];
            double *z = (double *)malloc((size_t)k * sizeof(double));
            if (!z) { st = ORACLE_ENOMEM; goto done; }
            lsqr_steps += lsqr_on_AF(m, row_ptr, col, val, &c, k, F, pos, rhs, opts->lsqr_atol,
                                     opts->lsqr_max_it, z, work);
            for (int64_t a = 0; a < k; ++a) xF[a] += z[a];
            free(z);
        }
        for (int64_t j = 0; j < n; ++j) x[j] = 0.0;
        for (int64_t a = 0; a < k; ++a) x[F[a]] = xF[a];
        compute_y(m, n, row_ptr, col, val, &c, b, x, inF, resid, y);
        zero_small(x, n, opts->zero_tol);
        zero_small(y, n, opts->zero_tol);
    }

    memcpy(x_out, x, (size_t)n * sizeof(double));
    if (y_out) memcpy(y_out, y, (size_t)n * sizeof(double));
    if (inF_out) memcpy(inF_out, inF, (size_t)n);
    if (info) {
        info->iters = iters;
        info->final_k = k;
        info->lsqr_steps = lsqr_steps;
    }
    st = ORACLE_OK;
done:
    free(G); free(S); free(cvec); free(x); free(y); free(resid); free(inF); free(infeasible);
    free(F); free(pos); free(xF); free(rhs); free(work);
    csc_free(&c);
    return st;
}
