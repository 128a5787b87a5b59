/* Host sanitizer run of the CPU oracle (test infrastructure only).
 *
 * This translation unit includes the oracle's source so that one compile
 * with -fsanitize=address,undefined instruments both.  It drives every
 * oracle entry point over small seeded problems: square and tall shapes,
 * n = 1, an empty column, a dense block, each inner solver and final step,
 * p_max = 0 (single-exchange fallback from the first failure) and 3.
 * Exit status 0 iff every call returns ORACLE_OK and every x is >= 0; a
 * sanitizer report aborts the run. */
#include "../../oracle/tsnnls_oracle.c"

#include <stdio.h>

static uint64_t g_state = 0x9e3779b97f4a7c15ull;

static uint64_t next_u64(void) { /* splitmix64 */
    uint64_t z = (g_state += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

static double unit(void) { return (double)(next_u64() >> 11) * (1.0 / 9007199254740992.0); }

/* m x n CSR: A[i][i] = 1 for i < n (full column rank), plus each other
 * entry present with probability density, values in (-1, 1); column
 * empty_col (if >= 0) holds nothing. */
static void make_problem(int64_t m, int64_t n, double density, int64_t empty_col, int64_t **rp,
                         int32_t **ci, double **va, double **b) {
    *rp = malloc(sizeof(int64_t) * (size_t)(m + 1));
    *ci = malloc(sizeof(int32_t) * (size_t)(m * n + 1));
    *va = malloc(sizeof(double) * (size_t)(m * n + 1));
    *b = malloc(sizeof(double) * (size_t)m);
    int64_t e = 0;
    (*rp)[0] = 0;
    for (int64_t i = 0; i < m; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            if (j == empty_col) continue;
            const int diag = i == j;
            if (diag || unit() < density) {
                (*ci)[e] = (int32_t)j;
                (*va)[e] = diag ? 1.0 : 2.0 * unit() - 1.0;
                ++e;
            }
        }
        (*rp)[i + 1] = e;
        (*b)[i] = 2.0 * unit() - 1.0;
    }
}

static int run_case(int64_t m, int64_t n, double density, int64_t empty_col) {
    int64_t *rp;
    int32_t *ci;
    double *va, *b;
    make_problem(m, n, density, empty_col, &rp, &ci, &va, &b);
    int bad = 0;
    double *x = malloc(sizeof(double) * (size_t)n), *y = malloc(sizeof(double) * (size_t)n);
    uint8_t *inF = malloc((size_t)n);
    int64_t trace[64 * 6];
    const int32_t inners[2] = {ORACLE_INNER_CHOLESKY, ORACLE_INNER_LSQR};
    const int32_t finals[3] = {ORACLE_FINAL_NONE, ORACLE_FINAL_QR, ORACLE_FINAL_LSQR};
    const int64_t pmaxs[2] = {0, 3};
    for (int a = 0; a < 2; ++a)
        for (int f = 0; f < 3; ++f)
            for (int p = 0; p < 2; ++p) {
                oracle_opts o = {1e-12, pmaxs[p], 10 * n + 100, inners[a], finals[f], 1e-15, 4 * n + 100};
                oracle_info info;
                const int st = oracle_bpp_solve(m, n, rp, ci, va, b, &o, x, y, inF, &info, trace, 64);
                if (st != ORACLE_OK) {
                    fprintf(stderr, "bpp m=%lld n=%lld inner=%d final=%d pmax=%lld: status %d\n",
                            (long long)m, (long long)n, a, f, (long long)pmaxs[p], st);
                    bad = 1;
                }
                for (int64_t j = 0; j < n && st == ORACLE_OK; ++j)
                    if (!(x[j] >= 0.0)) bad = 1;
            }
    double *G = malloc(sizeof(double) * (size_t)(n * n)), *c = malloc(sizeof(double) * (size_t)n);
    if (oracle_gram(m, n, rp, ci, va, G) != ORACLE_OK || oracle_atb(m, n, rp, ci, va, b, c) != ORACLE_OK)
        bad = 1;
    if (empty_col < 0) { /* A^T A is positive definite: factor and solve */
        double *z = malloc(sizeof(double) * (size_t)n);
        if (oracle_cholesky(n, G) != ORACLE_OK) bad = 1;
        else oracle_cholesky_solve(n, G, c, z);
        free(z);
    }
    /* dense least squares on A itself (row-major m x n copy) */
    double *M = calloc((size_t)(m * n), sizeof(double)), *rhs = malloc(sizeof(double) * (size_t)m);
    double *zz = malloc(sizeof(double) * (size_t)n);
    for (int64_t i = 0; i < m; ++i) {
        rhs[i] = b[i];
        for (int64_t q = rp[i]; q < rp[i + 1]; ++q) M[i * n + ci[q]] = va[q];
    }
    if (empty_col < 0 && oracle_qr_lstsq(m, n, M, rhs, zz) != ORACLE_OK) bad = 1;
    free(M), free(rhs), free(zz), free(G), free(c), free(x), free(y), free(inF);
    free(rp), free(ci), free(va), free(b);
    return bad;
}

int main(void) {
    int bad = 0;
    bad |= run_case(2, 1, 0.5, -1);
    bad |= run_case(9, 6, 0.3, -1);
    bad |= run_case(30, 20, 0.15, 7);
    bad |= run_case(60, 40, 0.9, -1);
    bad |= run_case(120, 70, 0.05, -1);
    if (bad) fprintf(stderr, "oracle sanitizer run: failures\n");
    return bad;
}
