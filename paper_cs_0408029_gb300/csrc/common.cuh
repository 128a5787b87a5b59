// Internal declarations shared by the kernels and the engine of the GB300
// block principal pivoting NNLS library.  Nothing here is part of the C ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "tsnnls.h"

namespace tsnnls {

// Device-resident state of one pivot loop, read by the host once per pivot
// (and once per refinement step) through a pinned mirror.
struct DevStatus {
    int32_t k;          // |F|
    int32_t n_inf;      // infeasible count of the last test
    int64_t N;          // smallest infeasible count so far (INT64_MAX = infinity)
    int32_t p;          // backup exchanges left
    int32_t branch;     // 0: count dropped, 1: backup full exchange, 2: single exchange
    int32_t done;       // 1 once (x_F, y_G) is feasible
    int32_t iters;      // pivots performed
    int32_t chol_info;  // 0, or 1 + column of the first non-positive pivot
    int32_t timeout;    // 1 if a bounded device wait gave up
    int32_t maxiter_hit;
    int32_t unsettled;  // entries whose sign / zeroing decision the last check left open
    int32_t border_a;   // variables in F but not in the factored base set (border.cu)
    int32_t border_r;   // variables of the base set no longer in F
    int32_t moved;      // index the single exchange moved (branch 2), else -1
    int32_t pad_;
    double dnorm;       // ||dx_F||_inf of the last refinement step
    double xnorm;       // ||x_F||_inf after it
    double kkt_viol;      // quality.cu: violation of Eq. 3 / ||A^T b||_2 at the final x
    double resid_change;  // quality.cu: ||A dx||_2 / ||b - A x||_2 of the last correction
};

constexpr int kSpinLimit = 1 << 22;  // bounded polls (with backoff) before a wait gives up

__host__ __device__ inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ inline int64_t round_up(int64_t a, int64_t b) { return cdiv(a, b) * b; }

// Streaming multiprocessors of the current device (queried once per device;
// launch sizes are multiples of it).
int num_sms();

// Launch accounting: every launcher below calls note_launches() once per
// kernel it starts; the engine reads the per-thread count around a solve.
void note_launches(int n);
int64_t launches_so_far();

// ---- kernel launchers (each returns the launch error, never synchronises) --

// CSR -> CSC transpose, rows ascending inside each column.
cudaError_t launch_csr_to_csc(cudaStream_t s, int64_t m, int64_t n, int64_t nnz,
                              const int64_t *row_ptr, const int32_t *col, const double *val,
                              int64_t *col_ptr, int32_t *row_idx, double *cval,
                              int32_t *work /* n+1 ints */, int64_t *scan_work /* n+1 */);

// Section 3: lower triangle of G = A^T A (column-major, ld) and c = A^T b.
template <typename T>
cudaError_t launch_gram(cudaStream_t s, int64_t m, int64_t n, const int64_t *row_ptr,
                        const int32_t *col, const double *val, const int64_t *col_ptr,
                        const int32_t *row_idx, const double *cval, const double *b, T *G,
                        int64_t ldg, double *c);

// Lower triangle of S = G_FF from the lower triangle of G.
template <typename T>
cudaError_t launch_gather(cudaStream_t s, const T *G, int64_t ldg, const int32_t *F,
                          const int32_t *k_dev, int64_t k_max, T *S, int64_t lds);

// Tensor-core update context for the FP32 factorisation: K-major hi / lo
// copies of each step's panel (rows x 128 FP32 each) and their TMA maps.
struct TcPanel {
    CUtensorMap map_hi, map_lo;
    float *xhi = nullptr, *xlo = nullptr;
    int64_t rows = 0;
    bool ok = false;
};

bool tc_available();
bool tc_encode_panel_map(void *buf, int64_t rows, CUtensorMap *out);
// Prepare tc over two caller-owned buffers of rows x 128 floats; false if the
// tensor maps cannot be encoded (the factorisation then uses the SIMT update).
bool tc_panel_init(TcPanel &tc, float *xhi, float *xlo, int64_t rows);
cudaError_t launch_tc_update(cudaStream_t s, const CUtensorMap &hi, const CUtensorMap &lo, float *S,
                             int64_t k, int64_t lds, int64_t T0, DevStatus *st, int64_t tile0 = 0);

// Optional per-kernel timing hooks (profiling only).
struct KernelTimer {
    virtual void begin(int phase) = 0;
    virtual void end(double bytes, double flops) = 0;
};

// In-place blocked lower Cholesky of the k x k matrix S (column-major, lds).
// tc (FP32 only, may be NULL) selects the tensor-core trailing update.
// S must be 16-byte aligned and lds a multiple of 32 (cudaErrorInvalidValue
// otherwise, nothing launched).
// fs (may be NULL): a second stream and three events for look-ahead, i.e.
// the panel rows of the next diagonal block, that block's update and its
// factor run on fs->side while the rest of the panel and of the trailing
// update run on s.  Ignored when kt is given (kernels timed one
// by one, in order).
struct FactorStreams {
    cudaStream_t side;
    cudaEvent_t fork, head, join;
};
template <typename T>
cudaError_t launch_cholesky(cudaStream_t s, T *S, int64_t k, int64_t lds, DevStatus *st,
                            const TcPanel *tc = nullptr, KernelTimer *kt = nullptr,
                            const FactorStreams *fs = nullptr);

// rhs <- (L L^T)^{-1} rhs with the blocked chained triangular solves.
// scratch: device memory of chol_solve_scratch_bytes(k, sizeof(T)) bytes,
// 256-byte aligned (flags and per-CTA partial sums; its contents on entry do
// not matter).
size_t chol_solve_scratch_bytes(int64_t k, size_t elem);
template <typename T>
cudaError_t launch_chol_solve(cudaStream_t s, const T *L, int64_t k, int64_t lds, T *rhs,
                              void *scratch, DevStatus *st);
// the two halves: rhs <- L^-1 rhs, rhs <- L^-T rhs
template <typename T>
cudaError_t launch_trsv_fwd(cudaStream_t s, const T *L, int64_t k, int64_t lds, T *rhs, void *scratch,
                            DevStatus *st);
template <typename T>
cudaError_t launch_trsv_bwd(cudaStream_t s, const T *L, int64_t k, int64_t lds, T *rhs, void *scratch,
                            DevStatus *st);
// q right-hand sides rhs + j rhs_ld at once (dirs: 1 forward, 2 backward, 3
// both), each solved by its own chain of CTAs in one launch; scratch of
// trsv_multi_scratch_bytes(k, sizeof(T), q) bytes, 256-byte aligned.
size_t trsv_multi_scratch_bytes(int64_t k, size_t elem, int q);
template <typename T>
cudaError_t launch_trsv_multi(cudaStream_t s, const T *L, int64_t k, int64_t lds, T *rhs, int64_t rhs_ld, int q,
                              void *scratch, DevStatus *st, int dirs);

// One bounded device wait on *flag >= 1 (limit polls), st->timeout = 1 when
// it gives up (self-test of the waits' failure path).
cudaError_t launch_wait_probe(cudaStream_t s, const int32_t *flag, int64_t limit, DevStatus *st);

// out = alpha * M x + beta * z over a CSR (or CSC viewed as CSR of M^T).
cudaError_t launch_spmv(cudaStream_t s, int64_t rows, const int64_t *ptr, const int32_t *idx,
                        const double *val, double alpha, const double *x, int64_t xlen, double beta,
                        const double *z, double *out, double avg_nnz);

// Pivot-loop glue kernels (exchange.cu).
cudaError_t launch_init_state(cudaStream_t s, int64_t n, const double *c, double *x, double *y,
                              uint8_t *inF, int32_t p_max, DevStatus *st);
cudaError_t launch_exchange(cudaStream_t s, int64_t n, double *x, double *y, uint8_t *inF,
                            int32_t *F, double zero_tol, int32_t p_max, int32_t max_iter,
                            int32_t apply_zeroing, DevStatus *st);
template <typename T>
cudaError_t launch_gather_rhs(cudaStream_t s, const double *v, int64_t n, const int32_t *F, int64_t k,
                              T *out);  // out[a] = v[F[a]], v of n entries
template <typename T>
cudaError_t launch_update_x(cudaStream_t s, const T *delta, const int32_t *F, int64_t k,
                            double *x, int64_t n, DevStatus *st);  // x of n entries
// ---- reuse of a factor across pivots (border.cu) ----
constexpr int kBorderMax = 32;  // added and removed variables handled at most (each)
struct BorderBuffers {
    int32_t *Bl;      // base list (the F of the factored pivot), n entries
    uint8_t *inB;     // base flags, n entries
    int32_t *Ul;      // U = base list with removed entries -1, then the added ones
    int32_t *Al;      // added variables (<= kBorderMax)
    int32_t *Rpos;    // base positions of the removed ones (<= kBorderMax)
    void *Pt;         // P^T = L^-1 G_BA, kb x a, leading dimension ldp
    void *Z;          // H^-1 E_R, u x r, leading dimension ldz
    double *GAA, *Lq, *Lc;  // kBorderMax^2 each: G_AA, factor of G_AA - P P^T, factor of Z_R
    double *mu;
    int32_t *bad;     // set by the setup when a small factor is not positive definite
    void *multi;      // scratch of kBorderMax simultaneous triangular solves
    int64_t ldp, ldz;
};
size_t border_bytes(int64_t n, size_t elem);
BorderBuffers border_carve(void *base, int64_t n, size_t elem);
// st->border_a / border_r: how many variables F' adds to and removes from the base
cudaError_t launch_border_count(cudaStream_t s, int64_t n, const uint8_t *inF, const BorderBuffers &b,
                                DevStatus *st);
// A, R and U for the new flags against the base (counts in st->border_a / border_r)
cudaError_t launch_border_diff(cudaStream_t s, int64_t n, const uint8_t *inF, const BorderBuffers &b, int64_t kb,
                               DevStatus *st);
// P^T, the factor of G_AA - P P^T, Z and the factor of Z_R for a <= kBorderMax
// added and r <= kBorderMax removed variables (L: the base factor, kb x kb)
template <typename T>
cudaError_t launch_border_setup(cudaStream_t s, const T *G, int64_t ldg, const T *L, int64_t kb, int64_t lds,
                                int a, int r, const BorderBuffers &b, DevStatus *st);
// z (u = kb + a entries, U order) <- solution of G_F'F' z_F' = z_F' with z_R = 0
template <typename T>
cudaError_t launch_border_solve(cudaStream_t s, const T *L, int64_t kb, int64_t lds, int a, int r,
                                const BorderBuffers &b, T *z, void *trsv_scratch, DevStatus *st);

// c = |A|^T (|A| 1): c_i bounds sum_f |(A^T A)_if| (t: m doubles of scratch).
cudaError_t launch_gram_row_bound(cudaStream_t s, int64_t m, int64_t n, const int64_t *row_ptr,
                                  const double *val, const int64_t *col_ptr, const int32_t *row_idx,
                                  const double *cval, double *t, double *c);
// st->unsettled = entries of x_F (error <= E) and y_G = -s_G (error <= c_j E)
// that may still fall on either side of 0 or +-zero_tol.
cudaError_t launch_settled(cudaStream_t s, int64_t n, const uint8_t *inF, const double *x,
                           const double *sv, const double *c, double E, double zero_tol, DevStatus *st);
// 1-norm estimate helpers (see exchange.cu): probe fill (mode 0 uniform
// 1/k, 1 unit vector e_j, 2 alternating (-1)^i (1 + i/(k-1))), ||y||_1 and
// sign(y) into out[0] / xi, max |z_i| / first argmax / z^T x (x uniform for
// mode 0, e_jprev for mode 1) into out[1..3].
template <typename T>
cudaError_t launch_est_fill(cudaStream_t s, T *v, int64_t k, int32_t mode, int64_t j);
template <typename T>
cudaError_t launch_est_norm_sign(cudaStream_t s, const T *y, int64_t k, T *xi, double *out);
template <typename T>
cudaError_t launch_est_argmax(cudaStream_t s, const T *z, int64_t k, int32_t mode, int64_t jprev, double *out);
// *out = ||G_FF||_1 for the symmetric block whose lower triangle G (ldg) holds;
// scratch: gram_norm_scratch_bytes(k) bytes.
size_t gram_norm_scratch_bytes(int64_t k);
template <typename T>
cudaError_t launch_gram_norm1(cudaStream_t s, const T *G, int64_t ldg, const int32_t *F, int64_t k,
                              double *scratch, double *out);
cudaError_t launch_y_from_s(cudaStream_t s, int64_t n, const double *sv, const uint8_t *inF,
                            double *y);

// Quality of a finished solve (quality.cu): st->kkt_viol and st->resid_change
// from the final x, s = A^T (b - A x), c = A^T b, r = b - A x and the last
// correction (delta over list[0..len), list entries -1 skipped; NULL: none).
// scratch: quality_scratch_bytes(m, n) bytes, 256-byte aligned.
size_t quality_scratch_bytes(int64_t m, int64_t n);
template <typename T>
cudaError_t launch_quality(cudaStream_t s, int64_t m, int64_t n, const int64_t *row_ptr, const int32_t *col,
                           const double *val, double avg_row, const double *x, const double *sv,
                           const double *c, const double *r, const T *delta, const int32_t *list,
                           int64_t len, void *scratch, DevStatus *st);
// The same with the correction given as D z on the columns of F (LSQR path).
template <typename V>
cudaError_t launch_quality_scaled(cudaStream_t s, int64_t m, int64_t n, const int64_t *row_ptr,
                                  const int32_t *col, const double *val, double avg_row, const double *x,
                                  const double *sv, const double *c, const double *r, const V *D,
                                  const V *z, const uint8_t *inF, bool have_delta, void *scratch,
                                  DevStatus *st);

}  // namespace tsnnls

namespace tsnnls {

// Validation of a device CSR matrix and right-hand side: writes a nonzero
// code to *bad on the first problem found (1 row_ptr, 2 column index,
// 3 ordering, 4 non-finite value).
cudaError_t launch_validate(cudaStream_t s, int64_t m, int64_t n, int64_t nnz,
                            const int64_t *row_ptr, const int32_t *col, const double *val,
                            const double *b, int32_t *bad);

}  // namespace tsnnls
