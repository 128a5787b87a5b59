// LSQR path: every pivot's least-squares problem (Eq. 4) solved on A_F by the
// LSQR method of Paige and Saunders (the solver Section 3 uses for the final
// recomputation) instead of the cached normal equations, for instances whose
// A^T A does not fit (or is not wanted).
//
// Outer loop (FP64): r = b - A x, then an inner LSQR run on
//     min || (A_F D) z - r ||,   D = diag(1 / ||a_j||)  (column scaling)
// in the value type V (FP32 for MIXED, FP64 for FP64), and x_F += D z, until
// the correction is below rel_tol * ||x_F||.  One inner iteration is three
// kernels:
//   av:  u^ = A (D v) - (alpha / beta_prev) u^_prev  (CSR, rows; D v kept as
//        its own vector, so one gather per nonzero)   + partial ||u^||^2
//   atu: v^ = D A^T (u^ / beta) - beta v            (CSC, columns, F only) + partial ||v^||^2
//   upd: alpha = ||v^||, v = v^ / alpha, D v, plane rotation, z += (phi/rho) w,
//        w = v - (theta/rho) w
// Short rows (the usual case) get one thread each with all their loads in
// flight at once; the FP64 scalar recurrences are evaluated by one thread
// per CTA (FP64 issue is scarce) and broadcast through shared memory.
// Norms are reduced through per-CTA partials that every consumer CTA sums in
// the same order, so the result is deterministic and needs no atomics and no
// extra launch.  The scalar recurrences live in device memory, double-buffered
// by iteration parity, so the inner loop never returns to the host.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "check.cuh"
#include "engine.h"

namespace tsnnls {

struct LsqrScalars {
    double alpha, beta, rhobar, phibar;
};

constexpr int kLT = 256;
constexpr int kMaxPartials = 4096;  // capacity of the per-CTA partial sums

// CTAs of a reduction kernel: eight per SM at most (every CTA of the next
// kernel sums all the partials, so more CTAs than fit at once only add reads)
inline int64_t partial_cap() { return std::min<int64_t>(kMaxPartials, (int64_t)num_sms() * 8); }

// Sum of `count` partials in a fixed order, broadcast to the CTA.
__device__ __forceinline__ double sum_partials(const double *__restrict__ part, int count,
                                               double *sh) {
    double v = 0.0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) v += part[i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        sh[0] = t;
    }
    __syncthreads();
    const double r = sh[0];
    __syncthreads();
    return r;
}

__device__ __forceinline__ void write_partial(double v, double *part, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        part[blockIdx.x] = t;
    }
}

__device__ __forceinline__ double safe_div(double a, double b) { return b != 0.0 ? a / b : 0.0; }

// Per-CTA broadcast of a scalar computed by thread 0.
__device__ __forceinline__ double cta_bcast(double v, double *sh) {
    __syncthreads();
    if (threadIdx.x == 0) sh[0] = v;
    __syncthreads();
    const double r = sh[0];
    __syncthreads();
    return r;
}


// Column scale D_j = 1 / ||a_j|| (1 for an empty column) and value copies in V.
template <typename V>
__global__ void lsqr_prep_kernel(int64_t n, const int64_t *__restrict__ col_ptr,
                                 const double *__restrict__ cval, V *__restrict__ D) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int64_t p = col_ptr[j]; p < col_ptr[j + 1]; ++p) s += cval[p] * cval[p];
        D[j] = (V)(s > 0.0 ? 1.0 / sqrt(s) : 1.0);
    }
}

template <typename V>
__global__ void convert_kernel(int64_t count, const double *__restrict__ src, V *__restrict__ dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (V)src[i];
}

// u^ = r (in V) and partial ||r||^2; v, w, z cleared.
template <typename V>
__global__ void __launch_bounds__(kLT)
    lsqr_start_kernel(int64_t m, int64_t n, const double *__restrict__ r, V *__restrict__ u,
                      V *__restrict__ v, V *__restrict__ w, V *__restrict__ z,
                      double *__restrict__ part_u) {
    __shared__ double sh[kLT / 32];
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        u[i] = (V)r[i];
        acc += r[i] * r[i];  // beta_1 = ||r|| from the FP64 residual
    }
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        v[j] = V(0);
        w[j] = V(0);
        z[j] = V(0);
    }
    write_partial(acc, part_u, sh);
}

// First direction of the bidiagonalisation, alpha_1 v_1 = (A_F D)^T u_1 with
// u_1 = r / beta_1, taken from the FP64 product s = A^T r: near convergence
// A_F^T r is far smaller than ||A|| ||r||, and forming it from an FP32 copy of
// r would bury it under rounding; with an accurate v_1 the later FP32
// rounding enters scaled by alpha_1 and vanishes with it.
template <typename V>
__global__ void __launch_bounds__(kLT)
    lsqr_vstart_kernel(int64_t n, const double *__restrict__ s_atr, const V *__restrict__ D,
                       const uint8_t *__restrict__ inF, V *__restrict__ v,
                       const double *__restrict__ part_u, int n_part_u, LsqrScalars *nxt,
                       double *__restrict__ part_v) {
    __shared__ double sh[kLT / 32];
    const double ssq = sum_partials(part_u, n_part_u, sh);
    const double beta = cta_bcast(threadIdx.x == 0 ? sqrt(ssq) : 0.0, sh);
    if (blockIdx.x == 0 && threadIdx.x == 0) nxt->beta = beta;
    const double inv_beta = cta_bcast(threadIdx.x == 0 ? safe_div(1.0, beta) : 0.0, sh);
    double acc = 0.0;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const V vn = inF[j] ? (V)((double)D[j] * s_atr[j] * inv_beta) : V(0);
        v[j] = vn;
        acc += (double)vn * (double)vn;
    }
    write_partial(acc, part_v, sh);
}

// av: u^ <- A dv - (alpha / beta) u^, dv = D v   (TPR lanes per row; TPR = 1:
// one row per thread, its nonzeros loaded eight at a time; with vec (FP32
// values, index and value arrays 16-byte aligned) the entries from the
// row's first 16-byte boundary on come as int4 / float4 pairs, two of each
// before the gathers, so that fewer, wider loads are in flight; the sum is
// taken in the row's order either way)
template <typename V, int TPR>
__global__ void __launch_bounds__(kLT)
    lsqr_av_kernel(int64_t m, int64_t n, const int64_t *__restrict__ ptr, const int32_t *__restrict__ idx,
                   const V *__restrict__ val, const V *__restrict__ dv, V *__restrict__ u,
                   const LsqrScalars *__restrict__ cur, double *__restrict__ part_u, bool vec) {
    __shared__ double sh[kLT / 32];
    const double scale = cta_bcast(threadIdx.x == 0 ? safe_div(cur->alpha, cur->beta) : 0.0, sh);
    const V vscale = (V)scale;
    const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double acc = 0.0;
    if constexpr (TPR == 1) {
        const int64_t stride = (int64_t)gridDim.x * blockDim.x;
        for (int64_t r = gtid; r < m; r += stride) {
            const int64_t p0 = ptr[r], p1 = ptr[r + 1];
            V s = V(0);
            int64_t p = p0;
            if constexpr (sizeof(V) == 4) {
                if (vec) {
                    const int64_t pa = min(p1, (p0 + 3) & ~(int64_t)3);
                    for (; p < pa; ++p) {
                        const int32_t c = idx[p];
                        s += TS_IN(c, n) ? val[p] * dv[c] : V(0);
                    }
                    for (; p + 8 <= p1; p += 8) {
                        const int4 c0 = __ldcs(reinterpret_cast<const int4 *>(idx + p));
                        const int4 c1 = __ldcs(reinterpret_cast<const int4 *>(idx + p + 4));
                        const float4 a0 = __ldcs(reinterpret_cast<const float4 *>(val + p));
                        const float4 a1 = __ldcs(reinterpret_cast<const float4 *>(val + p + 4));
                        const int c[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
                        const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                        float g[8];
#pragma unroll
                        for (int q = 0; q < 8; ++q) g[q] = TS_IN(c[q], n) ? (float)dv[c[q]] : 0.f;
#pragma unroll
                        for (int q = 0; q < 8; ++q) s += a[q] * g[q];
                    }
                }
            }
            for (; p < p1; p += 8) {
                int32_t c[8];
                V a[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const bool in = p + q < p1;
                    c[q] = in ? idx[p + q] : 0;
                    a[q] = in ? val[p + q] : V(0);
                }
#pragma unroll
                for (int q = 0; q < 8; ++q) s += TS_IN(c[q], n) ? a[q] * dv[c[q]] : V(0);
            }
            const V un = s - vscale * u[r];
            u[r] = un;
            acc += (double)un * (double)un;
        }
    } else {
        const int64_t stride_rows = ((int64_t)gridDim.x * blockDim.x) / TPR;
        const int sub = threadIdx.x % TPR;
        const int64_t warp_row0 = ((gtid >> 5) << 5) / TPR;
        const int64_t my_off = (gtid / TPR) - warp_row0;
        for (int64_t r0 = warp_row0; r0 < m; r0 += stride_rows) {
            const int64_t r = r0 + my_off;
            V s = V(0);
            if (r < m) {
                const int64_t p1 = ptr[r + 1];
                for (int64_t p = ptr[r] + sub; p < p1; p += 4 * TPR) {
                    int32_t c[4];
                    V a[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const bool in = p + q * TPR < p1;
                        c[q] = in ? idx[p + q * TPR] : 0;
                        a[q] = in ? val[p + q * TPR] : V(0);
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q) s += TS_IN(c[q], n) ? a[q] * dv[c[q]] : V(0);
                }
            }
#pragma unroll
            for (int o = TPR / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, TPR);
            if (sub == 0 && r < m) {
                const V un = s - vscale * u[r];
                u[r] = un;
                acc += (double)un * (double)un;
            }
        }
    }
    write_partial(acc, part_u, sh);
}

// atu: beta = ||u^||, v^ = D A^T (u^ / beta) - beta v on F (0 on G).
// first != 0: v is zero (start of a run).  CTA 0 stores beta in nxt.
template <typename V, int TPR>
__global__ void __launch_bounds__(kLT)
    lsqr_atu_kernel(int64_t n, int64_t m, const int64_t *__restrict__ ptr, const int32_t *__restrict__ idx,
                    const V *__restrict__ val, const V *__restrict__ D,
                    const uint8_t *__restrict__ inF, const V *__restrict__ u, V *__restrict__ v,
                    const double *__restrict__ part_u, int n_part_u, LsqrScalars *nxt,
                    double *__restrict__ part_v) {
    __shared__ double sh[kLT / 32];
    const double ssq = sum_partials(part_u, n_part_u, sh);
    const double beta = cta_bcast(threadIdx.x == 0 ? sqrt(ssq) : 0.0, sh);
    if (blockIdx.x == 0 && threadIdx.x == 0) nxt->beta = beta;
    const V inv_beta = (V)cta_bcast(threadIdx.x == 0 ? safe_div(1.0, beta) : 0.0, sh);
    const V vbeta = (V)beta;
    const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride_rows = ((int64_t)gridDim.x * blockDim.x) / TPR;
    const int sub = threadIdx.x % TPR;
    const int64_t warp_row0 = ((gtid >> 5) << 5) / TPR;
    const int64_t my_off = (gtid / TPR) - warp_row0;
    double acc = 0.0;
    for (int64_t j0 = warp_row0; j0 < n; j0 += stride_rows) {
        const int64_t j = j0 + my_off;
        const bool active = j < n && inF[j];
        V s = V(0);
        if (active) {
            const int64_t p1 = ptr[j + 1];
            for (int64_t p = ptr[j] + sub; p < p1; p += 4 * TPR) {
                int32_t c[4];
                V a[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const bool in = p + q * TPR < p1;
                    c[q] = in ? idx[p + q * TPR] : 0;
                    a[q] = in ? val[p + q * TPR] : V(0);
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) s += TS_IN(c[q], m) ? a[q] * u[c[q]] : V(0);
            }
        }
#pragma unroll
        for (int o = TPR / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, TPR);
        if (sub == 0 && j < n) {
            const V vn = active ? D[j] * (s * inv_beta) - vbeta * v[j] : V(0);
            v[j] = vn;
            acc += (double)vn * (double)vn;
        }
    }
    write_partial(acc, part_v, sh);
}

// upd: alpha = ||v^||, v = v^/alpha; the plane rotation of the bidiagonal;
// z += (phi/rho) w, w = v - (theta/rho) w.  init != 0: first alpha (w = v).
template <typename V>
__global__ void __launch_bounds__(kLT)
    lsqr_update_kernel(int64_t n, V *__restrict__ v, V *__restrict__ w, V *__restrict__ z,
                       const V *__restrict__ D, V *__restrict__ dv, const double *__restrict__ part_v,
                       int n_part_v, const LsqrScalars *__restrict__ cur, LsqrScalars *nxt, int init) {
    __shared__ double sh[kLT / 32];
    __shared__ double scal[6];  // alpha, 1/alpha, f1, f2, next rhobar, next phibar
    const double ssq = sum_partials(part_v, n_part_v, sh);
    if (threadIdx.x == 0) {
        const double alpha = sqrt(ssq);
        scal[0] = alpha;
        scal[1] = safe_div(1.0, alpha);
        if (init) {
            scal[2] = scal[3] = 0.0;
            scal[4] = alpha;
            scal[5] = nxt->beta;
        } else {
            const double beta = nxt->beta;  // written by the preceding atu launch
            const double rhobar = cur->rhobar, phibar = cur->phibar;
            const double rho = sqrt(rhobar * rhobar + beta * beta);
            const double c = safe_div(rhobar, rho), s = safe_div(beta, rho);
            scal[2] = safe_div(c * phibar, rho);  // phi / rho
            scal[3] = safe_div(s * alpha, rho);   // theta / rho
            scal[4] = -c * alpha;
            scal[5] = s * phibar;
        }
    }
    __syncthreads();
    const V inv_alpha = (V)scal[1], f1 = (V)scal[2], f2 = (V)scal[3];
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const V vn = v[j] * inv_alpha;
        v[j] = vn;
        dv[j] = D[j] * vn;
        if (init) {
            w[j] = vn;
        } else {
            const V wj = w[j];
            z[j] += f1 * wj;
            w[j] = vn - f2 * wj;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        nxt->alpha = scal[0];
        nxt->rhobar = scal[4];
        nxt->phibar = scal[5];
    }
}

// x_F += D z (FP64), ||D z||_inf and ||x_F||_inf into the status.
template <typename V>
__global__ void __launch_bounds__(1024)
    lsqr_apply_kernel(int64_t n, const uint8_t *__restrict__ inF, const V *__restrict__ D,
                      const V *__restrict__ z, double *__restrict__ x, DevStatus *st) {
    __shared__ double shd[32], shx[32];
    double dm = 0.0, xm = 0.0;
    for (int64_t j = threadIdx.x; j < n; j += 1024) {
        if (!inF[j]) continue;
        const double d = (double)D[j] * (double)z[j];
        const double xn = x[j] + d;
        x[j] = xn;
        dm = fmax(dm, fabs(d));
        xm = fmax(xm, fabs(xn));
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, o));
        xm = fmax(xm, __shfl_xor_sync(0xffffffffu, xm, o));
    }
    if (lane == 0) { shd[warp] = dm; shx[warp] = xm; }
    __syncthreads();
    if (warp == 0) {
        dm = shd[lane];
        xm = shx[lane];
        for (int o = 16; o > 0; o >>= 1) {
            dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, o));
            xm = fmax(xm, __shfl_xor_sync(0xffffffffu, xm, o));
        }
        if (lane == 0) { st->dnorm = dm; st->xnorm = xm; }
    }
}

// After an exchange: keep x on F (warm start of the next LSQR run), 0 on G.
__global__ void keep_x_on_F_kernel(int64_t n, const uint8_t *__restrict__ inF,
                                   double *__restrict__ x, const double *__restrict__ x_prev) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x)
        x[j] = inF[j] ? x_prev[j] : 0.0;
}

namespace {

inline int grid_for(int64_t rows, int tpr) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(rows * tpr, kLT), partial_cap()));
}

template <typename V>
struct LsqrLaunch {
    cudaStream_t s;
    int64_t m, n;
    const int64_t *row_ptr, *col_ptr;
    const int32_t *col, *row_idx;
    const V *val, *cval;
    const V *D;
    const uint8_t *inF;
    V *u, *v, *w, *z, *dv;
    double *part_u, *part_v;
    LsqrScalars *sc;  // [2]
    int tpr_r, tpr_c;

    template <int TPR>
    void av(const LsqrScalars *cur) {
        const bool vec = sizeof(V) == 4 && (reinterpret_cast<uintptr_t>(col) & 15) == 0 &&
                         (reinterpret_cast<uintptr_t>(val) & 15) == 0;
        lsqr_av_kernel<V, TPR><<<grid_for(m, TPR), kLT, 0, s>>>(m, n, row_ptr, col, val, dv, u, cur, part_u, vec);
        note_launches(1);
    }
    template <int TPR>
    void atu(LsqrScalars *nxt) {
        lsqr_atu_kernel<V, TPR><<<grid_for(n, TPR), kLT, 0, s>>>(n, m, col_ptr, row_idx, cval, D, inF, u, v,
                                                                  part_u, grid_for(m, tpr_r), nxt, part_v);
        note_launches(1);
    }
    void av_any(const LsqrScalars *cur) {
        switch (tpr_r) {
            case 1: av<1>(cur); break;
            case 4: av<4>(cur); break;
            case 8: av<8>(cur); break;
            case 16: av<16>(cur); break;
            default: av<32>(cur); break;
        }
    }
    void atu_any(LsqrScalars *nxt) {
        switch (tpr_c) {
            case 4: atu<4>(nxt); break;
            case 8: atu<8>(nxt); break;
            case 16: atu<16>(nxt); break;
            default: atu<32>(nxt); break;
        }
    }
    void vstart(const double *s_atr, LsqrScalars *nxt) {
        const int g = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(n, kLT), partial_cap()));
        lsqr_vstart_kernel<V><<<g, kLT, 0, s>>>(n, s_atr, D, inF, v, part_u, grid_for(m, tpr_r), nxt, part_v);
        note_launches(1);
        vstart_grid = g;
    }
    int vstart_grid = 0;
    void upd(const LsqrScalars *cur, LsqrScalars *nxt, int init) {
        const int g = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(n, kLT), partial_cap()));
        const int nparts = init ? vstart_grid : grid_for(n, tpr_c);
        lsqr_update_kernel<V><<<g, kLT, 0, s>>>(n, v, w, z, D, dv, part_v, nparts, cur, nxt, init);
        note_launches(1);
    }
};

// lanes per row (column) of a sparse product by the average row length;
// rows of up to 16 nonzeros get a thread each
inline int tpr_for(double avg) { return avg <= 16 ? 1 : avg <= 24 ? 16 : 32; }
inline int tpr_for_cols(double avg) { return avg <= 6 ? 4 : avg <= 12 ? 8 : avg <= 24 ? 16 : 32; }

#define TRY_CUDA_L(expr)                   \
    do {                                   \
        cudaError_t e_ = (expr);           \
        if (e_ != cudaSuccess) {           \
            status = status_from_cuda(e_); \
            goto cleanup;                  \
        }                                  \
    } while (0)

template <typename V>
size_t lsqr_layout(int64_t m, int64_t n, int64_t nnz, bool host_in) {
    size_t b = 0;
    auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
    if (host_in) b += up(8 * (m + 1)) + up(4 * nnz) + up(8 * nnz) + up(8 * m);
    b += up(quality_scratch_bytes(m, n));
    b += up(8 * (n + 1)) + up(4 * nnz) + up(8 * nnz) + up(4 * (n + 1)) + up(8 * (n + 1));  // CSC
    b += 2 * up(sizeof(V) * nnz) + up(sizeof(V) * n);  // value copies, D
    b += 5 * up(8 * n) + up(8 * m);                     // c, x, y, s, xprev; r
    b += up(sizeof(V) * m) + 4 * up(sizeof(V) * n);     // u; v, w, z, D v
    b += up(n) + up(4 * n) + 2 * up(8 * kMaxPartials) + up(2 * sizeof(LsqrScalars));
    return b + 256;
}

}  // namespace

size_t lsqr_footprint(const tsnnls_csr &A, const tsnnls_opts &o) {
    const bool host_in = A.on_device == 0;
    return o.precision == TSNNLS_FP64 ? lsqr_layout<double>(A.m, A.n, A.nnz, host_in)
                                      : lsqr_layout<float>(A.m, A.n, A.nnz, host_in);
}

template <typename V>
int solve_lsqr_t(Context &ctx, Lane &lane, const tsnnls_csr &A, const double *b, double *x_out,
                 const tsnnls_opts &o, tsnnls_info *info, const SolveExtras *ex) {
    (void)ctx;
    const int64_t m = A.m, n = A.n, nnz = A.nnz;
    const bool host_in = A.on_device == 0;
    const bool mixed = o.precision == TSNNLS_MIXED;
    const int32_t max_iter = o.max_iter > 0 ? o.max_iter : (int32_t)std::min<int64_t>(10 * n + 100, INT32_MAX);
    // inner LSQR steps per outer FP64 correction
    const int inner = mixed ? 24 : 64;
    cudaStream_t s = lane.stream;
    int status = TSNNLS_OK;
    int outer_total = 0, inner_total = 0;
    int last_steps = 0;  // outer corrections of the last pivot (its z is the last one)
    double last_rel = 0.0;
    int64_t trace_rows = 0;
    const int64_t launch0 = launches_so_far();
    cudaGraphExec_t corr_exec = nullptr;  // one correction's launches, replayed
    int64_t corr_launches = 0;
    auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
    char *blk = nullptr;
    char *p = nullptr;
    auto take = [&](size_t bytes) {
        char *q = p;
        p += up(std::max<size_t>(bytes, 1));
        return q;
    };
    {
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&blk), lsqr_layout<V>(m, n, nnz, host_in), s);
        if (e != cudaSuccess) return status_from_cuda(e);
    }
    p = blk;
    const int64_t *row_ptr;
    const int32_t *col;
    const double *val;
    const double *bd;
    if (host_in) {
        int64_t *rp = (int64_t *)take(8 * (m + 1));
        int32_t *ci = (int32_t *)take(4 * nnz);
        double *va = (double *)take(8 * nnz);
        double *bb = (double *)take(8 * m);
        TRY_CUDA_L(cudaMemcpyAsync(rp, A.row_ptr, 8 * (m + 1), cudaMemcpyHostToDevice, s));
        if (nnz > 0) {
            TRY_CUDA_L(cudaMemcpyAsync(ci, A.col_idx, 4 * nnz, cudaMemcpyHostToDevice, s));
            TRY_CUDA_L(cudaMemcpyAsync(va, A.val, 8 * nnz, cudaMemcpyHostToDevice, s));
        }
        TRY_CUDA_L(cudaMemcpyAsync(bb, b, 8 * m, cudaMemcpyHostToDevice, s));
        row_ptr = rp;
        col = ci;
        val = va;
        bd = bb;
    } else {
        row_ptr = A.row_ptr;
        col = A.col_idx;
        val = A.val;
        bd = b;
    }
    {
        void *qscratch = take(quality_scratch_bytes(m, n));
        int64_t *col_ptr = (int64_t *)take(8 * (n + 1));
        int32_t *row_idx = (int32_t *)take(4 * nnz);
        double *cval = (double *)take(8 * nnz);
        int32_t *cnt = (int32_t *)take(4 * (n + 1));
        int64_t *next = (int64_t *)take(8 * (n + 1));
        V *val_v = (V *)take(sizeof(V) * nnz);
        V *cval_v = (V *)take(sizeof(V) * nnz);
        V *D = (V *)take(sizeof(V) * n);
        double *c = (double *)take(8 * n);
        double *x = (double *)take(8 * n);
        double *y = (double *)take(8 * n);
        double *sv = (double *)take(8 * n);
        double *xprev = (double *)take(8 * n);
        double *r = (double *)take(8 * m);
        V *u = (V *)take(sizeof(V) * m);
        V *v = (V *)take(sizeof(V) * n);
        V *w = (V *)take(sizeof(V) * n);
        V *z = (V *)take(sizeof(V) * n);
        V *dv = (V *)take(sizeof(V) * n);
        uint8_t *inF = (uint8_t *)take(n);
        int32_t *F = (int32_t *)take(4 * n);
        double *part_u = (double *)take(8 * kMaxPartials);
        double *part_v = (double *)take(8 * kMaxPartials);
        LsqrScalars *sc = (LsqrScalars *)take(2 * sizeof(LsqrScalars));
        const double avg_row = (double)nnz / (double)m, avg_col = (double)nnz / (double)n;
        const double csr_bytes = 12.0 * nnz + 8.0 * (m + 1);
        const double csc_bytes = 12.0 * nnz + 8.0 * (n + 1);
        LsqrLaunch<V> L{s, m, n, row_ptr, col_ptr, col, row_idx, val_v, cval_v, D, inF,
                        u, v, w, z, dv, part_u, part_v, sc, tpr_for(avg_row), tpr_for_cols(avg_col)};
        const int gconv = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(nnz, 256), num_sms() * 8));

        TRY_CUDA_L(cudaEventRecord(lane.ev0, s));
        prof_begin(lane, TSNNLS_PHASE_SETUP);
        TRY_CUDA_L(cudaMemsetAsync(lane.bad_dev, 0, sizeof(int32_t), s));
        TRY_CUDA_L(launch_validate(s, m, n, nnz, row_ptr, col, val, bd, lane.bad_dev));
        TRY_CUDA_L(cudaMemcpyAsync(lane.bad_host, lane.bad_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        TRY_CUDA_L(cudaStreamSynchronize(s));
        if (*lane.bad_host != 0) {
            status = TSNNLS_EINVAL;
            goto cleanup;
        }
        TRY_CUDA_L(launch_csr_to_csc(s, m, n, nnz, row_ptr, col, val, col_ptr, row_idx, cval, cnt, next));
        convert_kernel<V><<<gconv, 256, 0, s>>>(nnz, val, val_v);
        convert_kernel<V><<<gconv, 256, 0, s>>>(nnz, cval, cval_v);
        lsqr_prep_kernel<V><<<(int)std::max<int64_t>(1, std::min<int64_t>(cdiv(n, 256), num_sms() * 8)), 256, 0, s>>>(
            n, col_ptr, cval, D);
        note_launches(3);
        prof_end(lane, 2.0 * csr_bytes + 2.0 * csc_bytes + 2.0 * sizeof(V) * nnz, 0.0);
        // c = A^T b (FP64), then F = {}, x = 0, y = -c
        prof_begin(lane, TSNNLS_PHASE_SPMV);
        TRY_CUDA_L(launch_spmv(s, n, col_ptr, row_idx, cval, 1.0, bd, m, 0.0, nullptr, c, avg_col));
        prof_end(lane, csc_bytes + 8.0 * (m + n), 2.0 * nnz);
        TRY_CUDA_L(launch_init_state(s, n, c, x, y, inF, o.p_max, lane.st_dev));

        for (int pivot_range = 1;; ++pivot_range) {
            nvtx_pivot(lane, pivot_range);
            // keep the current x as the warm start of the next LSQR run
            TRY_CUDA_L(cudaMemcpyAsync(xprev, x, 8 * n, cudaMemcpyDeviceToDevice, s));
            prof_begin(lane, TSNNLS_PHASE_EXCHANGE);
            TRY_CUDA_L(launch_exchange(s, n, x, y, inF, F, o.zero_tol, o.p_max, max_iter,
                                       lane.st_host->iters > 0 ? 1 : 0, lane.st_dev));
            prof_end(lane, 38.0 * n, 0.0);
            {
                cudaError_t e = cudaMemcpyAsync(lane.st_host, lane.st_dev, sizeof(DevStatus),
                                                cudaMemcpyDeviceToHost, s);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s);
                TRY_CUDA_L(e);
            }
            const DevStatus st = *lane.st_host;
            if (st.done) {
                if (st.maxiter_hit) status = TSNNLS_EMAXITER;
                break;
            }
            if (ex && ex->trace && trace_rows < ex->trace_cap) {
                int64_t *t = ex->trace + kTraceCols * trace_rows;
                t[0] = st.n_inf;
                t[1] = -1;
                t[2] = st.p;
                t[3] = st.branch;
                t[4] = st.k;
                t[5] = st.moved;
            }
            keep_x_on_F_kernel<<<(int)std::max<int64_t>(1, std::min<int64_t>(cdiv(n, 256), num_sms() * 8)), 256, 0, s>>>(
                n, inF, x, xprev);
            note_launches(1);
            const int64_t k = st.k;
            double prev = 1e300;
            int steps = 0;
            bool conv = k == 0;
            for (;;) {
                // FP64 residual r = b - A x and, for y and the stop test, s = A^T r
                prof_begin(lane, TSNNLS_PHASE_SPMV);
                TRY_CUDA_L(launch_spmv(s, m, row_ptr, col, val, -1.0, x, n, 1.0, bd, r, avg_row));
                prof_end(lane, csr_bytes + 8.0 * (3.0 * m + n), 2.0 * nnz);
                if (conv) break;
                // inner LSQR on (A_F D) z = r.  The correction's launches are
                // the same every time (every choice above is fixed per solve,
                // the data lives on the device): captured into a graph on the
                // first correction and replayed after, so the device starts
                // each of its 3 inner + 4 kernels sooner
                prof_begin(lane, TSNNLS_PHASE_LSQR);
                {
                    auto issue = [&]() -> cudaError_t {
                        lsqr_start_kernel<V><<<grid_for(m, L.tpr_r), kLT, 0, s>>>(m, n, r, u, v, w, z, part_u);
                        note_launches(1);
                        const cudaError_t e = launch_spmv(s, n, col_ptr, row_idx, cval, 1.0, r, m, 0.0, nullptr,
                                                          sv, avg_col);
                        if (e != cudaSuccess) return e;
                        L.vstart(sv, &sc[0]);
                        L.upd(&sc[0], &sc[0], 1);
                        for (int it = 0; it < inner; ++it) {
                            LsqrScalars *cur = &sc[it & 1], *nxt = &sc[(it + 1) & 1];
                            L.av_any(cur);
                            L.atu_any(nxt);
                            L.upd(cur, nxt, 0);
                        }
                        return cudaGetLastError();
                    };
                    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
                    TRY_CUDA_L(cudaStreamIsCapturing(s, &cs));
                    if (corr_exec) {
                        TRY_CUDA_L(cudaGraphLaunch(corr_exec, s));
                        note_launches(corr_launches);
                    } else if (cs != cudaStreamCaptureStatusNone) {
                        TRY_CUDA_L(issue());  // inside a caller's own capture
                    } else {
                        const int64_t l0 = launches_so_far();
                        TRY_CUDA_L(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
                        const cudaError_t ei = issue();
                        cudaGraph_t graph = nullptr;
                        const cudaError_t ee = cudaStreamEndCapture(s, &graph);
                        if (ei != cudaSuccess || ee != cudaSuccess) {
                            if (graph) cudaGraphDestroy(graph);
                            TRY_CUDA_L(ei != cudaSuccess ? ei : ee);
                        }
                        const cudaError_t eg = cudaGraphInstantiate(&corr_exec, graph, 0);
                        cudaGraphDestroy(graph);
                        if (eg != cudaSuccess) corr_exec = nullptr;
                        TRY_CUDA_L(eg);
                        corr_launches = launches_so_far() - l0;
                        TRY_CUDA_L(cudaGraphLaunch(corr_exec, s));
                    }
                }
                // per inner step: both sparse products (index + value per nonzero,
                // the row/column pointers), the u and v vectors and D, F flags
                prof_end(lane, (double)inner * (2.0 * (4.0 + sizeof(V)) * nnz + 8.0 * (m + 1) +
                                                 8.0 * (n + 1) + sizeof(V) * (3.0 * m + 6.0 * n) + n),
                         (double)inner * 4.0 * nnz);
                inner_total += inner;
                prof_begin(lane, TSNNLS_PHASE_VECTOR);
                lsqr_apply_kernel<V><<<1, 1024, 0, s>>>(n, inF, D, z, x, lane.st_dev);
                note_launches(1);
                prof_end(lane, (2.0 * sizeof(V) + 17.0) * n, 0.0);
                {
                    cudaError_t e = cudaMemcpyAsync(lane.st_host, lane.st_dev, sizeof(DevStatus),
                                                    cudaMemcpyDeviceToHost, s);
                    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
                    TRY_CUDA_L(e);
                }
                ++steps;
                ++outer_total;
                const double d = lane.st_host->dnorm, xn = lane.st_host->xnorm;
                last_rel = xn > 0 ? d / xn : 0.0;
                if (d <= o.rel_tol * xn) conv = true;
                else if (steps > 2 && d > 0.5 * prev && d <= 1e-9 * xn) conv = true;
                else if (steps >= o.max_refine) {
                    if (d <= 1e-9 * xn) conv = true;
                    else { status = TSNNLS_ENOCONV; goto cleanup; }
                }
                prev = d;
            }
            prof_begin(lane, TSNNLS_PHASE_SPMV);
            TRY_CUDA_L(launch_spmv(s, n, col_ptr, row_idx, cval, 1.0, r, m, 0.0, nullptr, sv, avg_col));
            prof_end(lane, csc_bytes + 8.0 * (m + n), 2.0 * nnz);
            TRY_CUDA_L(launch_y_from_s(s, n, sv, inF, y));
            last_steps = steps;
            ++trace_rows;
        }
        if (status == TSNNLS_OK) {
            if (trace_rows == 0) {  // no pivot ran: r and s of x = 0
                TRY_CUDA_L(launch_spmv(s, m, row_ptr, col, val, -1.0, x, n, 1.0, bd, r, avg_row));
                TRY_CUDA_L(launch_spmv(s, n, col_ptr, row_idx, cval, 1.0, r, m, 0.0, nullptr, sv, avg_col));
            }
            // KKT violation and the residual change of the last correction D z
            prof_begin(lane, TSNNLS_PHASE_VECTOR);
            TRY_CUDA_L(launch_quality_scaled<V>(s, m, n, row_ptr, col, val, avg_row, x, sv, c, r, D, z, inF,
                                                last_steps > 0, qscratch, lane.st_dev));
            prof_end(lane, 8.0 * (2.0 * m + 4.0 * n) + (last_steps > 0 ? csr_bytes + 16.0 * m : 0.0), 0.0);
            TRY_CUDA_L(cudaEventRecord(lane.ev1, s));
            TRY_CUDA_L(cudaMemcpyAsync(lane.st_host, lane.st_dev, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
            const cudaMemcpyKind kind = host_in ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
            TRY_CUDA_L(cudaMemcpyAsync(x_out, x, 8 * n, kind, s));
            if (ex && ex->y_out) TRY_CUDA_L(cudaMemcpyAsync(ex->y_out, y, 8 * n, kind, s));
            if (ex && ex->inF_out) TRY_CUDA_L(cudaMemcpyAsync(ex->inF_out, inF, (size_t)n, kind, s));
            TRY_CUDA_L(cudaStreamSynchronize(s));
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, lane.ev0, lane.ev1) == cudaSuccess && info) info->time_ms = ms;
        }
        if (info) {
            info->iters = lane.st_host->iters;
            info->nF = lane.st_host->k;
            if (status == TSNNLS_OK) {
                info->kkt_viol = lane.st_host->kkt_viol;
                info->rel_resid_change = lane.st_host->resid_change;
            }
        }
    }
cleanup:
    cudaFreeAsync(blk, s);
    cudaStreamSynchronize(s);
    if (corr_exec) cudaGraphExecDestroy(corr_exec);
    prof_flush(lane);
    if (ex && ex->trace) {
        int64_t best = INT64_MAX;
        for (int64_t i = 0; i < std::min(trace_rows, ex->trace_cap); ++i) {
            ex->trace[kTraceCols * i + 1] = best;
            best = std::min(best, ex->trace[kTraceCols * i]);
        }
    }
    if (info) {
        info->status = status;
        info->refine_steps = outer_total;
        info->last_rel_step = last_rel;
        info->path_used = TSNNLS_PATH_LSQR;
        info->precision_used = o.precision;
        info->kernel_launches = launches_so_far() - launch0;
        (void)inner_total;
    }
    return status;
}

int solve_lsqr(Context &ctx, Lane &lane, const tsnnls_csr &A, const double *b, double *x_out,
               const tsnnls_opts &o, tsnnls_info *info, const SolveExtras *ex) {
    if (o.precision == TSNNLS_FP64) return solve_lsqr_t<double>(ctx, lane, A, b, x_out, o, info, ex);
    return solve_lsqr_t<float>(ctx, lane, A, b, x_out, o, info, ex);
}

}  // namespace tsnnls

TSNNLS_CHECK_UNIT("lsqr")
