// The exchange step of the block principal pivoting loop (Section 2,
// algorithm box) and the small vector kernels around the solve.
//
// The exchange runs in one CTA: it applies the 1e-12 zeroing, counts the
// infeasible variables (negative entries of x_F and y_G), runs the N / p
// state machine, flips the F/G flags, and rebuilds the ascending F list with
// a block-wide prefix sum.  Integer work only after the sign tests, so its
// decisions are exact.
#include <cuda_runtime.h>
#include <stdint.h>

#include "check.cuh"
#include "common.cuh"

namespace tsnnls {

constexpr int kExThreads = 1024;

__global__ void init_state_kernel(int64_t n, const double *__restrict__ c, double *__restrict__ x,
                                  double *__restrict__ y, uint8_t *__restrict__ inF, int32_t p_max,
                                  DevStatus *st) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        x[j] = 0.0;
        y[j] = -c[j];  // y = -A^T b, as printed (no zeroing of the initial y)
        inF[j] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->k = 0;
        st->n_inf = -1;
        st->N = INT64_MAX;
        st->p = p_max;
        st->branch = -1;
        st->moved = -1;
        st->done = 0;
        st->iters = 0;
        st->chol_info = 0;
        st->timeout = 0;
        st->maxiter_hit = 0;
        st->dnorm = 0.0;
        st->xnorm = 0.0;
    }
}

cudaError_t launch_init_state(cudaStream_t s, int64_t n, const double *c, double *x, double *y,
                              uint8_t *inF, int32_t p_max, DevStatus *st) {
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(n, 256), num_sms() * 8));
    init_state_kernel<<<g, 256, 0, s>>>(n, c, x, y, inF, p_max, st);
    note_launches(1);
    return cudaGetLastError();
}

// Block-wide sum / max helpers for 1024 threads.
__device__ __forceinline__ int64_t block_sum_i64(int64_t v, int64_t *sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = sh[lane];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sh[0] = v;
    }
    __syncthreads();
    return sh[0];
}

__device__ __forceinline__ int64_t block_max_i64(int64_t v, int64_t *sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = sh[lane];
        for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) sh[0] = v;
    }
    __syncthreads();
    return sh[0];
}

__device__ __forceinline__ bool infeasible(uint8_t f, double xv, double yv) {
    return f ? (xv < 0.0) : (yv < 0.0);
}

__global__ void __launch_bounds__(kExThreads)
    exchange_kernel(int64_t n, double *__restrict__ x, double *__restrict__ y,
                    uint8_t *__restrict__ inF, int32_t *__restrict__ F, double zero_tol,
                    int32_t p_max, int32_t max_iter, int32_t apply_zeroing, DevStatus *st) {
    __shared__ int64_t sh[32];
    __shared__ int32_t decision;  // -1: stop, 0/1: full exchange, 2: single
    __shared__ int64_t carry;
    const int tid = threadIdx.x;

    // zeroing of near-zero entries of x_F and y_G (Section 2); x_G = y_F = 0
    int64_t cnt = 0, largest = -1;
    for (int64_t j = tid; j < n; j += kExThreads) {
        const uint8_t f = inF[j];
        double xv = x[j], yv = y[j];
        if (apply_zeroing) {
            if (f) {
                if (fabs(xv) < zero_tol) xv = 0.0;
                yv = 0.0;
            } else {
                xv = 0.0;
                if (fabs(yv) < zero_tol) yv = 0.0;
            }
            x[j] = xv;
            y[j] = yv;
        }
        if (infeasible(f, xv, yv)) {
            ++cnt;
            largest = j;
        }
    }
    const int64_t n_inf = block_sum_i64(cnt, sh);
    const int64_t big = block_max_i64(largest, sh);

    if (tid == 0) {
        st->n_inf = (int32_t)n_inf;
        st->done = 0;
        int32_t d;
        if (n_inf == 0) {
            st->done = 1;
            d = -1;
        } else if (st->iters >= max_iter) {
            st->maxiter_hit = 1;
            st->done = 1;
            d = -1;
        } else if (n_inf < st->N) {
            st->N = n_inf;
            st->p = p_max;
            d = 0;
        } else if (st->p > 0) {
            st->p -= 1;
            d = 1;
        } else {
            d = 2;
        }
        st->branch = d;
        st->moved = d == 2 ? (int32_t)big : -1;
        decision = d;
    }
    __syncthreads();
    const int32_t d = decision;
    if (d < 0) return;

    // exchange between F and G
    if (d == 2) {
        if (tid == 0 && TS_IN(big, n)) inF[big] ^= 1;
    } else {
        for (int64_t j = tid; j < n; j += kExThreads)
            if (infeasible(inF[j], x[j], y[j])) inF[j] ^= 1;
    }
    __syncthreads();

    // ascending F list by prefix sum; x restarts from 0 for the new solve
    if (tid == 0) carry = 0;
    __syncthreads();
    const int lane = tid & 31, warp = tid >> 5;
    for (int64_t base = 0; base < n; base += kExThreads) {
        const int64_t j = base + tid;
        const int v = (j < n) ? (int)inF[j] : 0;
        const unsigned bal = __ballot_sync(0xffffffffu, v);
        const int before_in_warp = __popc(bal & ((1u << lane) - 1u));
        if (lane == 0) sh[warp] = __popc(bal);
        __syncthreads();
        if (warp == 0) {
            int64_t w = sh[lane];
            for (int o = 1; o < 32; o <<= 1) {
                int64_t t = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += t;
            }
            sh[lane] = w;  // inclusive warp prefix
        }
        __syncthreads();
        const int64_t pos = carry + (warp > 0 ? sh[warp - 1] : 0) + before_in_warp;
        if (v) F[pos] = (int32_t)j;
        if (j < n) x[j] = 0.0;
        __syncthreads();
        if (tid == 0) carry += sh[31];
        __syncthreads();
    }
    if (tid == 0) {
        st->k = (int32_t)carry;
        st->iters += 1;
    }
}

cudaError_t launch_exchange(cudaStream_t s, int64_t n, double *x, double *y, uint8_t *inF,
                            int32_t *F, double zero_tol, int32_t p_max, int32_t max_iter,
                            int32_t apply_zeroing, DevStatus *st) {
    exchange_kernel<<<1, kExThreads, 0, s>>>(n, x, y, inF, F, zero_tol, p_max, max_iter,
                                             apply_zeroing, st);
    note_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------

template <typename T>
__global__ void gather_rhs_kernel(const double *__restrict__ v, int64_t n, const int32_t *__restrict__ F,
                                  int64_t k, T *__restrict__ out) {
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < k;
         a += (int64_t)gridDim.x * blockDim.x) {
        const int32_t j = F[a];  // -1: a variable held at zero
        out[a] = j >= 0 && TS_IN(j, n) ? (T)v[j] : T(0);
    }
}

template <typename T>
cudaError_t launch_gather_rhs(cudaStream_t s, const double *v, int64_t n, const int32_t *F, int64_t k,
                              T *out) {
    if (k <= 0) return cudaSuccess;
    const int g = (int)std::min<int64_t>(cdiv(k, 256), num_sms() * 8);
    gather_rhs_kernel<T><<<g, 256, 0, s>>>(v, n, F, k, out);
    note_launches(1);
    return cudaGetLastError();
}

template cudaError_t launch_gather_rhs<float>(cudaStream_t, const double *, int64_t, const int32_t *,
                                              int64_t, float *);
template cudaError_t launch_gather_rhs<double>(cudaStream_t, const double *, int64_t, const int32_t *,
                                               int64_t, double *);

// x_F += delta (FP64), and ||delta||_inf, ||x_F||_inf into the status.
// x_F += delta (list order), with max |delta| and max |x_F| into st->dnorm /
// st->xnorm.  Several CTAs; the maxima of non-negative doubles combine through
// integer atomicMax on their bit patterns (same order as the values, so the
// result does not depend on the order of the CTAs).
template <typename T>
__global__ void __launch_bounds__(256)
    update_x_kernel(const T *__restrict__ delta, const int32_t *__restrict__ F, int64_t k,
                    double *__restrict__ x, int64_t n, DevStatus *st) {
    __shared__ double shd[8], shx[8];
    double dm = 0.0, xm = 0.0;
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < k; a += (int64_t)gridDim.x * blockDim.x) {
        const int32_t j = F[a];
        if (j < 0 || !TS_IN(j, n)) continue;  // -1: a variable held at zero
        const double d = (double)delta[a];
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
    if (lane == 0) {
        shd[warp] = dm;
        shx[warp] = xm;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) {
            dm = fmax(dm, shd[w]);
            xm = fmax(xm, shx[w]);
        }
        atomicMax(reinterpret_cast<unsigned long long *>(&st->dnorm), (unsigned long long)__double_as_longlong(dm));
        atomicMax(reinterpret_cast<unsigned long long *>(&st->xnorm), (unsigned long long)__double_as_longlong(xm));
    }
}

template <typename T>
cudaError_t launch_update_x(cudaStream_t s, const T *delta, const int32_t *F, int64_t k,
                            double *x, int64_t n, DevStatus *st) {
    static_assert(offsetof(DevStatus, xnorm) == offsetof(DevStatus, dnorm) + sizeof(double), "adjacent norms");
    cudaError_t e = cudaMemsetAsync(&st->dnorm, 0, 2 * sizeof(double), s);
    if (e != cudaSuccess) return e;
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(k, 256), num_sms()));
    update_x_kernel<T><<<g, 256, 0, s>>>(delta, F, k, x, n, st);
    note_launches(1);
    return cudaGetLastError();
}

template cudaError_t launch_update_x<float>(cudaStream_t, const float *, const int32_t *,
                                            int64_t, double *, int64_t, DevStatus *);
template cudaError_t launch_update_x<double>(cudaStream_t, const double *, const int32_t *,
                                             int64_t, double *, int64_t, DevStatus *);

// ---------------------------------------------------------------------------
// Settled decisions.  Before the last pivot only the signs of x_F and y_G
// (after the 1e-12 zeroing) enter the method (Section 3), so refinement may
// stop once no entry can change its side of the thresholds 0 and +-zero_tol.
// With x known to within E in the max norm, s_i = a_i^T (b - A x) is known
// to within c_i E, c_i = sum_r |a_ri| sum_j |a_rj| >= sum_f |(A^T A)_if|.

__global__ void abs_row_sum_kernel(int64_t m, const int64_t *__restrict__ row_ptr,
                                   const double *__restrict__ val, double *__restrict__ t) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m;
         r += (int64_t)gridDim.x * blockDim.x) {
        double a = 0.0;
        for (int64_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e) a += fabs(val[e]);
        t[r] = a;
    }
}

__global__ void abs_col_dot_kernel(int64_t n, const int64_t *__restrict__ col_ptr,
                                   const int32_t *__restrict__ row_idx, const double *__restrict__ cval,
                                   const double *__restrict__ t, double *__restrict__ c) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        double a = 0.0;
        for (int64_t e = col_ptr[j]; e < col_ptr[j + 1]; ++e) a += fabs(cval[e]) * t[row_idx[e]];
        c[j] = a;
    }
}

cudaError_t launch_gram_row_bound(cudaStream_t s, int64_t m, int64_t n, const int64_t *row_ptr,
                                  const double *val, const int64_t *col_ptr, const int32_t *row_idx,
                                  const double *cval, double *t, double *c) {
    const int gm = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(m, 256), num_sms() * 8));
    const int gn = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(n, 256), num_sms() * 8));
    abs_row_sum_kernel<<<gm, 256, 0, s>>>(m, row_ptr, val, t);
    abs_col_dot_kernel<<<gn, 256, 0, s>>>(n, col_ptr, row_idx, cval, t, c);
    note_launches(2);
    return cudaGetLastError();
}

__global__ void settled_kernel(int64_t n, const uint8_t *__restrict__ inF, const double *__restrict__ x,
                               const double *__restrict__ sv, const double *__restrict__ c, double E,
                               double zero_tol, DevStatus *st) {
    __shared__ int32_t sh[32];
    int32_t cnt = 0;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x) {
        const bool f = inF[j] != 0;
        const double v = fabs(f ? x[j] : sv[j]);  // |x_j| on F, |y_j| = |s_j| on G
        const double e = f ? E : c[j] * E;
        if (!(v >= zero_tol + e || v + e < zero_tol)) ++cnt;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (lane == 0) sh[warp] = cnt;
    __syncthreads();
    if (warp == 0) {
        cnt = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        if (lane == 0 && cnt > 0) atomicAdd(&st->unsettled, cnt);
    }
}

cudaError_t launch_settled(cudaStream_t s, int64_t n, const uint8_t *inF, const double *x,
                           const double *sv, const double *c, double E, double zero_tol, DevStatus *st) {
    cudaError_t e = cudaMemsetAsync(&st->unsettled, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(n, 256), num_sms() * 2));
    settled_kernel<<<g, 256, 0, s>>>(n, inF, x, sv, c, E, zero_tol, st);
    note_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Vector steps of the 1-norm estimate of G^-1 (Hager's method as refined by
// Higham, the estimator behind LAPACK's dpocon): fill a probe vector, take
// ||y||_1 and sign(y), find max_i |z_i| and z^T x.  One CTA each; fixed-order
// reductions.  out: [0] ||y||_1, [1] max |z_i|, [2] its first index, [3] z^T x.

template <typename T>
__global__ void est_fill_kernel(T *__restrict__ v, int64_t k, int32_t mode, int64_t j) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x) {
        double x;
        if (mode == 0) x = 1.0 / (double)k;                                  // uniform
        else if (mode == 1) x = (i == j) ? 1.0 : 0.0;                          // unit vector
        else x = ((i & 1) ? -1.0 : 1.0) * (1.0 + (double)i / (double)(k > 1 ? k - 1 : 1));  // alternating
        v[i] = (T)x;
    }
}

template <typename T>
__global__ void __launch_bounds__(kExThreads)
    est_norm_sign_kernel(const T *__restrict__ y, int64_t k, T *__restrict__ xi, double *out) {
    __shared__ double sh[32];
    double a = 0.0;
    for (int64_t i = threadIdx.x; i < k; i += kExThreads) {
        const double v = (double)y[i];
        a += fabs(v);
        xi[i] = v >= 0.0 ? T(1) : T(-1);
    }
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x < 32) {
        a = sh[threadIdx.x];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (threadIdx.x == 0) out[0] = a;
    }
}

template <typename T>
__global__ void __launch_bounds__(kExThreads)
    est_argmax_kernel(const T *__restrict__ z, int64_t k, int32_t mode, int64_t jprev, double *out) {
    __shared__ double shv[32], shd[32];
    __shared__ int64_t shi[32];
    double best = -1.0, dot = 0.0;
    int64_t arg = 0;
    for (int64_t i = threadIdx.x; i < k; i += kExThreads) {
        const double v = (double)z[i];
        if (fabs(v) > best) {
            best = fabs(v);
            arg = i;
        }
        if (mode == 0) dot += v;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int64_t oa = __shfl_xor_sync(0xffffffffu, arg, o);
        if (ob > best || (ob == best && oa < arg)) {
            best = ob;
            arg = oa;
        }
        dot += __shfl_xor_sync(0xffffffffu, dot, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        shv[warp] = best;
        shi[warp] = arg;
        shd[warp] = dot;
    }
    __syncthreads();
    if (warp == 0) {
        best = shv[lane];
        arg = shi[lane];
        dot = shd[lane];
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int64_t oa = __shfl_xor_sync(0xffffffffu, arg, o);
            if (ob > best || (ob == best && oa < arg)) {
                best = ob;
                arg = oa;
            }
            dot += __shfl_xor_sync(0xffffffffu, dot, o);
        }
        if (lane == 0) {
            out[1] = best;
            out[2] = (double)arg;
            out[3] = mode == 0 ? dot / (double)k : (double)z[jprev];
        }
    }
}

template <typename T>
cudaError_t launch_est_fill(cudaStream_t s, T *v, int64_t k, int32_t mode, int64_t j) {
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(k, 256), num_sms() * 4));
    est_fill_kernel<T><<<g, 256, 0, s>>>(v, k, mode, j);
    note_launches(1);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_est_norm_sign(cudaStream_t s, const T *y, int64_t k, T *xi, double *out) {
    est_norm_sign_kernel<T><<<1, kExThreads, 0, s>>>(y, k, xi, out);
    note_launches(1);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_est_argmax(cudaStream_t s, const T *z, int64_t k, int32_t mode, int64_t jprev, double *out) {
    est_argmax_kernel<T><<<1, kExThreads, 0, s>>>(z, k, mode, jprev, out);
    note_launches(1);
    return cudaGetLastError();
}
template cudaError_t launch_est_fill<float>(cudaStream_t, float *, int64_t, int32_t, int64_t);
template cudaError_t launch_est_fill<double>(cudaStream_t, double *, int64_t, int32_t, int64_t);
template cudaError_t launch_est_norm_sign<float>(cudaStream_t, const float *, int64_t, float *, double *);
template cudaError_t launch_est_norm_sign<double>(cudaStream_t, const double *, int64_t, double *, double *);
template cudaError_t launch_est_argmax<float>(cudaStream_t, const float *, int64_t, int32_t, int64_t, double *);
template cudaError_t launch_est_argmax<double>(cudaStream_t, const double *, int64_t, int32_t, int64_t, double *);

// Eq. 5 from s = A^T (b - A x): y_G = -s_G, y_F = 0.
__global__ void y_from_s_kernel(int64_t n, const double *__restrict__ sv,
                                const uint8_t *__restrict__ inF, double *__restrict__ y) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x)
        y[j] = inF[j] ? 0.0 : -sv[j];
}

cudaError_t launch_y_from_s(cudaStream_t s, int64_t n, const double *sv, const uint8_t *inF,
                            double *y) {
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(n, 256), num_sms() * 8));
    y_from_s_kernel<<<g, 256, 0, s>>>(n, sv, inF, y);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace tsnnls

TSNNLS_CHECK_UNIT("exchange")
