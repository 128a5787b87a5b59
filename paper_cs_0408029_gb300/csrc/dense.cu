// Gather of the F x F block of the cached A^T A (Section 3) into the
// factorisation workspace.  Column-major with an explicit leading dimension;
// only lower triangles are read or written.
#include <cuda_runtime.h>
#include <stdint.h>

#include "check.cuh"
#include "common.cuh"

namespace tsnnls {

// ---------------------------------------------------------------------------
// Gather S = G_FF (lower).  One CTA per 128 x 64 tile of S (tiles wholly
// above the diagonal return at once); the F indices of the tile's rows and
// columns are staged in shared memory.  Thread (tx, ty) owns rows
// a0 + 4 tx .. + 3 of the columns b0 + ty + 8 j, j < 8: its 32 gathered
// loads are all in flight before the first store, and each column's 4 rows
// go out as one vector store when VEC (S 16-byte aligned, lds % 4 == 0).

template <typename T>
__device__ __forceinline__ void st_vec4(T *p, const T (&v)[4]);
template <>
__device__ __forceinline__ void st_vec4<float>(float *p, const float (&v)[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
template <>
__device__ __forceinline__ void st_vec4<double>(double *p, const double (&v)[4]) {
    *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
    *reinterpret_cast<double2 *>(p + 2) = make_double2(v[2], v[3]);
}

constexpr int kGatherRows = 128, kGatherCols = 64;

template <typename T, bool VEC>
__global__ void __launch_bounds__(256)
    gather_kernel(const T *__restrict__ G, int64_t ldg, const int32_t *__restrict__ F,
                  const int32_t *__restrict__ k_dev, int64_t k_host, T *__restrict__ S,
                  int64_t lds) {
    __shared__ int32_t fr[kGatherRows], fc[kGatherCols];
    const int64_t k = k_dev ? (int64_t)*k_dev : k_host;
    const int64_t a0 = (int64_t)blockIdx.x * kGatherRows, b0 = (int64_t)blockIdx.y * kGatherCols;
    if (a0 >= k || b0 >= k || b0 > a0 + kGatherRows - 1) return;  // outside, or above the diagonal
    const int tid = threadIdx.x;
    if (tid < kGatherRows) {
        const int64_t a = a0 + tid;
        const int32_t f = a < k ? F[a] : 0;
        fr[tid] = TS_IN(f, ldg) ? f : 0;
    } else if (tid < kGatherRows + kGatherCols) {
        const int64_t b = b0 + tid - kGatherRows;
        const int32_t f = b < k ? F[b] : 0;
        fc[tid - kGatherRows] = TS_IN(f, ldg) ? f : 0;
    }
    __syncthreads();
    const int tx = tid & 31, ty = tid >> 5;
    const int64_t a = a0 + 4 * tx;
    T v[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int q = ty + 8 * j;
        const int64_t b = b0 + q;
        const T *gc = G + (int64_t)fc[q] * ldg;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t au = a + u;
            v[j][u] = (au < k && b < k && au >= b) ? gc[fr[4 * tx + u]] : T(0);
        }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int64_t b = b0 + ty + 8 * j;
        if (b >= k) continue;
        T *dst = S + a + b * lds;
        if (VEC && a + 3 < k && a >= b) {
            st_vec4<T>(dst, v[j]);
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (a + u < k && a + u >= b) dst[u] = v[j][u];
        }
    }
}

template <typename T>
cudaError_t launch_gather(cudaStream_t s, const T *G, int64_t ldg, const int32_t *F,
                          const int32_t *k_dev, int64_t k_max, T *S, int64_t lds) {
    if (k_max <= 0) return cudaSuccess;
    const dim3 grid((unsigned)cdiv(k_max, kGatherRows), (unsigned)cdiv(k_max, kGatherCols));
    if (lds % 4 == 0 && (reinterpret_cast<uintptr_t>(S) & 15) == 0)
        gather_kernel<T, true><<<grid, 256, 0, s>>>(G, ldg, F, k_dev, k_max, S, lds);
    else
        gather_kernel<T, false><<<grid, 256, 0, s>>>(G, ldg, F, k_dev, k_max, S, lds);
    note_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// ||G_FF||_1 of the symmetric block whose lower triangle G holds: column j
// sums |G(F_i, F_j)| over i >= j (its own column) and over i < j (row j of
// the lower triangle).  Per 128 x 64 tile: column sums over the tile's rows
// go to colpart[I][b], row sums over its strictly lower entries to
// rowpart[J][a] (fixed slots, so the totals are reduced in a fixed order).

template <typename T>
__global__ void __launch_bounds__(256)
    gram_norm_part_kernel(const T *__restrict__ G, int64_t ldg, const int32_t *__restrict__ F, int64_t k,
                          double *__restrict__ colpart, double *__restrict__ rowpart) {
    __shared__ int32_t fr[kGatherRows], fc[kGatherCols];
    __shared__ double rs[8][kGatherRows];
    const int64_t a0 = (int64_t)blockIdx.x * kGatherRows, b0 = (int64_t)blockIdx.y * kGatherCols;
    if (a0 >= k || b0 >= k || b0 > a0 + kGatherRows - 1) return;
    const int tid = threadIdx.x;
    if (tid < kGatherRows) {
        const int64_t a = a0 + tid;
        const int32_t f = a < k ? F[a] : 0;
        fr[tid] = TS_IN(f, ldg) ? f : 0;
    } else if (tid < kGatherRows + kGatherCols) {
        const int64_t b = b0 + tid - kGatherRows;
        const int32_t f = b < k ? F[b] : 0;
        fc[tid - kGatherRows] = TS_IN(f, ldg) ? f : 0;
    }
    __syncthreads();
    const int tx = tid & 31, ty = tid >> 5;
    const int64_t a = a0 + 4 * tx;
    double row[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int q = ty + 8 * j;
        const int64_t b = b0 + q;
        const T *gc = G + (int64_t)fc[q] * ldg;
        double col = 0.0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t au = a + u;
            const double v = (au < k && b < k && au >= b) ? fabs((double)gc[fr[4 * tx + u]]) : 0.0;
            col += v;
            if (au > b) row[u] += v;
        }
        for (int o = 16; o > 0; o >>= 1) col += __shfl_xor_sync(0xffffffffu, col, o);
        if (tx == 0 && b < k) colpart[(int64_t)blockIdx.x * k + b] = col;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) rs[ty][4 * tx + u] = row[u];
    __syncthreads();
    if (tid < kGatherRows && a0 + tid < k) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < 8; ++w) t += rs[w][tid];
        rowpart[(int64_t)blockIdx.y * k + a0 + tid] = t;
    }
}

__global__ void __launch_bounds__(1024)
    gram_norm_reduce_kernel(const double *__restrict__ colpart, const double *__restrict__ rowpart, int64_t k,
                            int64_t nrt, int64_t nct, double *__restrict__ out) {
    __shared__ double sh[32];
    double best = 0.0;
    for (int64_t j = threadIdx.x; j < k; j += blockDim.x) {
        double t = 0.0;
        for (int64_t I = 0; I < nrt; ++I) t += colpart[I * k + j];
        for (int64_t J = 0; J < nct; ++J) t += rowpart[J * k + j];
        best = fmax(best, t);
    }
    for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x < 32) {
        best = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
        if (threadIdx.x == 0) *out = best;
    }
}

size_t gram_norm_scratch_bytes(int64_t k) {
    return (size_t)(cdiv(k, kGatherRows) + cdiv(k, kGatherCols)) * (size_t)std::max<int64_t>(k, 1) * 8;
}

template <typename T>
cudaError_t launch_gram_norm1(cudaStream_t s, const T *G, int64_t ldg, const int32_t *F, int64_t k,
                              double *scratch, double *out) {
    if (k <= 0) return cudaMemsetAsync(out, 0, sizeof(double), s);
    const int64_t nrt = cdiv(k, kGatherRows), nct = cdiv(k, kGatherCols);
    cudaError_t e = cudaMemsetAsync(scratch, 0, gram_norm_scratch_bytes(k), s);
    if (e != cudaSuccess) return e;
    double *colpart = scratch, *rowpart = scratch + nrt * k;
    gram_norm_part_kernel<T><<<dim3((unsigned)nrt, (unsigned)nct), 256, 0, s>>>(G, ldg, F, k, colpart, rowpart);
    gram_norm_reduce_kernel<<<1, 1024, 0, s>>>(colpart, rowpart, k, nrt, nct, out);
    note_launches(2);
    return cudaGetLastError();
}

template cudaError_t launch_gram_norm1<float>(cudaStream_t, const float *, int64_t, const int32_t *, int64_t,
                                             double *, double *);
template cudaError_t launch_gram_norm1<double>(cudaStream_t, const double *, int64_t, const int32_t *, int64_t,
                                              double *, double *);

template cudaError_t launch_gather<float>(cudaStream_t, const float *, int64_t, const int32_t *,
                                          const int32_t *, int64_t, float *, int64_t);
template cudaError_t launch_gather<double>(cudaStream_t, const double *, int64_t,
                                           const int32_t *, const int32_t *, int64_t, double *,
                                           int64_t);

}  // namespace tsnnls

TSNNLS_CHECK_UNIT("dense")
