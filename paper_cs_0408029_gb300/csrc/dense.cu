// Gather of the F x F block of the cached A^T A (Section 3) into the
// factorisation workspace.  Column-major with an explicit leading dimension;
// only lower triangles are read or written.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace tsnnls {

// Map a linear block index onto the lower-triangular tile (I, J), I >= J.
__device__ __forceinline__ void tri_tile(int64_t b, int64_t &I, int64_t &J) {
    int64_t i = (int64_t)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
    while (i * (i + 1) / 2 > b) --i;
    while ((i + 1) * (i + 2) / 2 <= b) ++i;
    I = i;
    J = b - i * (i + 1) / 2;
}

// ---------------------------------------------------------------------------
// Gather S = G_FF (lower).  32 x 32 tiles of S; the F indices of the tile's
// rows and columns are staged in shared memory.

template <typename T>
__global__ void __launch_bounds__(256)
    gather_kernel(const T *__restrict__ G, int64_t ldg, const int32_t *__restrict__ F,
                  const int32_t *__restrict__ k_dev, int64_t k_host, T *__restrict__ S,
                  int64_t lds) {
    __shared__ int32_t fr[32], fc[32];
    const int64_t k = k_dev ? (int64_t)*k_dev : k_host;
    const int64_t T_ = cdiv(k, 32);
    int64_t I, J;
    tri_tile(blockIdx.x, I, J);
    if (I >= T_) return;
    const int64_t a0 = I * 32, b0 = J * 32;
    if (threadIdx.x < 32) {
        int64_t a = a0 + threadIdx.x;
        fr[threadIdx.x] = a < k ? F[a] : 0;
    } else if (threadIdx.x < 64) {
        int64_t b = b0 + threadIdx.x - 32;
        fc[threadIdx.x - 32] = b < k ? F[b] : 0;
    }
    __syncthreads();
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t a = a0 + tx;
    for (int q = ty; q < 32; q += 8) {
        const int64_t bcol = b0 + q;
        if (a < k && bcol < k && a >= bcol)
            S[a + bcol * lds] = G[(int64_t)fr[tx] + (int64_t)fc[q] * ldg];
    }
}

template <typename T>
cudaError_t launch_gather(cudaStream_t s, const T *G, int64_t ldg, const int32_t *F,
                          const int32_t *k_dev, int64_t k_max, T *S, int64_t lds) {
    if (k_max <= 0) return cudaSuccess;
    const int64_t t = cdiv(k_max, 32);
    gather_kernel<T><<<(unsigned)(t * (t + 1) / 2), 256, 0, s>>>(G, ldg, F, k_dev, k_max, S, lds);
    note_launches(1);
    return cudaGetLastError();
}

template cudaError_t launch_gather<float>(cudaStream_t, const float *, int64_t, const int32_t *,
                                          const int32_t *, int64_t, float *, int64_t);
template cudaError_t launch_gather<double>(cudaStream_t, const double *, int64_t,
                                           const int32_t *, const int32_t *, int64_t, double *,
                                           int64_t);

}  // namespace tsnnls
