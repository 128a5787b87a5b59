// Dense kernels of the normal-equations solver (Section 2): the gather of the
// F x F block of the cached A^T A (Section 3), a blocked right-looking
// Cholesky factorisation, and the two triangular solves through the factor.
//
// Layout: every matrix is column-major with an explicit leading dimension;
// only lower triangles are read or written.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cuda/atomic>

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

// ---------------------------------------------------------------------------
// Blocked Cholesky, right-looking, panel width NB:
//   for K = 0, NB, ...:
//     panel:  factor the diagonal block S_KK = L_KK L_KK^T (in shared memory)
//             and solve the block column below it, X L_KK^T = S_(K+NB:, K)
//     update: S_(K+NB:, K+NB:) -= X X^T on the lower tiles
// The panel kernel gives every CTA its own copy of the diagonal block (a few
// microseconds of redundant work) so that the block column needs no second
// launch.

template <typename T, int NB>
struct PanelSmem {
    T D[NB][NB + 1];
};

template <typename T, int NB, int PR>
__global__ void __launch_bounds__(256)
    chol_panel_kernel(T *__restrict__ S, int64_t k, int64_t lds, int64_t K, DevStatus *st) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T(*D)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(smem_raw);            // D[col][row]
    T(*X)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(smem_raw + sizeof(T) * NB * (NB + 1));  // X[row][col]
    __shared__ int bad;
    const int kb = (int)min((int64_t)NB, k - K);
    const int tid = threadIdx.x;
    if (tid == 0) bad = 0;
    for (int e = tid; e < kb * kb; e += blockDim.x) {
        const int c = e / kb, r = e % kb;
        if (r >= c) D[c][r] = S[(K + r) + (K + c) * lds];
    }
    __syncthreads();
    // unblocked Cholesky of the diagonal block, column by column
    for (int j = 0; j < kb; ++j) {
        if (tid == 0) {
            T d = D[j][j];
            if (!(d > T(0))) {
                if (!bad) bad = j + 1;
                d = T(1);
            }
            D[j][j] = sqrt(d);
        }
        __syncthreads();
        const T djj = D[j][j];
        for (int i = j + 1 + tid; i < kb; i += blockDim.x) D[j][i] /= djj;
        __syncthreads();
        const int rem = kb - j - 1;
        for (int e = tid; e < rem * rem; e += blockDim.x) {
            const int l = j + 1 + e / rem, i = j + 1 + e % rem;
            if (i >= l) D[l][i] -= D[j][i] * D[j][l];
        }
        __syncthreads();
    }
    if (blockIdx.x == 0) {
        if (tid == 0 && bad && st->chol_info == 0) st->chol_info = (int32_t)(K + bad);
        for (int e = tid; e < kb * kb; e += blockDim.x) {
            const int c = e / kb, r = e % kb;
            if (r >= c) S[(K + r) + (K + c) * lds] = D[c][r];
        }
        return;
    }
    // block column: rows R0 .. R0+PR-1 below the diagonal block
    const int64_t R0 = K + kb + (int64_t)(blockIdx.x - 1) * PR;
    const int nr = (int)min((int64_t)PR, k - R0);
    if (nr <= 0) return;
    for (int e = tid; e < nr * kb; e += blockDim.x) {
        const int c = e / nr, r = e % nr;
        X[r][c] = S[(R0 + r) + (K + c) * lds];
    }
    __syncthreads();
    // X L^T = B, one thread per row, forward over the columns
    for (int r = tid; r < nr; r += blockDim.x) {
        for (int c = 0; c < kb; ++c) {
            T s = X[r][c];
            for (int l = 0; l < c; ++l) s -= X[r][l] * D[l][c];
            X[r][c] = s / D[c][c];
        }
    }
    __syncthreads();
    for (int e = tid; e < nr * kb; e += blockDim.x) {
        const int c = e / nr, r = e % nr;
        S[(R0 + r) + (K + c) * lds] = X[r][c];
    }
}

// Trailing update on the lower tiles: C(i, j) -= sum_l P(i, l) P(j, l) with
// P = S(:, K : K+kb).  BM x BM output tile per CTA, 256 threads, TM x TM
// outputs per thread, P staged through shared memory in BK-wide slices.
template <typename T, int BM, int BK>
__global__ void __launch_bounds__(256)
    chol_update_kernel(T *__restrict__ S, int64_t k, int64_t lds, int64_t K, int kb) {
    constexpr int TM = BM / 16;  // 16 x 16 threads
    __shared__ T Pa[BK][BM + 4];
    __shared__ T Pb[BK][BM + 4];
    const int64_t T0 = K + kb;  // first trailing row/column
    int64_t I, J;
    tri_tile(blockIdx.x, I, J);
    const int64_t r0 = T0 + I * BM, c0 = T0 + J * BM;
    if (r0 >= k) return;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    T acc[TM][TM];
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TM; ++b) acc[a][b] = T(0);
    for (int l0 = 0; l0 < kb; l0 += BK) {
        for (int e = threadIdx.x; e < BK * BM; e += 256) {
            const int l = e / BM, i = e % BM;
            const int64_t gr = r0 + i, gc = c0 + i;
            const bool okl = l0 + l < kb;
            Pa[l][i] = (okl && gr < k) ? S[gr + (K + l0 + l) * lds] : T(0);
            Pb[l][i] = (okl && gc < k) ? S[gc + (K + l0 + l) * lds] : T(0);
        }
        __syncthreads();
#pragma unroll 4
        for (int l = 0; l < BK; ++l) {
            T av[TM], bv[TM];
#pragma unroll
            for (int a = 0; a < TM; ++a) av[a] = Pa[l][ty + 16 * a];
#pragma unroll
            for (int b = 0; b < TM; ++b) bv[b] = Pb[l][tx + 16 * b];
#pragma unroll
            for (int a = 0; a < TM; ++a)
#pragma unroll
                for (int b = 0; b < TM; ++b) acc[a][b] += av[a] * bv[b];
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < TM; ++a) {
        const int64_t gr = r0 + ty + 16 * a;
#pragma unroll
        for (int b = 0; b < TM; ++b) {
            const int64_t gc = c0 + tx + 16 * b;
            if (gr < k && gc < k && gr >= gc) S[gr + gc * lds] -= acc[a][b];
        }
    }
}

template <typename T>
struct CholCfg;
template <>
struct CholCfg<float> {
    static constexpr int NB = 64, PR = 128, BM = 64, BK = 16;
};
template <>
struct CholCfg<double> {
    static constexpr int NB = 32, PR = 128, BM = 64, BK = 8;
};

template <typename T>
cudaError_t launch_cholesky(cudaStream_t s, T *S, int64_t k, int64_t lds, DevStatus *st) {
    using C = CholCfg<T>;
    const size_t smem = sizeof(T) * (size_t)(C::NB + C::PR) * (C::NB + 1);
    auto panel = chol_panel_kernel<T, C::NB, C::PR>;
    cudaError_t e = cudaFuncSetAttribute(panel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    for (int64_t K = 0; K < k; K += C::NB) {
        const int kb = (int)std::min<int64_t>(C::NB, k - K);
        const int64_t below = k - K - kb;
        const int grid = 1 + (int)cdiv(below, C::PR);
        panel<<<grid, 256, smem, s>>>(S, k, lds, K, st);
        note_launches(1);
        if (below > 0) {
            const int64_t t = cdiv(below, C::BM);
            chol_update_kernel<T, C::BM, C::BK><<<(unsigned)(t * (t + 1) / 2), 256, 0, s>>>(
                S, k, lds, K, kb);
            note_launches(1);
        }
    }
    return cudaGetLastError();
}

template cudaError_t launch_cholesky<float>(cudaStream_t, float *, int64_t, int64_t,
                                            DevStatus *);
template cudaError_t launch_cholesky<double>(cudaStream_t, double *, int64_t, int64_t,
                                             DevStatus *);

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

// ---------------------------------------------------------------------------
// Triangular solves L z = r, then L^T w = z, in place on rhs.
//
// One CTA per 64-row block.  CTAs take their block number from a ticket
// counter in launch order, so a CTA only ever waits on blocks whose CTAs are
// already running (no deadlock whatever else occupies the GPU).  A block
// accumulates the off-diagonal products of every finished block in a fixed
// order, then one warp solves its 64 x 64 diagonal block by substitution,
// the unknowns broadcast lane to lane with shuffles, and publishes the result
// with a release flag.  Every wait is bounded: on timeout the CTA raises the
// launch's abort flag and st->timeout, and all CTAs return.

constexpr int kTB = 64;  // rows per block of the triangular solves

__device__ __forceinline__ int flag_load(const int32_t *p) {
    cuda::atomic_ref<const int32_t, cuda::thread_scope_device> a(*p);
    return a.load(cuda::memory_order_acquire);
}
__device__ __forceinline__ void flag_store(int32_t *p, int v) {
    cuda::atomic_ref<int32_t, cuda::thread_scope_device> a(*p);
    a.store(v, cuda::memory_order_release);
}

// Thread 0 waits for flags[j]; returns false (for the whole CTA) on abort.
__device__ __forceinline__ bool wait_block(const int32_t *flags, int32_t *abort_flag, int j,
                                           DevStatus *st, int *sh_ok) {
    if (threadIdx.x == 0) {
        int ok = 1;
        int spins = 0;
        while (flag_load(flags + j) == 0) {
            if (flag_load(abort_flag) != 0) { ok = 0; break; }
            if (++spins > kSpinLimit) {
                flag_store(abort_flag, 1);
                st->timeout = 1;
                ok = 0;
                break;
            }
            __nanosleep(64);
        }
        *sh_ok = ok;
    }
    __syncthreads();
    return *sh_ok != 0;
}

template <typename T>
__device__ __forceinline__ T ld_cg(const T *p) { return __ldcg(p); }

template <typename T>
__global__ void __launch_bounds__(256)
    trsv_lower_kernel(const T *__restrict__ L, int64_t k, int64_t lds, T *rhs, int32_t *flags,
                      int32_t *ticket, int32_t *abort_flag, DevStatus *st) {
    __shared__ T Dg[kTB][kTB + 1];  // diagonal block, Dg[col][row]
    __shared__ T zs[kTB];
    __shared__ T red[4][kTB];
    __shared__ int blk_sh, ok_sh;
    const int tid = threadIdx.x;
    if (tid == 0) blk_sh = atomicAdd(ticket, 1);
    __syncthreads();
    const int i = blk_sh;
    const int64_t row0 = (int64_t)i * kTB;
    const int nr = (int)min((int64_t)kTB, k - row0);
    for (int e = tid; e < kTB * kTB; e += 256) {
        const int c = e / kTB, r = e % kTB;
        Dg[c][r] = (r < nr && c < nr && r >= c) ? L[(row0 + r) + (row0 + c) * lds] : T(0);
    }
    const int row = tid & 63, cq = tid >> 6;
    T part = T(0);
    for (int j = 0; j < i; ++j) {
        if (!wait_block(flags, abort_flag, j, st, &ok_sh)) return;
        if (tid < kTB) zs[tid] = ld_cg(rhs + (int64_t)j * kTB + tid);
        __syncthreads();
        if (row < nr) {
            const T *Lp = L + (row0 + row) + ((int64_t)j * kTB + cq * 16) * lds;
#pragma unroll
            for (int c = 0; c < 16; ++c) part += Lp[c * lds] * zs[cq * 16 + c];
        }
        __syncthreads();
    }
    red[cq][row] = part;
    __syncthreads();
    if (tid < 32) {
        const int lane = tid;
        T v0 = T(0), v1 = T(0);
        if (lane < nr) v0 = rhs[row0 + lane] - (((red[0][lane] + red[1][lane]) + red[2][lane]) + red[3][lane]);
        if (lane + 32 < nr)
            v1 = rhs[row0 + lane + 32] -
                 (((red[0][lane + 32] + red[1][lane + 32]) + red[2][lane + 32]) + red[3][lane + 32]);
        for (int c = 0; c < nr; ++c) {
            const T src = c < 32 ? v0 : v1;
            const T zc = __shfl_sync(0xffffffffu, src, c & 31) / Dg[c][c];
            if (lane == (c & 31)) {
                if (c < 32) v0 = zc; else v1 = zc;
            }
            if (lane > c && lane < nr) v0 -= Dg[c][lane] * zc;
            if (lane + 32 > c && lane + 32 < nr) v1 -= Dg[c][lane + 32] * zc;
        }
        if (lane < nr) rhs[row0 + lane] = v0;
        if (lane + 32 < nr) rhs[row0 + lane + 32] = v1;
        __threadfence();
    }
    __syncthreads();
    if (tid == 0) flag_store(flags + i, 1);
}

template <typename T>
__global__ void __launch_bounds__(256)
    trsv_upper_kernel(const T *__restrict__ L, int64_t k, int64_t lds, T *rhs, int32_t *flags,
                      int32_t *ticket, int32_t *abort_flag, int nblk, DevStatus *st) {
    __shared__ T Dg[kTB][kTB + 1];   // diagonal block, Dg[col][row] of L
    __shared__ T Tt[kTB][kTB + 1];   // off-diagonal tile, Tt[row_of_w][c]
    __shared__ T ws[kTB];
    __shared__ T red[4][kTB];
    __shared__ int blk_sh, ok_sh;
    const int tid = threadIdx.x;
    if (tid == 0) blk_sh = nblk - 1 - atomicAdd(ticket, 1);
    __syncthreads();
    const int i = blk_sh;
    const int64_t row0 = (int64_t)i * kTB;
    const int nr = (int)min((int64_t)kTB, k - row0);
    for (int e = tid; e < kTB * kTB; e += 256) {
        const int c = e / kTB, r = e % kTB;
        Dg[c][r] = (r < nr && c < nr && r >= c) ? L[(row0 + r) + (row0 + c) * lds] : T(0);
    }
    const int row = tid & 63, cq = tid >> 6;
    T part = T(0);
    for (int j = nblk - 1; j > i; --j) {
        if (!wait_block(flags, abort_flag, j, st, &ok_sh)) return;
        const int64_t jr0 = (int64_t)j * kTB;
        const int njr = (int)min((int64_t)kTB, k - jr0);
        if (tid < kTB) ws[tid] = tid < njr ? ld_cg(rhs + jr0 + tid) : T(0);
        // (L^T)(row0 + r, jr0 + c) = L(jr0 + c, row0 + r); read coalesced along c
        for (int e = tid; e < kTB * kTB; e += 256) {
            const int r = e / kTB, c = e % kTB;
            Tt[r][c] = (c < njr && r < nr) ? L[(jr0 + c) + (row0 + r) * lds] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < 16; ++c) part += Tt[row][cq * 16 + c] * ws[cq * 16 + c];
        __syncthreads();
    }
    red[cq][row] = part;
    __syncthreads();
    if (tid < 32) {
        const int lane = tid;
        T v0 = T(0), v1 = T(0);
        if (lane < nr) v0 = rhs[row0 + lane] - (((red[0][lane] + red[1][lane]) + red[2][lane]) + red[3][lane]);
        if (lane + 32 < nr)
            v1 = rhs[row0 + lane + 32] -
                 (((red[0][lane + 32] + red[1][lane + 32]) + red[2][lane + 32]) + red[3][lane + 32]);
        for (int c = nr - 1; c >= 0; --c) {
            const T src = c < 32 ? v0 : v1;
            const T wc = __shfl_sync(0xffffffffu, src, c & 31) / Dg[c][c];
            if (lane == (c & 31)) {
                if (c < 32) v0 = wc; else v1 = wc;
            }
            // (L_ii^T)(r, c) = L_ii(c, r) for r < c
            if (lane < c) v0 -= Dg[lane][c] * wc;
            if (lane + 32 < c) v1 -= Dg[lane + 32][c] * wc;
        }
        if (lane < nr) rhs[row0 + lane] = v0;
        if (lane + 32 < nr) rhs[row0 + lane + 32] = v1;
        __threadfence();
    }
    __syncthreads();
    if (tid == 0) flag_store(flags + i, 1);
}

template <typename T>
cudaError_t launch_chol_solve(cudaStream_t s, const T *L, int64_t k, int64_t lds, T *rhs,
                              int32_t *flags, DevStatus *st) {
    if (k <= 0) return cudaSuccess;
    const int nblk = (int)cdiv(k, kTB);
    // flags[0..nblk) block done, flags[nblk] ticket, flags[nblk+1] abort
    const size_t bytes = sizeof(int32_t) * (size_t)(nblk + 2);
    cudaError_t e = cudaMemsetAsync(flags, 0, bytes, s);
    if (e != cudaSuccess) return e;
    trsv_lower_kernel<T><<<nblk, 256, 0, s>>>(L, k, lds, rhs, flags, flags + nblk, flags + nblk + 1,
                                              st);
    note_launches(1);
    e = cudaMemsetAsync(flags, 0, bytes, s);
    if (e != cudaSuccess) return e;
    trsv_upper_kernel<T><<<nblk, 256, 0, s>>>(L, k, lds, rhs, flags, flags + nblk,
                                              flags + nblk + 1, nblk, st);
    note_launches(1);
    return cudaGetLastError();
}

template cudaError_t launch_chol_solve<float>(cudaStream_t, const float *, int64_t, int64_t,
                                              float *, int32_t *, DevStatus *);
template cudaError_t launch_chol_solve<double>(cudaStream_t, const double *, int64_t, int64_t,
                                               double *, int32_t *, DevStatus *);

}  // namespace tsnnls
