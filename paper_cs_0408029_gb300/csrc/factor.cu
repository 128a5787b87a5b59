// Blocked Cholesky factorisation of the gathered normal-equations block
// (Section 2, "normal equations solver") and the two triangular solves
// through it (Eq. 4: x_F = L^-T L^-1 c_F).
//
// Right-looking, panel width NB (128 in FP32, 64 in FP64).  Step K:
//   diag    one CTA factors the NB x NB diagonal block in shared memory
//           (32-wide sub-panels: a warp factors each 32 x 32 block in
//           registers, the CTA solves and updates the rest) and inverts the
//           resulting L_KK (warp-level inverses of the 32 x 32 blocks, then
//           the off-diagonal blocks).  L_KK goes to the lower triangle, W_K =
//           L_KK^-1 transposed into the strict upper triangle of the block.
//   panel   X = B W_K^T for every row below the block: a small dense product,
//           fully parallel (no serial substitution down the panel).
//   update  C -= X X^T on the lower tiles of the trailing matrix.
// The solves walk the blocks in order; with W_K at hand a block costs two
// small matrix-vector products instead of an NB-step substitution.
//
// Layout: column-major, leading dimension lds; the upper triangle outside
// the diagonal blocks is never touched.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cuda/atomic>

#include "common.cuh"

namespace tsnnls {

template <typename T>
struct FactorCfg;
template <>
struct FactorCfg<float> {
    static constexpr int NB = 128;
};
template <>
struct FactorCfg<double> {
    static constexpr int NB = 64;
};

__device__ __forceinline__ void tri_tile2(int64_t b, int64_t &I, int64_t &J) {
    int64_t i = (int64_t)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
    while (i * (i + 1) / 2 > b) --i;
    while ((i + 1) * (i + 2) / 2 <= b) ++i;
    I = i;
    J = b - i * (i + 1) / 2;
}

// ---------------------------------------------------------------------------
// diag: factor + invert the NB x NB diagonal block (one CTA of 256 threads)

template <typename T, int NB>
__global__ void __launch_bounds__(256)
    chol_diag_kernel(T *__restrict__ S, int64_t k, int64_t lds, int64_t K, DevStatus *st) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T(*A)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(smem_raw);                              // A[col][row]
    T(*W)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(smem_raw + sizeof(T) * NB * (NB + 1));  // W[col][row]
    __shared__ int bad;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int kb = (int)min((int64_t)NB, k - K);
    if (tid == 0) bad = 0;
    // load the lower triangle; pad beyond kb with the identity
    for (int e = tid; e < NB * NB; e += 256) {
        const int c = e / NB, r = e % NB;
        T v = T(0);
        if (r >= c) {
            if (r < kb && c < kb) v = S[(K + r) + (K + c) * lds];
            else if (r == c) v = T(1);
        }
        A[c][r] = v;
    }
    __syncthreads();
    for (int jb = 0; jb < NB; jb += 32) {
        // a warp factors the 32 x 32 diagonal sub-block; lane = row
        if (warp == 0) {
            T a[32];
#pragma unroll
            for (int c = 0; c < 32; ++c) a[c] = c <= lane ? A[jb + c][jb + lane] : T(0);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                T d = __shfl_sync(0xffffffffu, a[j], j);
                if (!(d > T(0))) {
                    if (lane == 0 && !bad) bad = jb + j + 1;
                    d = T(1);
                }
                const T sd = sqrt(d);
                if (lane == j) a[j] = sd;
                else if (lane > j) a[j] = a[j] / sd;
#pragma unroll
                for (int l = j + 1; l < 32; ++l) {
                    const T llj = __shfl_sync(0xffffffffu, a[j], l);
                    if (lane >= l) a[l] -= a[j] * llj;
                }
            }
#pragma unroll
            for (int c = 0; c < 32; ++c)
                if (c <= lane) A[jb + c][jb + lane] = a[c];
        }
        __syncthreads();
        // rows below the sub-block: X L_jj^T = B, one thread per row
        for (int r = jb + 32 + tid; r < NB; r += 256) {
            T x[32];
#pragma unroll
            for (int c = 0; c < 32; ++c) x[c] = A[jb + c][r];
#pragma unroll
            for (int c = 0; c < 32; ++c) {
                T s = x[c];
#pragma unroll
                for (int l = 0; l < c; ++l) s -= x[l] * A[jb + l][jb + c];
                x[c] = s / A[jb + c][jb + c];
            }
#pragma unroll
            for (int c = 0; c < 32; ++c) A[jb + c][r] = x[c];
        }
        __syncthreads();
        // trailing sub-block update
        const int rem = NB - jb - 32;
        for (int e = tid; e < rem * rem; e += 256) {
            const int i = jb + 32 + e % rem, l = jb + 32 + e / rem;
            if (i >= l) {
                T s = T(0);
#pragma unroll 8
                for (int c = 0; c < 32; ++c) s += A[jb + c][i] * A[jb + c][l];
                A[l][i] -= s;
            }
        }
        __syncthreads();
    }
    // W = L^-1: inverses of the 32 x 32 diagonal blocks, one warp per block,
    // lane = column (forward substitution on the unit vector)
    constexpr int NBB = NB / 32;
    if (warp < NBB) {
        const int b0 = warp * 32;
        T y[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            T s = (i == lane) ? T(1) : T(0);
#pragma unroll
            for (int l = 0; l < i; ++l) s -= A[b0 + l][b0 + i] * y[l];
            y[i] = s / A[b0 + i][b0 + i];
        }
#pragma unroll
        for (int i = 0; i < 32; ++i) W[b0 + lane][b0 + i] = (i >= lane) ? y[i] : T(0);
    }
    __syncthreads();
    // off-diagonal blocks by distance d: W_IJ = -W_II sum_{l=J}^{I-1} L_Il W_lJ
    // (Tmp holds the sums; it reuses the strict upper part of W, unused here)
    for (int d = 1; d < NBB; ++d) {
        const int npairs = NBB - d;
        for (int e = tid; e < npairs * 1024; e += 256) {
            const int pr = e / 1024, q = e % 1024;
            const int J = pr, I = pr + d;
            const int r = q % 32, c = q / 32;
            T s = T(0);
            for (int l = J * 32; l < I * 32; ++l) s += A[l][I * 32 + r] * W[J * 32 + c][l];
            W[I * 32 + r][J * 32 + c] = s;  // transposed slot (upper part of W), free for now
        }
        __syncthreads();
        for (int e = tid; e < npairs * 1024; e += 256) {
            const int pr = e / 1024, q = e % 1024;
            const int J = pr, I = pr + d;
            const int r = q % 32, c = q / 32;
            T s = T(0);
            for (int l = 0; l <= r; ++l) s += W[I * 32 + l][I * 32 + r] * W[I * 32 + l][J * 32 + c];
            // W[col][row]: element (I*32 + r, J*32 + c) lives at W[J*32 + c][I*32 + r]
            W[J * 32 + c][I * 32 + r] = -s;
        }
        __syncthreads();
    }
    if (tid == 0 && bad && st->chol_info == 0) st->chol_info = (int32_t)(K + bad);
    // write back: L in the lower triangle, W^T in the strict upper triangle
    for (int e = tid; e < kb * kb; e += 256) {
        const int c = e / kb, r = e % kb;
        if (r >= c) S[(K + r) + (K + c) * lds] = A[c][r];
        else S[(K + r) + (K + c) * lds] = W[r][c];  // (r, c), r < c  <-  W(c, r)
    }
}

// ---------------------------------------------------------------------------
// panel: X = B W^T for the rows below the diagonal block (64 rows per CTA)

template <typename T, int NB>
__global__ void __launch_bounds__(256)
    chol_panel_kernel(T *__restrict__ S, int64_t k, int64_t lds, int64_t K) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T(*Wt)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(smem_raw);  // Wt[c][l] = W(c, l)
    T(*B)[65] = reinterpret_cast<T(*)[65]>(smem_raw + sizeof(T) * NB * (NB + 1));  // B[l][row]
    const int tid = threadIdx.x;
    const int kb = (int)min((int64_t)NB, k - K);
    const int64_t R0 = K + kb + (int64_t)blockIdx.x * 64;
    const int nr = (int)min((int64_t)64, k - R0);
    if (nr <= 0) return;
    for (int e = tid; e < kb * kb; e += 256) {
        const int c = e / kb, l = e % kb;
        T v = T(0);
        if (l < c) v = S[(K + l) + (K + c) * lds];                  // W(c, l), stored transposed
        else if (l == c) v = T(1) / S[(K + c) + (K + c) * lds];     // W(c, c) = 1 / L(c, c)
        Wt[c][l] = v;
    }
    for (int e = tid; e < kb * 64; e += 256) {
        const int l = e / 64, r = e % 64;
        B[l][r] = r < nr ? S[(R0 + r) + (K + l) * lds] : T(0);
    }
    __syncthreads();
    const int r = tid & 63, cq = tid >> 6;
    for (int c = cq; c < kb; c += 4) {
        T s = T(0);
        for (int l = 0; l <= c; ++l) s += B[l][r] * Wt[c][l];
        if (r < nr) S[(R0 + r) + (K + c) * lds] = s;
    }
}

// ---------------------------------------------------------------------------
// update: C(i, j) -= sum_l X(i, l) X(j, l) on the lower 128 x 128 tiles of the
// trailing matrix; 256 threads with 8 x 8 outputs each, X staged through
// double-buffered shared memory in 8-column slices.

template <typename T>
__global__ void __launch_bounds__(256)
    chol_update128_kernel(T *__restrict__ S, int64_t k, int64_t lds, int64_t K, int kb) {
    constexpr int BM = 128, BK = 8;
    __shared__ __align__(16) T As[2][BK][BM];
    __shared__ __align__(16) T Bs[2][BK][BM];
    const int64_t T0 = K + kb;
    int64_t I, J;
    tri_tile2(blockIdx.x, I, J);
    const int64_t r0 = T0 + I * BM, c0 = T0 + J * BM;
    if (r0 >= k) return;
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    T acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = T(0);
    // loader: thread -> (slice column l, 4 consecutive rows)
    const int ll = tid >> 5, li = (tid & 31) * 4;
    auto load = [&](int buf, int l0) {
        const int l = l0 + ll;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t gr = r0 + li + q, gc = c0 + li + q;
            As[buf][ll][li + q] = (l < kb && gr < k) ? S[gr + (K + l) * lds] : T(0);
            Bs[buf][ll][li + q] = (l < kb && gc < k) ? S[gc + (K + l) * lds] : T(0);
        }
    };
    load(0, 0);
    __syncthreads();
    int buf = 0;
    for (int l0 = 0; l0 < kb; l0 += BK) {
        if (l0 + BK < kb) load(buf ^ 1, l0 + BK);
#pragma unroll
        for (int l = 0; l < BK; ++l) {
            T a[8], b[8];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                a[q] = As[buf][l][ty * 4 + q];
                a[4 + q] = As[buf][l][64 + ty * 4 + q];
                b[q] = Bs[buf][l][tx * 4 + q];
                b[4 + q] = Bs[buf][l][64 + tx * 4 + q];
            }
#pragma unroll
            for (int x = 0; x < 8; ++x)
#pragma unroll
                for (int y = 0; y < 8; ++y) acc[x][y] += a[x] * b[y];
        }
        __syncthreads();
        buf ^= 1;
    }
#pragma unroll
    for (int x = 0; x < 8; ++x) {
        const int64_t gr = r0 + (x < 4 ? ty * 4 + x : 64 + ty * 4 + (x - 4));
#pragma unroll
        for (int y = 0; y < 8; ++y) {
            const int64_t gc = c0 + (y < 4 ? tx * 4 + y : 64 + tx * 4 + (y - 4));
            if (gr < k && gc < k && gr >= gc) S[gr + gc * lds] -= acc[x][y];
        }
    }
}

template <typename T>
cudaError_t launch_cholesky(cudaStream_t s, T *S, int64_t k, int64_t lds, DevStatus *st) {
    constexpr int NB = FactorCfg<T>::NB;
    const size_t smem_diag = 2 * sizeof(T) * NB * (NB + 1);
    const size_t smem_panel = sizeof(T) * NB * (NB + 1) + sizeof(T) * NB * 65;
    cudaError_t e = cudaFuncSetAttribute(chol_diag_kernel<T, NB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_diag);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(chol_panel_kernel<T, NB>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_panel);
    if (e != cudaSuccess) return e;
    for (int64_t K = 0; K < k; K += NB) {
        const int kb = (int)std::min<int64_t>(NB, k - K);
        const int64_t below = k - K - kb;
        chol_diag_kernel<T, NB><<<1, 256, smem_diag, s>>>(S, k, lds, K, st);
        note_launches(1);
        if (below > 0) {
            chol_panel_kernel<T, NB><<<(unsigned)cdiv(below, 64), 256, smem_panel, s>>>(S, k, lds, K);
            note_launches(1);
            const int64_t t = cdiv(below, 128);
            chol_update128_kernel<T><<<(unsigned)(t * (t + 1) / 2), 256, 0, s>>>(S, k, lds, K, kb);
            note_launches(1);
        }
    }
    return cudaGetLastError();
}

template cudaError_t launch_cholesky<float>(cudaStream_t, float *, int64_t, int64_t, DevStatus *);
template cudaError_t launch_cholesky<double>(cudaStream_t, double *, int64_t, int64_t, DevStatus *);

// ---------------------------------------------------------------------------
// Triangular solves: L z = r, then L^T w = z, in place on rhs.
//
// One CTA per NB-row block.  CTAs take their block from a ticket counter in
// launch order, so a CTA only waits on blocks whose CTAs already run.  While
// it waits for block j, a CTA already holds its tile of L for block j in
// registers; when the flag appears it adds that product, and after the last
// block it forms z_i = W_i (r_i - sum) with the stored inverse and publishes
// z_i with a release flag.  Every wait is bounded: on timeout the CTA raises
// the launch's abort flag and st->timeout and all CTAs return.

__device__ __forceinline__ int flag_load(const int32_t *p) {
    cuda::atomic_ref<const int32_t, cuda::thread_scope_device> a(*p);
    return a.load(cuda::memory_order_acquire);
}
__device__ __forceinline__ void flag_store(int32_t *p, int v) {
    cuda::atomic_ref<int32_t, cuda::thread_scope_device> a(*p);
    a.store(v, cuda::memory_order_release);
}

__device__ __forceinline__ bool wait_flag(const int32_t *flags, int32_t *abort_flag, int j,
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
            if (spins > 64) __nanosleep(32);
        }
        *sh_ok = ok;
    }
    __syncthreads();
    return *sh_ok != 0;
}

// Forward: thread (r = tid % NB, part = tid / NB) owns row r and a slice of
// NB / P columns of every tile, P = 256 / NB parts.
template <typename T, int NB>
__global__ void __launch_bounds__(256)
    trsv_fwd_kernel(const T *__restrict__ L, int64_t k, int64_t lds, T *rhs, int32_t *flags,
                    int32_t *ticket, int32_t *abort_flag, DevStatus *st) {
    constexpr int P = 256 / NB, CW = NB / P;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T(*Ws)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(smem_raw);  // Ws[l][r] = W(r, l)
    __shared__ T zs[NB];
    __shared__ T red[P][NB];
    __shared__ int blk_sh, ok_sh;
    const int tid = threadIdx.x;
    if (tid == 0) blk_sh = atomicAdd(ticket, 1);
    __syncthreads();
    const int i = blk_sh;
    const int64_t row0 = (int64_t)i * NB;
    const int nr = (int)min((int64_t)NB, k - row0);
    const int r = tid % NB, part = tid / NB;
    for (int e = tid; e < NB * NB; e += 256) {
        const int rr = e / NB, l = e % NB;  // coalesced reads of the stored W^T (row l of column rr)
        T v = T(0);
        if (rr < nr && l < nr) {
            if (l < rr) v = L[(row0 + l) + (row0 + rr) * lds];
            else if (l == rr) v = T(1) / L[(row0 + rr) + (row0 + rr) * lds];
        }
        Ws[l][rr] = v;
    }
    T acc = T(0);
    T tile[CW];
    if (i > 0 && r < nr) {
#pragma unroll
        for (int c = 0; c < CW; ++c) tile[c] = L[(row0 + r) + (int64_t)(part * CW + c) * lds];
    }
    for (int j = 0; j < i; ++j) {
        if (!wait_flag(flags, abort_flag, j, st, &ok_sh)) return;
        if (tid < NB) zs[tid] = __ldcg(rhs + (int64_t)j * NB + tid);
        __syncthreads();
        if (r < nr) {
#pragma unroll
            for (int c = 0; c < CW; ++c) acc += tile[c] * zs[part * CW + c];
            if (j + 1 < i) {
#pragma unroll
                for (int c = 0; c < CW; ++c)
                    tile[c] = L[(row0 + r) + ((int64_t)(j + 1) * NB + part * CW + c) * lds];
            }
        }
        __syncthreads();
    }
    red[part][r] = acc;
    __syncthreads();
    if (tid < NB) {
        T sum = T(0);
#pragma unroll
        for (int q = 0; q < P; ++q) sum += red[q][tid];
        zs[tid] = tid < nr ? rhs[row0 + tid] - sum : T(0);
    }
    __syncthreads();
    T z = T(0);
#pragma unroll 8
    for (int c = 0; c < CW; ++c) z += Ws[part * CW + c][r] * zs[part * CW + c];
    red[part][r] = z;
    __syncthreads();
    if (tid < nr) {
        T sum = T(0);
#pragma unroll
        for (int q = 0; q < P; ++q) sum += red[q][tid];
        rhs[row0 + tid] = sum;
        __threadfence();
    }
    __syncthreads();
    if (tid == 0) flag_store(flags + i, 1);
}

// Backward: (L^T)(row0 + r, jr0 + c) = L(jr0 + c, row0 + r).  Warp w owns the
// columns r = w, w + 8, ... of L (NB / 8 of them); its lanes run down each
// column (coalesced) and reduce by shuffles.
template <typename T, int NB>
__global__ void __launch_bounds__(256)
    trsv_bwd_kernel(const T *__restrict__ L, int64_t k, int64_t lds, T *rhs, int32_t *flags,
                    int32_t *ticket, int32_t *abort_flag, int nblk, DevStatus *st) {
    constexpr int CPW = NB / 8;   // columns per warp
    constexpr int RPL = NB / 32;  // rows per lane per column
    constexpr int P = 256 / NB, CW = NB / P;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T(*Ws)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(smem_raw);  // Ws[l][r] = W(r, l)
    __shared__ T ws[NB];
    __shared__ T accs[NB];
    __shared__ T red[P][NB];
    __shared__ int blk_sh, ok_sh;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) blk_sh = nblk - 1 - atomicAdd(ticket, 1);
    __syncthreads();
    const int i = blk_sh;
    const int64_t row0 = (int64_t)i * NB;
    const int nr = (int)min((int64_t)NB, k - row0);
    for (int e = tid; e < NB * NB; e += 256) {
        const int rr = e / NB, l = e % NB;
        T v = T(0);
        if (rr < nr && l < nr) {
            if (l < rr) v = L[(row0 + l) + (row0 + rr) * lds];
            else if (l == rr) v = T(1) / L[(row0 + rr) + (row0 + rr) * lds];
        }
        Ws[l][rr] = v;
    }
    T acc[CPW];
#pragma unroll
    for (int q = 0; q < CPW; ++q) acc[q] = T(0);
    T tile[CPW][RPL];
    auto fetch = [&](int j) {
        const int64_t jr0 = (int64_t)j * NB;
        const int njr = (int)min((int64_t)NB, k - jr0);
#pragma unroll
        for (int q = 0; q < CPW; ++q) {
            const int rc = warp + 8 * q;
#pragma unroll
            for (int t = 0; t < RPL; ++t) {
                const int c = lane + 32 * t;
                tile[q][t] = (rc < nr && c < njr) ? L[(jr0 + c) + (row0 + rc) * lds] : T(0);
            }
        }
    };
    if (i + 1 < nblk) fetch(nblk - 1);
    for (int j = nblk - 1; j > i; --j) {
        if (!wait_flag(flags, abort_flag, j, st, &ok_sh)) return;
        const int64_t jr0 = (int64_t)j * NB;
        const int njr = (int)min((int64_t)NB, k - jr0);
        if (tid < NB) ws[tid] = tid < njr ? __ldcg(rhs + jr0 + tid) : T(0);
        __syncthreads();
#pragma unroll
        for (int q = 0; q < CPW; ++q) {
            T s = T(0);
#pragma unroll
            for (int t = 0; t < RPL; ++t) s += tile[q][t] * ws[lane + 32 * t];
            acc[q] += s;
        }
        if (j - 1 > i) fetch(j - 1);
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < CPW; ++q) {
        T s = acc[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) accs[warp + 8 * q] = s;
    }
    __syncthreads();
    if (tid < NB) ws[tid] = tid < nr ? rhs[row0 + tid] - accs[tid] : T(0);
    __syncthreads();
    // w_i = W^T ws: w(r) = sum_{l >= r} W(l, r) ws(l) = sum_l Ws[r][l] ws(l)
    const int r = tid % NB, part = tid / NB;
    T w = T(0);
#pragma unroll 8
    for (int c = 0; c < CW; ++c) w += Ws[r][part * CW + c] * ws[part * CW + c];
    red[part][r] = w;
    __syncthreads();
    if (tid < nr) {
        T sum = T(0);
#pragma unroll
        for (int q = 0; q < P; ++q) sum += red[q][tid];
        rhs[row0 + tid] = sum;
        __threadfence();
    }
    __syncthreads();
    if (tid == 0) flag_store(flags + i, 1);
}

template <typename T>
cudaError_t launch_chol_solve(cudaStream_t s, const T *L, int64_t k, int64_t lds, T *rhs,
                              int32_t *flags, DevStatus *st) {
    constexpr int NB = FactorCfg<T>::NB;
    if (k <= 0) return cudaSuccess;
    const int nblk = (int)cdiv(k, NB);
    // flags[0..nblk) block done, flags[nblk] ticket, flags[nblk+1] abort
    const size_t bytes = sizeof(int32_t) * (size_t)(nblk + 2);
    const size_t smem = sizeof(T) * NB * (NB + 1);
    cudaError_t e = cudaFuncSetAttribute(trsv_fwd_kernel<T, NB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(trsv_bwd_kernel<T, NB>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaMemsetAsync(flags, 0, bytes, s);
    if (e != cudaSuccess) return e;
    trsv_fwd_kernel<T, NB><<<nblk, 256, smem, s>>>(L, k, lds, rhs, flags, flags + nblk, flags + nblk + 1, st);
    note_launches(1);
    e = cudaMemsetAsync(flags, 0, bytes, s);
    if (e != cudaSuccess) return e;
    trsv_bwd_kernel<T, NB><<<nblk, 256, smem, s>>>(L, k, lds, rhs, flags, flags + nblk, flags + nblk + 1,
                                                   nblk, st);
    note_launches(1);
    return cudaGetLastError();
}

template cudaError_t launch_chol_solve<float>(cudaStream_t, const float *, int64_t, int64_t,
                                              float *, int32_t *, DevStatus *);
template cudaError_t launch_chol_solve<double>(cudaStream_t, const double *, int64_t, int64_t,
                                               double *, int32_t *, DevStatus *);

}  // namespace tsnnls
