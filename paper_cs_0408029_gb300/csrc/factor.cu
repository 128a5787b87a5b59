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
    // load the lower triangle; pad beyond kb with the identity; W starts at 0
    // (eight loads in flight per thread before any shared-memory store)
    for (int e0 = 0; e0 < NB * NB; e0 += 256 * 8) {
        T v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = e0 + u * 256 + tid;
            const int c = e / NB, r = e % NB;
            v[u] = (r >= c && r < kb && c < kb) ? S[(K + r) + (K + c) * lds] : T(0);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = e0 + u * 256 + tid;
            const int c = e / NB, r = e % NB;
            A[c][r] = (r == c && r >= kb) ? T(1) : v[u];
            W[c][r] = T(0);
        }
    }
    __syncthreads();
    for (int jb = 0; jb < NB; jb += 32) {
        if (warp == 0) {
            // factor the 32 x 32 diagonal sub-block in registers (lane = row)
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
            __syncwarp();
            // its inverse, lane = column: forward substitution on the unit vector
            T y[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                T s = (i == lane) ? T(1) : T(0);
#pragma unroll
                for (int l = 0; l < i; ++l) s -= A[jb + l][jb + i] * y[l];
                y[i] = s / A[jb + i][jb + i];
            }
#pragma unroll
            for (int i = 0; i < 32; ++i) W[jb + lane][jb + i] = (i >= lane) ? y[i] : T(0);
        }
        __syncthreads();
        const int rem = NB - jb - 32;
        if (rem == 0) break;
        // rows below: X = B W_jj^T, one thread per row, independent columns
        for (int r = jb + 32 + tid; r < NB; r += 256) {
            T bq[32];
#pragma unroll
            for (int l = 0; l < 32; ++l) bq[l] = A[jb + l][r];
#pragma unroll
            for (int c = 0; c < 32; ++c) {
                T s = T(0);
#pragma unroll
                for (int l = 0; l <= c; ++l) s += bq[l] * W[jb + l][jb + c];
                A[jb + c][r] = s;
            }
        }
        __syncthreads();
        // trailing update, 4 x 4 register tiles on the lower triangle
        const int tq = rem / 4;
        const int ntile = tq * (tq + 1) / 2;
        for (int tb = tid; tb < ntile; tb += 256) {
            int ti = (int)((sqrtf(8.f * tb + 1.f) - 1.f) * 0.5f);
            while (ti * (ti + 1) / 2 > tb) --ti;
            while ((ti + 1) * (ti + 2) / 2 <= tb) ++ti;
            const int tl = tb - ti * (ti + 1) / 2;
            const int i0 = jb + 32 + ti * 4, l0 = jb + 32 + tl * 4;
            T acc[4][4] = {};
#pragma unroll 4
            for (int c = 0; c < 32; ++c) {
                T x[4], z[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    x[q] = A[jb + c][i0 + q];
                    z[q] = A[jb + c][l0 + q];
                }
#pragma unroll
                for (int p = 0; p < 4; ++p)
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[p][q] += x[p] * z[q];
            }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (i0 + p >= l0 + q) A[l0 + q][i0 + p] -= acc[p][q];
        }
        __syncthreads();
    }
    // off-diagonal blocks of W = L^-1 by distance d:
    //   T_IJ = sum_{m=J}^{I-1} L_Im W_mJ  (kept in the free upper part of W),  W_IJ = -W_II T_IJ
    constexpr int NBB = NB / 32;
    for (int d = 1; d < NBB; ++d) {
        const int npairs = NBB - d;
        for (int w = tid; w < npairs * 64; w += 256) {
            const int pr = w / 64, q = w % 64;
            const int J = pr, I = pr + d;
            const int r0 = (q % 8) * 4, c0 = (q / 8) * 4;
            T acc[4][4] = {};
            for (int l = J * 32; l < I * 32; ++l) {
                T x[4], z[4];
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    x[p] = A[l][I * 32 + r0 + p];
                    z[p] = W[J * 32 + c0 + p][l];
                }
#pragma unroll
                for (int p = 0; p < 4; ++p)
#pragma unroll
                    for (int t = 0; t < 4; ++t) acc[p][t] += x[p] * z[t];
            }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int t = 0; t < 4; ++t) W[I * 32 + r0 + p][J * 32 + c0 + t] = acc[p][t];
        }
        __syncthreads();
        for (int w = tid; w < npairs * 64; w += 256) {
            const int pr = w / 64, q = w % 64;
            const int J = pr, I = pr + d;
            const int r0 = (q % 8) * 4, c0 = (q / 8) * 4;
            T acc[4][4] = {};
            for (int l = 0; l < r0 + 4; ++l) {
                T x[4], z[4];
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    x[p] = W[I * 32 + l][I * 32 + r0 + p];  // W_II(r0 + p, l), 0 above the diagonal
                    z[p] = W[I * 32 + l][J * 32 + c0 + p];  // T_IJ(l, c0 + p)
                }
#pragma unroll
                for (int p = 0; p < 4; ++p)
#pragma unroll
                    for (int t = 0; t < 4; ++t) acc[p][t] += x[p] * z[t];
            }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int t = 0; t < 4; ++t) W[J * 32 + c0 + t][I * 32 + r0 + p] = -acc[p][t];
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
// panel: X = B W^T for the rows below the diagonal block: 64 rows per CTA,
// each thread a 4 x (NB/16) register tile of X

template <typename T, int NB>
__global__ void __launch_bounds__(256)
    chol_panel_kernel(T *__restrict__ S, int64_t k, int64_t lds, int64_t K, float *__restrict__ xhi,
                      float *__restrict__ xlo) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T(*Wl)[NB + 4] = reinterpret_cast<T(*)[NB + 4]>(smem_raw);  // Wl[l][c] = W(c, l)
    T(*B)[68] = reinterpret_cast<T(*)[68]>(smem_raw + sizeof(T) * NB * (NB + 4));  // B[l][row]
    const int tid = threadIdx.x;
    const int kb = (int)min((int64_t)NB, k - K);
    const int64_t R0 = K + kb + (int64_t)blockIdx.x * 64;
    const int nr = (int)min((int64_t)64, k - R0);
    if (nr <= 0) return;
    for (int e0 = 0; e0 < NB * NB; e0 += 256 * 8) {
        T v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = e0 + u * 256 + tid;
            const int c = e / NB, l = e % NB;
            // W(c, l) for l < c is stored transposed; W(c, c) = 1 / L(c, c)
            v[u] = (c < kb && l <= c) ? S[(K + l) + (K + c) * lds] : T(0);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = e0 + u * 256 + tid;
            const int c = e / NB, l = e % NB;
            Wl[l][c] = (l == c && c < kb) ? T(1) / v[u] : v[u];
        }
    }
    for (int e0 = 0; e0 < NB * 64; e0 += 256 * 8) {
        T v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = e0 + u * 256 + tid;
            const int l = e / 64, r = e % 64;
            v[u] = (r < nr && l < kb) ? S[(R0 + r) + (K + l) * lds] : T(0);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = e0 + u * 256 + tid;
            B[e / 64][e % 64] = v[u];
        }
    }
    __syncthreads();
    constexpr int CT = NB / 16;              // columns per thread
    const int tr = tid & 15, tc = tid >> 4;  // rows tr*4 .. +4, columns tc*CT .. +CT
    T acc[4][CT] = {};
#pragma unroll 4
    for (int l = 0; l < NB; ++l) {
        T x[4], w[CT];
#pragma unroll
        for (int p = 0; p < 4; ++p) x[p] = B[l][tr * 4 + p];
#pragma unroll
        for (int q = 0; q < CT; ++q) w[q] = Wl[l][tc * CT + q];
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
            for (int q = 0; q < CT; ++q) acc[p][q] += x[p] * w[q];
    }
#pragma unroll
    for (int q = 0; q < CT; ++q) {
        const int c = tc * CT + q;
        if (c >= kb) continue;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const int r = tr * 4 + p;
            if (r < nr) S[(R0 + r) + (K + c) * lds] = acc[p][q];
        }
    }
    if (xhi) {
        // K-major hi / lo split of X for the tensor-core update: hi keeps the
        // top 10 mantissa bits (exact in TF32), lo = x - hi is exact in FP32
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const int r = tr * 4 + p;
            if (r >= nr) continue;
#pragma unroll
            for (int q = 0; q < CT; ++q) {
                const int c = tc * CT + q;
                const float v = (float)acc[p][q];
                const float hi = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
                xhi[(R0 + r) * 128 + c] = hi;
                xlo[(R0 + r) * 128 + c] = v - hi;
            }
        }
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
    // loads of C first, then the stores (see the tensor-core epilogue)
#pragma unroll
    for (int x = 0; x < 8; ++x) {
        const int64_t gr = r0 + (x < 4 ? ty * 4 + x : 64 + ty * 4 + (x - 4));
        T cv[8];
#pragma unroll
        for (int y = 0; y < 8; ++y) {
            const int64_t gc = c0 + (y < 4 ? tx * 4 + y : 64 + tx * 4 + (y - 4));
            cv[y] = (gr < k && gc < k && gr >= gc) ? S[gr + gc * lds] : T(0);
        }
#pragma unroll
        for (int y = 0; y < 8; ++y) {
            const int64_t gc = c0 + (y < 4 ? tx * 4 + y : 64 + tx * 4 + (y - 4));
            if (gr < k && gc < k && gr >= gc) S[gr + gc * lds] = cv[y] - acc[x][y];
        }
    }
}

template <typename T>
cudaError_t launch_cholesky(cudaStream_t s, T *S, int64_t k, int64_t lds, DevStatus *st,
                            const TcPanel *tc) {
    constexpr int NB = FactorCfg<T>::NB;
    const size_t smem_diag = 2 * sizeof(T) * NB * (NB + 1);
    const size_t smem_panel = sizeof(T) * NB * (NB + 4) + sizeof(T) * NB * 68;
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
            const bool use_tc = NB == 128 && sizeof(T) == 4 && tc && tc->ok && tc->rows >= k;
            chol_panel_kernel<T, NB><<<(unsigned)cdiv(below, 64), 256, smem_panel, s>>>(
                S, k, lds, K, use_tc ? tc->xhi : nullptr, use_tc ? tc->xlo : nullptr);
            note_launches(1);
            if (use_tc) {
                e = launch_tc_update(s, tc->map_hi, tc->map_lo, reinterpret_cast<float *>(S), k, lds,
                                     K + kb, st);
                if (e != cudaSuccess) return e;
            } else {
                const int64_t t = cdiv(below, 128);
                chol_update128_kernel<T><<<(unsigned)(t * (t + 1) / 2), 256, 0, s>>>(S, k, lds, K, kb);
                note_launches(1);
            }
        }
    }
    return cudaGetLastError();
}

template cudaError_t launch_cholesky<float>(cudaStream_t, float *, int64_t, int64_t, DevStatus *,
                                            const TcPanel *);
template cudaError_t launch_cholesky<double>(cudaStream_t, double *, int64_t, int64_t, DevStatus *,
                                             const TcPanel *);

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
    for (int e0 = 0; e0 < NB * NB; e0 += 256 * 8) {  // coalesced reads of the stored W^T
        T v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = e0 + u * 256 + tid;
            const int rr = e / NB, l = e % NB;
            v[u] = (rr < nr && l <= rr) ? L[(row0 + l) + (row0 + rr) * lds] : T(0);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = e0 + u * 256 + tid;
            const int rr = e / NB, l = e % NB;
            Ws[l][rr] = (l == rr && rr < nr) ? T(1) / v[u] : v[u];
        }
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
    for (int e0 = 0; e0 < NB * NB; e0 += 256 * 8) {  // coalesced reads of the stored W^T
        T v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = e0 + u * 256 + tid;
            const int rr = e / NB, l = e % NB;
            v[u] = (rr < nr && l <= rr) ? L[(row0 + l) + (row0 + rr) * lds] : T(0);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = e0 + u * 256 + tid;
            const int rr = e / NB, l = e % NB;
            Ws[l][rr] = (l == rr && rr < nr) ? T(1) / v[u] : v[u];
        }
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
