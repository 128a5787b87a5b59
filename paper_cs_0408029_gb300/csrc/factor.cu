// Blocked Cholesky factorisation of the gathered normal-equations block
// (Section 2, "normal equations solver") and the two triangular solves
// through it (Eq. 4: x_F = L^-T L^-1 c_F).
//
// Right-looking, panel width NB (128 in FP32, 64 in FP64).  Step K:
//   diag    one CTA factors the NB x NB diagonal block in shared memory and
//           builds its inverse in the same column sweep (all 256 threads,
//           one barrier per column).  L_KK goes to the lower triangle, W_K =
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

// ---- warp-level 32 x 32 factor + inverse -------------------------------------
// Lane i holds row i of the block (a[32]); step J, fully unrolled through
// template recursion so that every register index is a compile-time
// constant:  L(J, J) = sqrt(a_J[J]), L(i, J) = a_i[J] / L(J, J), and
// a_i[l] -= L(i, J) L(l, J) for J < l <= i.  The same shuffles of column J
// drive the inverse, lane c holding column c of W = L^-1:
//   W(J, c) = (delta_Jc - acc_c[J]) / L(J, J),  acc_c[l] += L(l, J) W(J, c)  (l > J).
template <typename T>
struct WarpChol {
    T a[32], acc[32], w[32];
};

__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }

template <typename T, int J>
__device__ __forceinline__ void warp_chol_step(WarpChol<T> &s, int lane, int &bad, int base) {
    T d = __shfl_sync(0xffffffffu, s.a[J], J);
    if (!(d > T(0))) {
        if (!bad) bad = base + J + 1;
        d = T(1);
    }
    const T inv = rsqrt_t(d);
    const T lij = (lane > J) ? s.a[J] * inv : (lane == J ? d * inv : s.a[J]);
    s.a[J] = lij;
    const T wj = (J >= lane) ? (((J == lane) ? T(1) : T(0)) - s.acc[J]) * inv : T(0);
    s.w[J] = wj;
#pragma unroll
    for (int l = J + 1; l < 32; ++l) {
        const T llj = __shfl_sync(0xffffffffu, lij, l);
        if (lane >= l) s.a[l] -= lij * llj;
        s.acc[l] += llj * wj;
    }
    if constexpr (J + 1 < 32) warp_chol_step<T, J + 1>(s, lane, bad, base);
}

// Factor A(j0.., j0..) (32 x 32, lower) in place and write its inverse to W.
template <typename T, int NB>
__device__ __forceinline__ void warp_chol_inv(T (*A)[NB + 4], T (*W)[NB + 4], int j0, int lane,
                                              int &bad) {
    WarpChol<T> s;
#pragma unroll
    for (int c = 0; c < 32; ++c) {
        s.a[c] = c <= lane ? A[j0 + c][j0 + lane] : T(0);
        s.acc[c] = T(0);
    }
    warp_chol_step<T, 0>(s, lane, bad, j0);
#pragma unroll
    for (int c = 0; c < 32; ++c) {
        if (c <= lane) A[j0 + c][j0 + lane] = s.a[c];
        W[j0 + lane][j0 + c] = s.w[c];  // column `lane` of W, rows c (0 above the diagonal)
    }
}

// ---- CTA-level small products on shared-memory blocks -------------------------
// out(r, c) = sum_{t < K} X(r, t) Y(t, c) for r < M, c < N (multiples of 4),
// 4 x 4 register tiles, at most 256 tiles (one per thread); tri: only the
// lower tiles (r block >= c block) of a square output.  All reads happen
// before the barrier, all writes (fo) after it, so the output may overwrite
// a source.
template <typename T, typename FX, typename FY, typename FO>
__device__ __forceinline__ void cta_prod(int M, int N, int K, bool tri, FX fx, FY fy, FO fo) {
    const int tid = threadIdx.x;
    const int nt_r = M / 4, nt_c = N / 4;
    const int ntiles = tri ? nt_r * (nt_r + 1) / 2 : nt_r * nt_c;
    // waves of 256 tiles; an output that overwrites a source must fit in one
    for (int base = 0; base < ntiles; base += 256) {
        const int tile = base + tid;
        const bool active = tile < ntiles;
        T acc[4][4] = {};
        int tr = 0, tc = 0;
        if (active) {
            if (tri) {
                int i = (int)((sqrtf(8.f * tile + 1.f) - 1.f) * 0.5f);
                while (i * (i + 1) / 2 > tile) --i;
                while ((i + 1) * (i + 2) / 2 <= tile) ++i;
                tr = i;
                tc = tile - i * (i + 1) / 2;
            } else {
                tr = tile % nt_r;
                tc = tile / nt_r;
            }
            for (int t = 0; t < K; ++t) {
                T x[4], y[4];
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    x[p] = fx(tr * 4 + p, t);
                    y[p] = fy(t, tc * 4 + p);
                }
#pragma unroll
                for (int p = 0; p < 4; ++p)
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[p][q] += x[p] * y[q];
            }
        }
        __syncthreads();
        if (active) {
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) fo(tr * 4 + p, tc * 4 + q, acc[p][q]);
        }
        __syncthreads();
    }
}

template <typename T, int NB>
__global__ void __launch_bounds__(256)
    chol_diag_kernel(T *__restrict__ S, int64_t k, int64_t lds, int64_t K, DevStatus *st) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T(*A)[NB + 4] = reinterpret_cast<T(*)[NB + 4]>(smem_raw);                              // A[col][row]
    T(*W)[NB + 4] = reinterpret_cast<T(*)[NB + 4]>(smem_raw + sizeof(T) * NB * (NB + 4));  // W[col][row]
    __shared__ int bad_sh;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int kb = (int)min((int64_t)NB, k - K);
    if (tid == 0) bad_sh = 0;
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
    constexpr int NBB = NB / 32;
    for (int jb = 0; jb < NBB; ++jb) {
        const int j0 = jb * 32;
        if (warp == 0) {
            int bad = 0;
            warp_chol_inv<T, NB>(A, W, j0, lane, bad);
            if (lane == 0 && bad && !bad_sh) bad_sh = bad;
        }
        __syncthreads();
        const int R = NB - j0 - 32;
        if (R > 0) {
            // rows below: X = B W_jj^T, in place over B
            cta_prod<T>(R, 32, 32, false,
                        [&](int r, int t) { return A[j0 + t][j0 + 32 + r]; },
                        [&](int t, int c) { return W[j0 + t][j0 + c]; },  // W_jj(c, t)
                        [&](int r, int c, T v) { A[j0 + c][j0 + 32 + r] = v; });
            // trailing update: A(r, c) -= sum_t X(r, t) X(c, t) on the lower part
            cta_prod<T>(R, R, 32, true,
                        [&](int r, int t) { return A[j0 + t][j0 + 32 + r]; },
                        [&](int t, int c) { return A[j0 + t][j0 + 32 + c]; },
                        [&](int r, int c, T v) {
                            if (r >= c) A[j0 + 32 + c][j0 + 32 + r] -= v;
                        });
        }
    }
    // off-diagonal blocks of W = L^-1, level by level: for sibling blocks a
    // (at a0) and b (at b0 = a0 + sz) of size sz,  W_ba = -W_bb L_ba W_aa.
    // T1 = L_ba W_aa is kept in the free upper block (rows a, columns b) of W.
    for (int sz = 32; sz < NB; sz *= 2) {
        for (int a0 = 0; a0 < NB; a0 += 2 * sz) {
            const int b0 = a0 + sz;
            cta_prod<T>(sz, sz, sz, false,
                        [&](int r, int t) { return A[a0 + t][b0 + r]; },   // L_ba(r, t)
                        [&](int t, int c) { return W[a0 + c][a0 + t]; },   // W_aa(t, c)
                        [&](int r, int c, T v) { W[b0 + r][a0 + c] = v; });  // T1(r, c) at (a0 + c, b0 + r)
            cta_prod<T>(sz, sz, sz, false,
                        [&](int r, int t) { return W[b0 + t][b0 + r]; },   // W_bb(r, t)
                        [&](int t, int c) { return W[b0 + t][a0 + c]; },   // T1(t, c)
                        [&](int r, int c, T v) { W[a0 + c][b0 + r] = -v; });  // W_ba(r, c)
            // the scratch sits in the upper triangle of the next level's W_aa / W_bb
            for (int e = tid; e < sz * sz; e += 256) W[b0 + e % sz][a0 + e / sz] = T(0);
            __syncthreads();
        }
    }
    if (tid == 0 && bad_sh && bad_sh <= kb && st->chol_info == 0) st->chol_info = (int32_t)(K + bad_sh);
    // write back: L in the lower triangle, W^T in the strict upper triangle
    for (int e = tid; e < NB * NB; e += 256) {
        const int c = e / NB, r = e % NB;
        if (r < kb && c < kb) S[(K + r) + (K + c) * lds] = r >= c ? A[c][r] : W[r][c];  // W(c, r) for r < c
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
    constexpr int LB = 16;  // loads in flight per thread
    for (int e0 = 0; e0 < NB * NB; e0 += 256 * LB) {
        T v[LB];
#pragma unroll
        for (int u = 0; u < LB; ++u) {
            const int e = e0 + u * 256 + tid;
            const int c = e / NB, l = e % NB;
            // W(c, l) for l < c is stored transposed; W(c, c) = 1 / L(c, c)
            v[u] = (c < kb && l <= c) ? S[(K + l) + (K + c) * lds] : T(0);
        }
#pragma unroll
        for (int u = 0; u < LB; ++u) {
            const int e = e0 + u * 256 + tid;
            const int c = e / NB, l = e % NB;
            Wl[l][c] = (l == c && c < kb) ? T(1) / v[u] : v[u];
        }
    }
    for (int e0 = 0; e0 < NB * 64; e0 += 256 * LB) {
        T v[LB];
#pragma unroll
        for (int u = 0; u < LB; ++u) {
            const int e = e0 + u * 256 + tid;
            const int l = e / 64, r = e % 64;
            v[u] = (r < nr && l < kb) ? S[(R0 + r) + (K + l) * lds] : T(0);
        }
#pragma unroll
        for (int u = 0; u < LB; ++u) {
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
        if constexpr (sizeof(T) == 4) {  // 16-byte shared loads (rows are 16-byte aligned)
            const float4 xv = *reinterpret_cast<const float4 *>(&B[l][tr * 4]);
            x[0] = xv.x; x[1] = xv.y; x[2] = xv.z; x[3] = xv.w;
#pragma unroll
            for (int q = 0; q < CT; q += 4) {
                const float4 wv = *reinterpret_cast<const float4 *>(&Wl[l][tc * CT + q]);
                w[q] = wv.x; w[q + 1] = wv.y; w[q + 2] = wv.z; w[q + 3] = wv.w;
            }
        } else {
#pragma unroll
            for (int p = 0; p < 4; ++p) x[p] = B[l][tr * 4 + p];
#pragma unroll
            for (int q = 0; q < CT; ++q) w[q] = Wl[l][tc * CT + q];
        }
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
                            const TcPanel *tc, KernelTimer *kt) {
    constexpr int NB = FactorCfg<T>::NB;
    const size_t smem_diag = 2 * sizeof(T) * NB * (NB + 4);
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
        // algorithmic work of each kernel (for the optional per-kernel timing)
        const double kbd = kb, bel = (double)below;
        if (kt) kt->begin(TSNNLS_PHASE_FACTOR_DIAG);
        chol_diag_kernel<T, NB><<<1, 256, smem_diag, s>>>(S, k, lds, K, st);
        note_launches(1);
        if (kt) kt->end(2.0 * sizeof(T) * kbd * kbd, 2.0 * kbd * kbd * kbd / 3.0);
        if (below > 0) {
            const bool use_tc = NB == 128 && sizeof(T) == 4 && tc && tc->ok && tc->rows >= k;
            if (kt) kt->begin(TSNNLS_PHASE_FACTOR_PANEL);
            chol_panel_kernel<T, NB><<<(unsigned)cdiv(below, 64), 256, smem_panel, s>>>(
                S, k, lds, K, use_tc ? tc->xhi : nullptr, use_tc ? tc->xlo : nullptr);
            note_launches(1);
            // read B and W, write X (and its hi / lo copies)
            if (kt) kt->end(sizeof(T) * (2.0 * bel * kbd + kbd * kbd) + (use_tc ? 8.0 * bel * kbd : 0.0),
                            bel * kbd * kbd);
            if (kt) kt->begin(TSNNLS_PHASE_FACTOR_UPDATE);
            if (use_tc) {
                e = launch_tc_update(s, tc->map_hi, tc->map_lo, reinterpret_cast<float *>(S), k, lds,
                                     K + kb, st);
                if (e != cudaSuccess) return e;
            } else {
                const int64_t t = cdiv(below, 128);
                chol_update128_kernel<T><<<(unsigned)(t * (t + 1) / 2), 256, 0, s>>>(S, k, lds, K, kb);
                note_launches(1);
            }
            // read and write the lower trailing matrix once, read the panel
            // (both copies for the tensor-core split); 2 kb flops per element
            if (kt) kt->end(2.0 * sizeof(T) * bel * (bel + 1.0) / 2.0 + (use_tc ? 8.0 : sizeof(T)) * bel * kbd,
                            bel * (bel + 1.0) * kbd);
        }
    }
    return cudaGetLastError();
}

template cudaError_t launch_cholesky<float>(cudaStream_t, float *, int64_t, int64_t, DevStatus *,
                                            const TcPanel *, KernelTimer *);
template cudaError_t launch_cholesky<double>(cudaStream_t, double *, int64_t, int64_t, DevStatus *,
                                             const TcPanel *, KernelTimer *);

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
