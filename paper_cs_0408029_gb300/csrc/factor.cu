// Blocked Cholesky factorisation of the gathered normal-equations block
// (Section 2, "normal equations solver") and the two triangular solves
// through it (Eq. 4: x_F = L^-T L^-1 c_F).
//
// Right-looking, panel width NB (128 in FP32, 64 in FP64).  Step K:
//   diag    one CTA factors the NB x NB diagonal block in shared memory and
//           inverts it (dense_block.cuh): per 32-column block, warp 0
//           factors and inverts the 32 x 32 diagonal block, then the CTA
//           forms the rows below and updates the trailing triangle; the
//           inverse's off-diagonal blocks follow level by level.  L_KK goes
//           to the lower triangle, W_K = L_KK^-1 transposed into the strict
//           upper triangle of the block.
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

#include <algorithm>

#include <cuda/atomic>

#include "common.cuh"
#include "dense_block.cuh"

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

// ---- diag: factor + invert the NB x NB diagonal block (one CTA, 256 threads)
// Shared memory: A[col][row] holds the block (then L), W[col][row] = L^-1.
// For each 32-column block jb: warp 0 factors and inverts the 32 x 32
// diagonal block, the CTA forms X = B W_jj^T for the rows below it (in place)
// and subtracts X X^T from the trailing lower triangle.  The off-diagonal
// blocks of W follow level by level: for sibling blocks a, b of size sz,
// W_ba = -W_bb (L_ba W_aa).
template <typename T, int NB>
__global__ void __launch_bounds__(256)
    chol_diag_kernel(T *__restrict__ S, int64_t k, int64_t lds, int64_t K, DevStatus *st) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T(*A)[NB + 4] = reinterpret_cast<T(*)[NB + 4]>(smem_raw);                              // A[col][row]
    T(*W)[NB + 4] = reinterpret_cast<T(*)[NB + 4]>(smem_raw + sizeof(T) * NB * (NB + 4));  // W[col][row]
    __shared__ int bad_sh;
    __shared__ __align__(16) T col[2][32];
    const int tid = threadIdx.x;
    const int kb = (int)min((int64_t)NB, k - K);
    if (tid == 0) bad_sh = 0;
    // load the lower triangle in 4-row vectors (all in flight before any
    // shared-memory store); rows >= kb read zero, the identity pads the
    // diagonal beyond kb; W starts at 0.  Columns hold lds >= K + kb rows
    // rounded up to 32, so a vector that starts below kb stays inside them.
    constexpr int NV = NB * NB / 4 / 256;  // vectors per thread
    {
        T v[NV][4];
#pragma unroll
        for (int u = 0; u < NV; ++u) {
            const int e = (u * 256 + tid) * 4;
            const int c = e / NB, r = e % NB;
            if (c < kb && r < kb && r + 3 >= c) {
                ld4(&S[(K + r) + (K + c) * lds], v[u]);
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) v[u][q] = T(0);
            }
        }
#pragma unroll
        for (int u = 0; u < NV; ++u) {
            const int e = (u * 256 + tid) * 4;
            const int c = e / NB, r = e % NB;
            T o[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int rr = r + q;
                o[q] = (rr == c && rr >= kb) ? T(1) : ((rr >= c && rr < kb) ? v[u][q] : T(0));
            }
            st4(&A[c][r], o);
            const T z[4] = {T(0), T(0), T(0), T(0)};
            st4(&W[c][r], z);
        }
    }
    __syncthreads();
    diag_block_core<T, NB>(A, W, col, &bad_sh);
    if (tid == 0 && bad_sh && bad_sh <= kb && st->chol_info == 0) st->chol_info = (int32_t)(K + bad_sh);
    // write back the block as A now holds it: L in the lower triangle, W^T
    // in the strict upper triangle (W(c, r) for r < c), in 4-row vectors; a
    // vector that crosses kb is written element by element
    for (int e = tid * 4; e < NB * NB; e += 256 * 4) {
        const int c = e / NB, r = e % NB;
        if (c >= kb || r >= kb) continue;
        T o[4];
        ld4(&A[c][r], o);
        T *dst = &S[(K + r) + (K + c) * lds];
        if (r + 3 < kb) {
            st4(dst, o);
        } else {
            for (int q = 0; q < 4 && r + q < kb; ++q) dst[q] = o[q];
        }
    }
}

// ---------------------------------------------------------------------------
// panel: X = B W^T for rows [r_begin, r_end) below the diagonal block (a
// multiple of 4 apart from k): kPanelRows rows per CTA (enough CTAs to cover
// the SMs for the panel heights that occur), each thread a (kPanelRows/16) x
// (NB/16) register tile of X

constexpr int kPanelRows = 32;
constexpr int kHeadPanelRows = 16;  // the look-ahead's head rows, on the critical chain

template <typename T, int NB, int PR = kPanelRows>
__global__ void __launch_bounds__(256)
    chol_panel_kernel(T *__restrict__ S, int64_t k, int64_t lds, int64_t K, int64_t r_begin, int64_t r_end,
                      float *__restrict__ xhi, float *__restrict__ xlo) {
    constexpr int RT = PR / 16, BP = PR + 4;  // rows per thread, B pitch
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T(*Wl)[NB + 4] = reinterpret_cast<T(*)[NB + 4]>(smem_raw);  // Wl[l][c] = W(c, l)
    T(*B)[BP] = reinterpret_cast<T(*)[BP]>(smem_raw + sizeof(T) * NB * (NB + 4));  // B[l][row]
    const int tid = threadIdx.x;
    const int kb = (int)min((int64_t)NB, k - K);
    const int64_t R0 = r_begin + (int64_t)blockIdx.x * PR;  // rows [r_begin, r_end) below the block
    const int nr = (int)min((int64_t)PR, r_end - R0);
    if (nr <= 0) return;
    // W: thread -> column c of the stored block, 8 consecutive rows l (two
    // 4-vectors, one 32-byte sector in FP32); column c holds W(c, l) for l < c
    // and L(c, c) on the diagonal, so Wl[l][c] = W(c, l) with W(c, c) =
    // 1 / L(c, c).  Rows stay below K + kb rounded up to 8 <= lds.
    constexpr int NW = NB * NB / 8 / 256;   // 8-row chunks of W per thread
    constexpr int NBV = NB * PR / 4 / 256;  // 4-row vectors of B per thread
    constexpr int VPC = PR / 4;             // 4-row vectors per column of B
    {
        T v[NW][8];
#pragma unroll
        for (int u = 0; u < NW; ++u) {
            const int e = u * 256 + tid;
            const int c = e % NB, l0 = (e / NB) * 8;
            if (c < kb && l0 <= c) {
                const T *src = &S[(K + l0) + (K + c) * lds];
                T lo4[4], hi4[4];
                ld4(src, lo4);
                ld4(src + 4, hi4);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    v[u][q] = lo4[q];
                    v[u][4 + q] = hi4[q];
                }
            } else {
#pragma unroll
                for (int q = 0; q < 8; ++q) v[u][q] = T(0);
            }
        }
        // B: thread -> column l, 4 consecutive rows (coalesced down the column)
        T bv[NBV][4];
#pragma unroll
        for (int u = 0; u < NBV; ++u) {
            const int e = u * 256 + tid;
            const int l = e / VPC, r0 = (e % VPC) * 4;
            if (l < kb && r0 < nr) {
                ld4(&S[(R0 + r0) + (K + l) * lds], bv[u]);
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) bv[u][q] = T(0);
            }
        }
#pragma unroll
        for (int u = 0; u < NW; ++u) {
            const int e = u * 256 + tid;
            const int c = e % NB, l0 = (e / NB) * 8;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int l = l0 + q;
                if (l != c) Wl[l][c] = (c >= kb || l > c) ? T(0) : v[u][q];
            }
        }
        // the diagonal of W (written by no one else), one reciprocal per thread
        if (tid < NB) Wl[tid][tid] = tid < kb ? T(1) / S[(K + tid) + (K + tid) * lds] : T(0);
#pragma unroll
        for (int u = 0; u < NBV; ++u) {
            const int e = u * 256 + tid;
            const int l = e / VPC, r0 = (e % VPC) * 4;
            T o[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) o[q] = r0 + q < nr ? bv[u][q] : T(0);
            st4(&B[l][r0], o);
        }
    }
    __syncthreads();
    constexpr int CT = NB / 16;              // columns per thread
    const int tr = tid & 15, tc = tid >> 4;  // rows tr*RT .. +RT, columns tc*CT .. +CT
    T acc[RT][CT] = {};
#pragma unroll 4
    for (int l = 0; l < NB; ++l) {
        T x[RT], w[CT];
#pragma unroll
        for (int p = 0; p < RT; ++p) x[p] = B[l][tr * RT + p];
        if constexpr (sizeof(T) == 4) {  // 16-byte shared loads (rows are 16-byte aligned)
#pragma unroll
            for (int q = 0; q < CT; q += 4) {
                const float4 wv = *reinterpret_cast<const float4 *>(&Wl[l][tc * CT + q]);
                w[q] = wv.x; w[q + 1] = wv.y; w[q + 2] = wv.z; w[q + 3] = wv.w;
            }
        } else {
#pragma unroll
            for (int q = 0; q < CT; ++q) w[q] = Wl[l][tc * CT + q];
        }
#pragma unroll
        for (int p = 0; p < RT; ++p)
#pragma unroll
            for (int q = 0; q < CT; ++q) acc[p][q] += x[p] * w[q];
    }
    const int r0 = tr * RT;
#pragma unroll
    for (int q = 0; q < CT; ++q) {
        const int c = tc * CT + q;
        if (c >= kb) continue;
        T *dst = &S[(R0 + r0) + (K + c) * lds];
#pragma unroll
        for (int p = 0; p < RT; ++p)
            if (r0 + p < nr) dst[p] = acc[p][q];
    }
    if (xhi) {
        // K-major hi / lo split of X for the tensor-core update: hi keeps the
        // top 10 mantissa bits (exact in TF32), lo = x - hi is exact in FP32
#pragma unroll
        for (int p = 0; p < RT; ++p) {
            const int r = r0 + p;
            if (r >= nr) continue;
#pragma unroll
            for (int q = 0; q < CT; q += 4) {
                float h4[4], l4[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float v = (float)acc[p][q + u];
                    h4[u] = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
                    l4[u] = v - h4[u];
                }
                st4(&xhi[(R0 + r) * 128 + tc * CT + q], h4);
                st4(&xlo[(R0 + r) * 128 + tc * CT + q], l4);
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
    chol_update128_kernel(T *__restrict__ S, int64_t k, int64_t lds, int64_t K, int kb, int64_t tile0) {
    constexpr int BM = 128, BK = 8;
    __shared__ __align__(16) T As[2][BK][BM];
    __shared__ __align__(16) T Bs[2][BK][BM];
    const int64_t T0 = K + kb;
    int64_t I, J;
    tri_tile2(blockIdx.x + tile0, I, J);  // tiles before tile0 are done elsewhere
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

// ---------------------------------------------------------------------------
// look-ahead: step K's contribution to the first 128 x 128 tile of the
// trailing matrix (which holds the next diagonal block) alone,
//     C(Kn.., Kn..) -= X X^T,  X = S(Kn .. Kn + 128, K .. K + NB)  (lower part),
// so the next diagonal block can be factored while the update kernels, which
// skip that tile, do the rest.  One CTA per lower 32 x 32 sub-block (10),
// 2 x 2 outputs per thread.

template <typename T, int NB>
__global__ void __launch_bounds__(256)
    chol_tile_update_kernel(T *__restrict__ S, int64_t k, int64_t lds, int64_t K, int64_t Kn) {
    __shared__ __align__(16) T Xr[NB][36];  // Xr[t][r] = X(rb + r, t)
    __shared__ __align__(16) T Xc[NB][36];  // Xc[t][c] = X(cb + c, t)
    int64_t I, J;
    tri_tile2(blockIdx.x, I, J);
    const int kb = (int)min((int64_t)128, k - Kn);  // the update kernels' tile size
    const int rb = (int)I * 32, cb = (int)J * 32;
    if (rb >= kb) return;
    const int tid = threadIdx.x;
    constexpr int NL = NB * 32 / 256;  // elements of each operand per thread, all loads in flight
    T vr[NL], vc[NL];
#pragma unroll
    for (int u = 0; u < NL; ++u) {
        const int e = u * 256 + tid;
        const int t = e / 32, r = e % 32;
        vr[u] = rb + r < kb ? S[(Kn + rb + r) + (K + t) * lds] : T(0);
        vc[u] = cb + r < kb ? S[(Kn + cb + r) + (K + t) * lds] : T(0);
    }
#pragma unroll
    for (int u = 0; u < NL; ++u) {
        const int e = u * 256 + tid;
        Xr[e / 32][e % 32] = vr[u];
        Xc[e / 32][e % 32] = vc[u];
    }
    const int rr = (tid % 16) * 2, cc = (tid / 16) * 2;
    // this thread's entries of C, loaded before the products need the barrier
    T cv[2][2];
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int gr = rb + rr + p, gc = cb + cc + q;
            cv[p][q] = (gr < kb && gc < kb && gr >= gc) ? S[(Kn + gr) + (Kn + gc) * lds] : T(0);
        }
    __syncthreads();
    T a00 = T(0), a01 = T(0), a10 = T(0), a11 = T(0);
#pragma unroll 8
    for (int t = 0; t < NB; ++t) {
        T x[2], y[2];
        ld2(&Xr[t][rr], x);  // 2-vector shared loads (even offsets, 8-byte aligned rows)
        ld2(&Xc[t][cc], y);
        a00 += x[0] * y[0];
        a01 += x[0] * y[1];
        a10 += x[1] * y[0];
        a11 += x[1] * y[1];
    }
    const T acc[2][2] = {{a00, a01}, {a10, a11}};
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int gr = rb + rr + p, gc = cb + cc + q;
            if (gr < kb && gc < kb && gr >= gc) S[(Kn + gr) + (Kn + gc) * lds] = cv[p][q] - acc[p][q];
        }
}

template <typename T>
cudaError_t launch_cholesky(cudaStream_t s, T *S, int64_t k, int64_t lds, DevStatus *st,
                            const TcPanel *tc, KernelTimer *kt, const FactorStreams *fs) {
    constexpr int NB = FactorCfg<T>::NB;
    // the kernels move 4-element vectors: columns must start 16-byte aligned
    // and hold whole 32-row groups (reads run up to K + kb rounded up to 8)
    if (k > 0 && (lds % 32 != 0 || (reinterpret_cast<uintptr_t>(S) & 15) != 0)) return cudaErrorInvalidValue;
    const size_t smem_diag = 2 * sizeof(T) * NB * (NB + 4);
    const size_t smem_panel = sizeof(T) * NB * (NB + 4) + sizeof(T) * NB * (kPanelRows + 4);
    cudaError_t e = cudaFuncSetAttribute(chol_diag_kernel<T, NB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_diag);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(chol_panel_kernel<T, NB>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_panel);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(chol_panel_kernel<T, NB, kHeadPanelRows>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_panel);
    if (e != cudaSuccess) return e;
    const bool ahead = fs != nullptr && kt == nullptr;
    const bool use_tc = NB == 128 && sizeof(T) == 4 && tc && tc->ok && tc->rows >= k;
    auto panel = [&](cudaStream_t st_, int64_t K, int64_t r0, int64_t r1) {
        if (r1 > r0)
            chol_panel_kernel<T, NB><<<(unsigned)cdiv(r1 - r0, kPanelRows), 256, smem_panel, st_>>>(
                S, k, lds, K, r0, r1, use_tc ? tc->xhi : nullptr, use_tc ? tc->xlo : nullptr);
        note_launches(r1 > r0 ? 1 : 0);
    };
    auto update = [&](int64_t K, int kb, int64_t tile0) -> cudaError_t {
        if (use_tc)
            return launch_tc_update(s, tc->map_hi, tc->map_lo, reinterpret_cast<float *>(S), k, lds, K + kb,
                                    st, tile0);
        const int64_t t = cdiv(k - K - kb, 128);
        const int64_t tiles = t * (t + 1) / 2 - tile0;
        if (tiles > 0) {
            chol_update128_kernel<T><<<(unsigned)tiles, 256, 0, s>>>(S, k, lds, K, kb, tile0);
            note_launches(1);
        }
        return cudaSuccess;
    };
    if (!ahead) {
        // in order: diagonal block, panel, trailing update (optionally each timed)
        for (int64_t K = 0; K < k; K += NB) {
            const int kb = (int)std::min<int64_t>(NB, k - K);
            const int64_t below = k - K - kb;
            // algorithmic work of each kernel (for the optional per-kernel timing)
            const double kbd = kb, bel = (double)below;
            if (kt) kt->begin(TSNNLS_PHASE_FACTOR_DIAG);
            chol_diag_kernel<T, NB><<<1, 256, smem_diag, s>>>(S, k, lds, K, st);
            note_launches(1);
            // the method's own work: the block's Cholesky, kb^3 / 3 (the inverse
            // built alongside, another kb^3 / 3, is this design's extra work)
            if (kt) kt->end(2.0 * sizeof(T) * kbd * kbd, kbd * kbd * kbd / 3.0);
            if (below == 0) break;
            if (kt) kt->begin(TSNNLS_PHASE_FACTOR_PANEL);
            panel(s, K, K + kb, k);
            // read B and W, write X (and its hi / lo copies)
            if (kt) kt->end(sizeof(T) * (2.0 * bel * kbd + kbd * kbd) + (use_tc ? 8.0 * bel * kbd : 0.0),
                            bel * kbd * kbd);
            if (kt) kt->begin(TSNNLS_PHASE_FACTOR_UPDATE);
            e = update(K, kb, 0);
            if (e != cudaSuccess) return e;
            // read and write the lower trailing matrix once, read the panel
            // (both copies for the tensor-core split); 2 kb flops per element
            if (kt) kt->end(2.0 * sizeof(T) * bel * (bel + 1.0) / 2.0 + (use_tc ? 8.0 : sizeof(T)) * bel * kbd,
                            bel * (bel + 1.0) * kbd);
        }
        return cudaGetLastError();
    }
    // Look-ahead.  Step K, after the main stream has finished step K - 1:
    //   side:  panel rows of the first trailing tile (its 128 rows) -> "head"
    //          event; that tile's share of this step's update; the next
    //          diagonal block -> "join" event
    //   main:  panel of the remaining rows; wait "head"; trailing update
    //          without the first tile; wait "join"
    // so the chain from one diagonal block to the next is a short panel, the
    // tile update and the diagonal kernel, while the long panel and the
    // trailing update run beside it.
    chol_diag_kernel<T, NB><<<1, 256, smem_diag, s>>>(S, k, lds, 0, st);
    note_launches(1);
    for (int64_t K = 0; K + NB < k; K += NB) {
        const int64_t Kn = K + NB, head_end = std::min<int64_t>(Kn + 128, k);
        e = cudaEventRecord(fs->fork, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(fs->side, fs->fork, 0);
        if (e != cudaSuccess) return e;
        // the head rows in 16-row CTAs: twice the CTAs, half the work on the chain each
        chol_panel_kernel<T, NB, kHeadPanelRows>
            <<<(unsigned)cdiv(head_end - Kn, kHeadPanelRows), 256, smem_panel, fs->side>>>(
                S, k, lds, K, Kn, head_end, use_tc ? tc->xhi : nullptr, use_tc ? tc->xlo : nullptr);
        note_launches(1);
        e = cudaEventRecord(fs->head, fs->side);
        if (e != cudaSuccess) return e;
        chol_tile_update_kernel<T, NB><<<10, 256, 0, fs->side>>>(S, k, lds, K, Kn);
        chol_diag_kernel<T, NB><<<1, 256, smem_diag, fs->side>>>(S, k, lds, Kn, st);
        note_launches(2);
        e = cudaEventRecord(fs->join, fs->side);
        if (e != cudaSuccess) return e;
        panel(s, K, head_end, k);
        e = cudaStreamWaitEvent(s, fs->head, 0);
        if (e == cudaSuccess) e = update(K, NB, 1);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, fs->join, 0);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

template cudaError_t launch_cholesky<float>(cudaStream_t, float *, int64_t, int64_t, DevStatus *,
                                            const TcPanel *, KernelTimer *, const FactorStreams *);
template cudaError_t launch_cholesky<double>(cudaStream_t, double *, int64_t, int64_t, DevStatus *,
                                             const TcPanel *, KernelTimer *, const FactorStreams *);

// ---------------------------------------------------------------------------
// Triangular solves: L z = r, then L^T w = z, in place on rhs.
//
// Block row i of a solve needs the m off-diagonal tiles of its row (L_ij,
// j < i, forward; L_ji^T, j > i, backward) times the already solved blocks
// z_j, then z_i = W_i (r_i - sum) with the stored diagonal-block inverse.
// The row is shared out by distance d from the diagonal (d = 0 nearest):
//   helpers    the far part of the row (d >= 4) in at most 8 contiguous
//              segments; each multiplies its tiles as their z_j appear,
//              writes its partial vector to its own slot and counts itself
//              done;
//   finisher   first collects the helpers' partials (their z_j are at least
//              four links old, so this is off the chain), then takes d < 4
//              as each z_j appears, solves the diagonal block and publishes
//              z_i.
// So the chain from z_{i-1} to z_i is one tile product and the diagonal
// solve, and long rows stream through many SMs.  In FP32 a solved entry is
// published as one 64-bit word (tag 1 in the high half, the value's bits in
// the low half) in a buffer cleared before the launch: a consumer polls the
// words it needs directly, one round trip, with no flag and no fence on the
// chain.  FP64 values do not fit beside a tag; they go through rhs with a
// fence and a per-block release flag.
// CTAs draw tickets in launch order; every row's helpers come before its
// finisher and rows come in solve order, so a CTA only ever waits on CTAs
// with smaller tickets, which are running or done.  Every wait is bounded:
// on timeout the CTA raises the launch's abort flag and st->timeout, and all
// CTAs return.

__device__ __forceinline__ int flag_load(const int32_t *p) {
    cuda::atomic_ref<const int32_t, cuda::thread_scope_device> a(*p);
    return a.load(cuda::memory_order_acquire);
}
__device__ __forceinline__ void flag_store(int32_t *p, int v) {
    cuda::atomic_ref<int32_t, cuda::thread_scope_device> a(*p);
    a.store(v, cuda::memory_order_release);
}
__device__ __forceinline__ void count_add(int32_t *p) {
    cuda::atomic_ref<int32_t, cuda::thread_scope_device> a(*p);
    a.fetch_add(1, cuda::memory_order_release);
}
__device__ __forceinline__ uint64_t word_load(const uint64_t *p) {
    cuda::atomic_ref<const uint64_t, cuda::thread_scope_device> a(*p);
    return a.load(cuda::memory_order_relaxed);
}
__device__ __forceinline__ void word_store(uint64_t *p, uint64_t v) {
    cuda::atomic_ref<uint64_t, cuda::thread_scope_device> a(*p);
    a.store(v, cuda::memory_order_relaxed);
}

// Thread 0 polls until *p >= target (bounded), the CTA learns the outcome.
// Ordering: the producer writes its data, then publishes with a release
// store (flag_store / count_add); thread 0 reads the flag with an acquire
// load, so the producer's writes happen before everything thread 0 does
// next, and the CTA barrier below extends that to every thread of the CTA,
// whose reads of the published data come after the barrier.
__device__ __forceinline__ bool wait_at_least(const int32_t *p, int target, int32_t *abort_flag,
                                              DevStatus *st, int *sh_ok) {
    if (threadIdx.x == 0) {
        int ok = 1;
        int spins = 0;
        while (flag_load(p) < target) {
            if (flag_load(abort_flag) != 0) { ok = 0; break; }
            if (++spins > kSpinLimit) {
                flag_store(abort_flag, 1);
                st->timeout = 1;
                ok = 0;
                break;
            }
            if (spins > 8) __nanosleep(32);
        }
        *sh_ok = ok;
    }
    __syncthreads();
    return *sh_ok != 0;
}

// Self-test of the bounded waits: thread 0 polls a flag that nothing sets for
// at most `limit` polls, then records the timeout and returns.
__global__ void wait_probe_kernel(const int32_t *flag, int64_t limit, DevStatus *st) {
    if (threadIdx.x != 0) return;
    int64_t spins = 0;
    while (flag_load(flag) < 1) {
        if (++spins > limit) {
            st->timeout = 1;
            return;
        }
        if (spins > 8) __nanosleep(32);
    }
}

cudaError_t launch_wait_probe(cudaStream_t s, const int32_t *flag, int64_t limit, DevStatus *st) {
    wait_probe_kernel<<<1, 32, 0, s>>>(flag, limit, st);
    note_launches(1);
    return cudaGetLastError();
}

constexpr int kTrsvSeg = 4;      // tiles kept by the finisher, and the helpers' target length
constexpr int kTrsvHelpers = 8;  // helpers per row at most

__host__ __device__ constexpr int trsv_helpers(int m) {
    return m > kTrsvSeg ? ((m - kTrsvSeg + kTrsvSeg - 1) / kTrsvSeg < kTrsvHelpers
                               ? (m - kTrsvSeg + kTrsvSeg - 1) / kTrsvSeg
                               : kTrsvHelpers)
                        : 0;
}

int64_t trsv_ctas(int64_t nblk) {
    int64_t t = 0;
    for (int64_t m = 0; m < nblk; ++m) t += 1 + trsv_helpers((int)m);
    return t;
}

// Scratch: done[nblk], helper counts[nblk], ticket, abort, then (FP32) one
// 64-bit word per row -- all zeroed before each launch -- then one NB-vector
// partial slot per CTA.
static int64_t trsv_zeroed_bytes(int64_t nblk, int64_t nb, size_t elem) {
    const int64_t flags = round_up(4 * (2 * nblk + 2), 256);
    return flags + (elem == sizeof(float) ? round_up(8 * nblk * nb, 256) : 0);
}

size_t chol_solve_scratch_bytes(int64_t k, size_t elem) {
    const int64_t nb = elem == sizeof(float) ? FactorCfg<float>::NB : FactorCfg<double>::NB;
    const int64_t nblk = cdiv(std::max<int64_t>(k, 1), nb);
    return (size_t)trsv_zeroed_bytes(nblk, nb, elem) + (size_t)trsv_ctas(nblk) * (size_t)nb * elem;
}

struct TrsvRole {
    int i;           // block row
    int m;           // off-diagonal tiles in the row
    int nh;          // helpers of the row
    int d_lo, d_hi;  // this CTA's distances [d_lo, d_hi)
    bool finisher;
    int64_t base;    // ticket of the row's first CTA (the helpers' slots follow it)
};

__device__ __forceinline__ TrsvRole trsv_role(int64_t t, int nblk, bool fwd) {
    TrsvRole r{};
    int64_t base = 0;
    for (int q = 0; q < nblk; ++q) {
        const int i = fwd ? q : nblk - 1 - q;
        const int m = fwd ? i : nblk - 1 - i;
        const int nh = trsv_helpers(m);
        if (t < base + nh + 1) {
            const int mf = m < kTrsvSeg ? m : kTrsvSeg;
            const int local = (int)(t - base);
            r.i = i;
            r.m = m;
            r.nh = nh;
            r.base = base;
            r.finisher = local == nh;
            if (r.finisher) {
                r.d_lo = 0;
                r.d_hi = mf;
            } else {
                const int rem = m - mf, lh = (rem + nh - 1) / nh;
                const int h = nh - 1 - local;  // farthest segment first
                r.d_lo = min(m, mf + h * lh);
                r.d_hi = min(m, mf + (h + 1) * lh);
            }
            return r;
        }
        base += nh + 1;
    }
    r.i = -1;
    return r;
}

template <typename T, int NB>
struct TrsvScratch {
    int32_t *done, *hcnt, *ticket, *abort_flag;
    uint64_t *words;  // FP32: published entries (tag << 32 | bits)
    T *part;
    int nblk;
};

template <typename T, int NB>
__host__ TrsvScratch<T, NB> trsv_scratch(void *base, int64_t k) {
    TrsvScratch<T, NB> s;
    s.nblk = (int)cdiv(k, NB);
    s.done = static_cast<int32_t *>(base);
    s.hcnt = s.done + s.nblk;
    s.ticket = s.hcnt + s.nblk;
    s.abort_flag = s.ticket + 1;
    char *p = static_cast<char *>(base) + round_up(4 * (2 * (int64_t)s.nblk + 2), 256);
    s.words = sizeof(T) == sizeof(float) ? reinterpret_cast<uint64_t *>(p) : nullptr;
    s.part = reinterpret_cast<T *>(static_cast<char *>(base) + trsv_zeroed_bytes(s.nblk, NB, sizeof(T)));
    return s;
}

// The same scratch layout `bytes` further on (one region per right-hand side
// of a multi-vector launch).
template <typename T, int NB>
__device__ __forceinline__ TrsvScratch<T, NB> trsv_shift(TrsvScratch<T, NB> s, int64_t bytes) {
    auto mv = [&](auto *p) { return reinterpret_cast<decltype(p)>(reinterpret_cast<char *>(p) + bytes); };
    s.done = mv(s.done);
    s.hcnt = mv(s.hcnt);
    s.ticket = mv(s.ticket);
    s.abort_flag = mv(s.abort_flag);
    if (s.words) s.words = mv(s.words);
    s.part = mv(s.part);
    return s;
}

// zs[0..NB) <- solved block j (nvalid entries, zeros beyond), once available.
// Uniform across the CTA; false when the launch was aborted or a wait timed out.
// tight: every thread polls its own word from the start (one round trip; used
// for the link on the chain, where the block is due any moment).
template <typename T, int NB>
__device__ __forceinline__ bool trsv_get(const TrsvScratch<T, NB> &sc, const T *rhs, int j, int nvalid,
                                         T *zs, DevStatus *st, int *sh_ok, bool tight = false) {
    const int tid = threadIdx.x;
    if constexpr (sizeof(T) == sizeof(float)) {
        // otherwise one thread watches the block's first word, so waiting
        // CTAs leave the memory system to the others; once it is there the
        // rest follow within a few polls each
        if (tid == 0 && tight) *sh_ok = 1;
        if (tid == 0 && !tight) {
            const uint64_t *w0 = sc.words + (int64_t)j * NB;
            int ok = 1, spins = 0;
            while ((word_load(w0) >> 32) == 0) {
                if (++spins > kSpinLimit) {
                    flag_store(sc.abort_flag, 1);
                    st->timeout = 1;
                    ok = 0;
                    break;
                }
                if ((spins & 15) == 0 && flag_load(sc.abort_flag) != 0) { ok = 0; break; }
                if (spins > 8) __nanosleep(32);
            }
            *sh_ok = ok;
        }
        __syncthreads();
        int ok = *sh_ok;
        if (tid < NB) {
            T v = T(0);
            if (ok && tid < nvalid) {
                const uint64_t *w = sc.words + (int64_t)j * NB + tid;
                uint64_t x;
                int spins = 0;
                while (((x = word_load(w)) >> 32) == 0) {
                    if (++spins > kSpinLimit) {
                        flag_store(sc.abort_flag, 1);
                        st->timeout = 1;
                        ok = 0;
                        break;
                    }
                    if ((spins & 15) == 0 && flag_load(sc.abort_flag) != 0) { ok = 0; break; }
                    __nanosleep(32);
                }
                v = ok ? __uint_as_float((uint32_t)x) : T(0);
            }
            zs[tid] = v;
        }
        return __syncthreads_and(ok) != 0;
    } else {
        if (!wait_at_least(sc.done + j, 1, sc.abort_flag, st, sh_ok)) return false;
        if (tid < NB) zs[tid] = tid < nvalid ? __ldcg(rhs + (int64_t)j * NB + tid) : T(0);
        __syncthreads();
        return true;
    }
}

// Publish the nr entries of solved block i (thread tid holds entry tid).
template <typename T, int NB>
__device__ __forceinline__ void trsv_put(const TrsvScratch<T, NB> &sc, T *rhs, int i, int nr, T z) {
    const int tid = threadIdx.x;
    const int64_t row0 = (int64_t)i * NB;
    if constexpr (sizeof(T) == sizeof(float)) {
        if (tid < nr) {
            rhs[row0 + tid] = z;
            word_store(sc.words + row0 + tid, (uint64_t(1) << 32) | __float_as_uint(z));
        }
    } else {
        if (tid < nr) {
            rhs[row0 + tid] = z;
            __threadfence();
        }
        __syncthreads();
        if (tid == 0) flag_store(sc.done + i, 1);
    }
}

// Forward: thread (r = tid % NB, part = tid / NB) owns row r and a slice of
// NB / P columns of every tile, P = 256 / NB parts.
template <typename T, int NB>
__global__ void __launch_bounds__(256)
    trsv_fwd_kernel(const T *__restrict__ L, int64_t k, int64_t lds, T *rhs, TrsvScratch<T, NB> sc,
                    DevStatus *st, int64_t rhs_ld, int64_t sc_stride) {
    constexpr int P = 256 / NB, CW = NB / P;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T(*Wr)[NB + 4] = reinterpret_cast<T(*)[NB + 4]>(smem_raw);  // Wr[r][l] = W(r, l)
    __shared__ __align__(16) T zs[NB];
    __shared__ T red[P][NB];
    __shared__ int64_t tk_sh;
    __shared__ int ok_sh;
    const int tid = threadIdx.x;
    if (blockIdx.y > 0) {  // right-hand side blockIdx.y of a multi-vector launch: its own chain
        rhs += (int64_t)blockIdx.y * rhs_ld;
        sc = trsv_shift(sc, (int64_t)blockIdx.y * sc_stride);
    }
    if (tid == 0) tk_sh = atomicAdd(sc.ticket, 1);
    __syncthreads();
    const int64_t tk = tk_sh;
    const TrsvRole ro = trsv_role(tk, sc.nblk, true);
    if (ro.i < 0) return;
    const int i = ro.i;
    const int64_t row0 = (int64_t)i * NB;
    const int nr = (int)min((int64_t)NB, k - row0);
    const int r = tid % NB, part = tid / NB;
    // tiles in the order their z_j appear: j = i - 1 - d, d from d_hi - 1 down
    T tile[CW];
    auto fetch = [&](int j) {
        if (r < nr) {
#pragma unroll
            for (int c = 0; c < CW; ++c) tile[c] = L[(row0 + r) + ((int64_t)j * NB + part * CW + c) * lds];
        }
    };
    if (ro.d_hi > ro.d_lo) fetch(i - ro.d_hi);
    T ri = T(0), hsum = T(0);
    if (ro.finisher) {
        if (tid < nr) ri = rhs[row0 + tid];
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
                if (l != rr) Wr[rr][l] = v[u];
            }
        }
        // the diagonal of W (written by no one else), one reciprocal per thread
        if (tid < NB) Wr[tid][tid] = tid < nr ? T(1) / L[(row0 + tid) + (row0 + tid) * lds] : T(0);
        if (ro.nh > 0) {
            if (!wait_at_least(sc.hcnt + i, ro.nh, sc.abort_flag, st, &ok_sh)) return;
            if (tid < NB)
                for (int h = 0; h < ro.nh; ++h) hsum += __ldcg(sc.part + (ro.base + h) * NB + tid);
        }
    }
    // four partial sums per product (short dependency chains), z read as
    // 4-vectors (broadcast shared loads)
    T acc4[4] = {T(0), T(0), T(0), T(0)};
    for (int d = ro.d_hi - 1; d >= ro.d_lo; --d) {
        const int j = i - 1 - d;
        if (!trsv_get<T, NB>(sc, rhs, j, NB, zs, st, &ok_sh, ro.finisher && d == 0)) return;
        if (r < nr) {
#pragma unroll
            for (int c = 0; c < CW; c += 4) {
                T zv[4];
                ld4(&zs[part * CW + c], zv);
#pragma unroll
                for (int u = 0; u < 4; ++u) acc4[u] += tile[c + u] * zv[u];
            }
        }
        if (d > ro.d_lo) fetch(j + 1);
        __syncthreads();
    }
    const T acc = (acc4[0] + acc4[1]) + (acc4[2] + acc4[3]);
    red[part][r] = acc;
    __syncthreads();
    if (!ro.finisher) {
        if (tid < NB) {
            T sum = T(0);
#pragma unroll
            for (int q = 0; q < P; ++q) sum += red[q][tid];
            sc.part[tk * NB + tid] = sum;
            __threadfence();
        }
        __syncthreads();
        if (tid == 0) count_add(sc.hcnt + i);
        return;
    }
    if (tid < NB) {
        T sum = hsum;
#pragma unroll
        for (int q = 0; q < P; ++q) sum += red[q][tid];
        zs[tid] = tid < nr ? ri - sum : T(0);
    }
    __syncthreads();
    T z4[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll 4
    for (int c = 0; c < CW; c += 4) {
        T wv[4], zv[4];
        ld4(&Wr[r][part * CW + c], wv);
        ld4(&zs[part * CW + c], zv);
#pragma unroll
        for (int u = 0; u < 4; ++u) z4[u] += wv[u] * zv[u];
    }
    red[part][r] = (z4[0] + z4[1]) + (z4[2] + z4[3]);
    __syncthreads();
    T zi = T(0);
    if (tid < nr) {
#pragma unroll
        for (int q = 0; q < P; ++q) zi += red[q][tid];
    }
    trsv_put<T, NB>(sc, rhs, i, nr, zi);
}

// Backward: (L^T)(row0 + r, jr0 + c) = L(jr0 + c, row0 + r).  Warp w owns the
// columns r = w, w + 8, ... of L (NB / 8 of them); its lanes run down each
// column (coalesced) and reduce by shuffles.
template <typename T, int NB>
__global__ void __launch_bounds__(256)
    trsv_bwd_kernel(const T *__restrict__ L, int64_t k, int64_t lds, T *rhs, TrsvScratch<T, NB> sc,
                    DevStatus *st, int64_t rhs_ld, int64_t sc_stride) {
    constexpr int CPW = NB / 8;   // columns per warp
    constexpr int RPL = NB / 32;  // rows per lane per column
    constexpr int P = 256 / NB, CW = NB / P;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T(*Ws)[NB + 4] = reinterpret_cast<T(*)[NB + 4]>(smem_raw);  // Ws[l][r] = W(r, l)
    __shared__ __align__(16) T ws[NB];
    __shared__ T accs[NB];
    __shared__ T red[P][NB];
    __shared__ int64_t tk_sh;
    __shared__ int ok_sh;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (blockIdx.y > 0) {  // right-hand side blockIdx.y of a multi-vector launch: its own chain
        rhs += (int64_t)blockIdx.y * rhs_ld;
        sc = trsv_shift(sc, (int64_t)blockIdx.y * sc_stride);
    }
    if (tid == 0) tk_sh = atomicAdd(sc.ticket, 1);
    __syncthreads();
    const int64_t tk = tk_sh;
    const TrsvRole ro = trsv_role(tk, sc.nblk, false);
    if (ro.i < 0) return;
    const int i = ro.i;
    const int64_t row0 = (int64_t)i * NB;
    const int nr = (int)min((int64_t)NB, k - row0);
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
    // tiles in the order their w_j appear: j = i + 1 + d, d from d_hi - 1 down
    if (ro.d_hi > ro.d_lo) fetch(i + ro.d_hi);
    T ri = T(0), hsum = T(0);
    if (ro.finisher) {
        if (tid < nr) ri = rhs[row0 + tid];
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
                if (l != rr) Ws[l][rr] = v[u];
            }
        }
        // the diagonal of W (written by no one else), one reciprocal per thread
        if (tid < NB) Ws[tid][tid] = tid < nr ? T(1) / L[(row0 + tid) + (row0 + tid) * lds] : T(0);
        if (ro.nh > 0) {
            if (!wait_at_least(sc.hcnt + i, ro.nh, sc.abort_flag, st, &ok_sh)) return;
            if (tid < NB)
                for (int h = 0; h < ro.nh; ++h) hsum += __ldcg(sc.part + (ro.base + h) * NB + tid);
        }
    }
    T acc[CPW];
#pragma unroll
    for (int q = 0; q < CPW; ++q) acc[q] = T(0);
    for (int d = ro.d_hi - 1; d >= ro.d_lo; --d) {
        const int j = i + 1 + d;
        const int njr = (int)min((int64_t)NB, k - (int64_t)j * NB);
        if (!trsv_get<T, NB>(sc, rhs, j, njr, ws, st, &ok_sh, ro.finisher && d == 0)) return;
#pragma unroll
        for (int q = 0; q < CPW; ++q) {
            T s = T(0);
#pragma unroll
            for (int t = 0; t < RPL; ++t) s += tile[q][t] * ws[lane + 32 * t];
            acc[q] += s;
        }
        if (d > ro.d_lo) fetch(j - 1);
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
    if (!ro.finisher) {
        if (tid < NB) {
            sc.part[tk * NB + tid] = accs[tid];
            __threadfence();
        }
        __syncthreads();
        if (tid == 0) count_add(sc.hcnt + i);
        return;
    }
    if (tid < NB) ws[tid] = tid < nr ? ri - (accs[tid] + hsum) : T(0);
    __syncthreads();
    // w_i = W^T ws: w(r) = sum_{l >= r} W(l, r) ws(l) = sum_l Ws[r][l] ws(l)
    const int r = tid % NB, part = tid / NB;
    T w4[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll 4
    for (int c = 0; c < CW; c += 4) {
        T wv[4], zv[4];
        ld4(&Ws[r][part * CW + c], wv);
        ld4(&ws[part * CW + c], zv);
#pragma unroll
        for (int u = 0; u < 4; ++u) w4[u] += wv[u] * zv[u];
    }
    red[part][r] = (w4[0] + w4[1]) + (w4[2] + w4[3]);
    __syncthreads();
    T wi = T(0);
    if (tid < nr) {
#pragma unroll
        for (int q = 0; q < P; ++q) wi += red[q][tid];
    }
    trsv_put<T, NB>(sc, rhs, i, nr, wi);
}

// dir: bit 0 = forward (L z = rhs), bit 1 = backward (L^T w = rhs), in that order
size_t trsv_multi_scratch_bytes(int64_t k, size_t elem, int q) {
    return (size_t)std::max(q, 1) * (size_t)round_up((int64_t)chol_solve_scratch_bytes(k, elem), 256);
}

// dir: bit 0 = forward (L z = rhs), bit 1 = backward (L^T w = rhs), in that
// order; q right-hand sides rhs + j rhs_ld, each with its own chain of CTAs
// (grid y) and scratch region.
template <typename T>
static cudaError_t launch_trsv_dirs(cudaStream_t s, const T *L, int64_t k, int64_t lds, T *rhs, void *scratch,
                                    DevStatus *st, int dirs, int q = 1, int64_t rhs_ld = 0) {
    constexpr int NB = FactorCfg<T>::NB;
    if (k <= 0 || q <= 0) return cudaSuccess;
    const TrsvScratch<T, NB> sc = trsv_scratch<T, NB>(scratch, k);
    const int64_t ctas = trsv_ctas(sc.nblk);
    const int64_t stride = q > 1 ? round_up((int64_t)chol_solve_scratch_bytes(k, sizeof(T)), 256) : 0;
    // flags, ticket, abort and the published words start at zero for each pass
    const size_t bytes = q > 1 ? (size_t)(stride * q) : (size_t)trsv_zeroed_bytes(sc.nblk, NB, sizeof(T));
    const dim3 grid((unsigned)ctas, (unsigned)q);
    const size_t smem = sizeof(T) * NB * (NB + 4);
    cudaError_t e = cudaFuncSetAttribute(trsv_fwd_kernel<T, NB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(trsv_bwd_kernel<T, NB>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (dirs & 1) {
        e = cudaMemsetAsync(sc.done, 0, bytes, s);
        if (e != cudaSuccess) return e;
        trsv_fwd_kernel<T, NB><<<grid, 256, smem, s>>>(L, k, lds, rhs, sc, st, rhs_ld, stride);
        note_launches(1);
    }
    if (dirs & 2) {
        e = cudaMemsetAsync(sc.done, 0, bytes, s);
        if (e != cudaSuccess) return e;
        trsv_bwd_kernel<T, NB><<<grid, 256, smem, s>>>(L, k, lds, rhs, sc, st, rhs_ld, stride);
        note_launches(1);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_chol_solve(cudaStream_t s, const T *L, int64_t k, int64_t lds, T *rhs, void *scratch,
                              DevStatus *st) {
    return launch_trsv_dirs<T>(s, L, k, lds, rhs, scratch, st, 3);
}
template <typename T>
cudaError_t launch_trsv_fwd(cudaStream_t s, const T *L, int64_t k, int64_t lds, T *rhs, void *scratch,
                            DevStatus *st) {
    return launch_trsv_dirs<T>(s, L, k, lds, rhs, scratch, st, 1);
}
template <typename T>
cudaError_t launch_trsv_bwd(cudaStream_t s, const T *L, int64_t k, int64_t lds, T *rhs, void *scratch,
                            DevStatus *st) {
    return launch_trsv_dirs<T>(s, L, k, lds, rhs, scratch, st, 2);
}
template <typename T>
cudaError_t launch_trsv_multi(cudaStream_t s, const T *L, int64_t k, int64_t lds, T *rhs, int64_t rhs_ld, int q,
                              void *scratch, DevStatus *st, int dirs) {
    return launch_trsv_dirs<T>(s, L, k, lds, rhs, scratch, st, dirs, q, rhs_ld);
}
template cudaError_t launch_trsv_multi<float>(cudaStream_t, const float *, int64_t, int64_t, float *, int64_t, int,
                                              void *, DevStatus *, int);
template cudaError_t launch_trsv_multi<double>(cudaStream_t, const double *, int64_t, int64_t, double *, int64_t,
                                               int, void *, DevStatus *, int);
template cudaError_t launch_trsv_fwd<float>(cudaStream_t, const float *, int64_t, int64_t, float *, void *,
                                            DevStatus *);
template cudaError_t launch_trsv_fwd<double>(cudaStream_t, const double *, int64_t, int64_t, double *, void *,
                                             DevStatus *);
template cudaError_t launch_trsv_bwd<float>(cudaStream_t, const float *, int64_t, int64_t, float *, void *,
                                            DevStatus *);
template cudaError_t launch_trsv_bwd<double>(cudaStream_t, const double *, int64_t, int64_t, double *, void *,
                                             DevStatus *);

template cudaError_t launch_chol_solve<float>(cudaStream_t, const float *, int64_t, int64_t,
                                              float *, void *, DevStatus *);
template cudaError_t launch_chol_solve<double>(cudaStream_t, const double *, int64_t, int64_t,
                                               double *, void *, DevStatus *);

}  // namespace tsnnls
