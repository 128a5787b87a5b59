// Batched dense solves: many small or uneven NNLS problems at once.
//
// Each problem i has a dense FP32 A_i (m_i x n_i, row-major), FP64 b_i and x_i.
// The work is two kernels, captured once into a CUDA graph and replayed:
//   1. batched precompute (Section 3): G_i = A_i^T A_i (lower tiles; MIXED
//      on the tensor cores, TF32 with a hi/lo split) and c_i = A_i^T b_i
//      (FP64), over one flat list of (problem, tile) work items;
//   2. one persistent kernel: each CTA takes problems from an atomic queue,
//      largest first, and runs the whole pivot loop of Section 2 for it --
//      exchange, gather of G_FF, blocked Cholesky, triangular solves, FP64
//      iterative refinement (MIXED) and y_G -- with CTA barriers only, so
//      no CTA ever waits on another.
// The Cholesky panel width of each problem comes from a per-size table that
// the autotuner (tsnnls_batch_autotune) fills by timing the candidates.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "check.cuh"
#include "dense_block.cuh"
#include "engine.h"

namespace tsnnls {

struct BatchProb {
    const float *A;  // m x n row-major
    const double *b;
    double *x;       // caller's output (also the iterate)
    float *G;        // n x ld lower (FP32 precompute)
    void *S;         // n x ld factor workspace (float or double)
    double *Gd;      // FP64 path: n x ld lower Gram in FP64 (else null)
    double *c, *y, *s, *r;
    double *cb;      // MIXED: c = |A|^T (|A| 1), the settle test's bound (else null)
    void *rhs;       // n (factor type)
    int32_t *F;
    uint8_t *inF;
    int64_t *trace;  // optional pivot trace, trace_cap rows of 6 (else null)
    int32_t m, n, ld, nb, trace_cap;
};

struct BatchOut {
    int32_t status, iters, refine, nF;
    double flops;  // algorithmic flops of the pivot loop (factors, solves, residuals)
};

struct BatchParams {
    double zero_tol, rel_tol;
    int32_t p_max, max_iter, max_refine, mixed;
    int32_t scratch_bytes;  // bytes of the panel area free outside the factorisation
    int32_t settle;         // MIXED: intermediate pivots stop refining once their signs are settled
};

// ---------------------------------------------------------------------------
// 1. precompute: G = A^T A lower 64 x 64 tiles (MIXED: FP32 on the tensor
//    cores, batch_gram_tc_kernel below; FP64: FP64 products); c = A^T b in FP64.

struct GramItem {
    int32_t prob, I, J;
};

// FP64 Gram for the plain FP64 path (same tiling, FP64 products of the FP32 data).
__global__ void __launch_bounds__(256)
    batch_gram64_kernel(const BatchProb *__restrict__ probs, const GramItem *__restrict__ items,
                        int32_t nitems) {
    __shared__ double As[8][68];
    __shared__ double Bs[8][68];
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const GramItem w = items[it];
        const BatchProb P = probs[w.prob];
        const int n = P.n, m = P.m;
        const int r0 = w.I * 64, c0 = w.J * 64;
        const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
        double acc[4][4] = {};
        for (int k0 = 0; k0 < m; k0 += 8) {
            for (int e = threadIdx.x; e < 8 * 64; e += 256) {
                const int kk = e / 64, i = e % 64;
                const int row = k0 + kk;
                As[kk][i] = (row < m && r0 + i < n) ? (double)P.A[(int64_t)row * n + r0 + i] : 0.0;
                Bs[kk][i] = (row < m && c0 + i < n) ? (double)P.A[(int64_t)row * n + c0 + i] : 0.0;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
                double a[4], bb[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    a[q] = As[kk][ty + 16 * q];
                    bb[q] = Bs[kk][tx + 16 * q];
                }
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int t = 0; t < 4; ++t) acc[q][t] += a[q] * bb[t];
            }
            __syncthreads();
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = r0 + ty + 16 * q;
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int j = c0 + tx + 16 * t;
                if (i < n && j < n && i >= j) P.Gd[i + (int64_t)j * P.ld] = acc[q][t];
            }
        }
    }
}

// c = A^T b in FP64, one CTA per problem, threads over columns (coalesced).
__global__ void __launch_bounds__(256)
    batch_atb_kernel(const BatchProb *__restrict__ probs, int32_t count) {
    for (int p = blockIdx.x; p < count; p += gridDim.x) {
        const BatchProb P = probs[p];
        for (int j = threadIdx.x; j < P.n; j += blockDim.x) {
            double s = 0.0;
            for (int r = 0; r < P.m; ++r) s += (double)P.A[(int64_t)r * P.n + j] * P.b[r];
            P.c[j] = s;
        }
    }
}

// ---------------------------------------------------------------------------
// 2. the persistent pivot-loop kernel

constexpr int kBT = 512;            // threads per CTA
constexpr int kBWarps = kBT / 32;
constexpr int kMaxPanelRows = 1024;  // n <= 1024 for this path

// pitch of the shared-memory panel rows P[row * pitch + l]
template <typename T>
__host__ __device__ __forceinline__ int panel_pitch(int nb) {
    return (sizeof(T) == 4 && nb == 32) ? 36 : nb + 1;
}

// ---- trailing update on the tensor cores (FP32 path, panel width 32) ------
// C(R0 + i, R0 + j) -= sum_l X(i, l) X(j, l) on the lower triangle, X the
// 32-column panel in shared memory (pitch 36).  Each warp takes 32 x 32
// tiles: 2 x 4 mma.sync.m16n8k8 TF32 tiles, K = 32 in four steps.  TF32 keeps
// 10 mantissa bits, so every operand is split into hi (rounded to TF32) and
// lo (the rest, rounded to TF32) and the product is accumulated as
// hi*hi + hi*lo + lo*hi in FP32, which carries about FP32 accuracy.
// Fragment layout of m16n8k8 (g = lane / 4, t = lane % 4): A (16 x 8)
// a0 = (g, t), a1 = (g + 8, t), a2 = (g, t + 4), a3 = (g + 8, t + 4);
// B (8 x 8) b0 = (t, g), b1 = (t + 4, g); C (16 x 8) c0 = (g, 2t),
// c1 = (g, 2t + 1), c2 = (g + 8, 2t), c3 = (g + 8, 2t + 1).
__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ void split_tf32(float x, uint32_t &hi, uint32_t &lo) {
    hi = to_tf32(x);
    lo = to_tf32(x - __uint_as_float(hi));
}
__device__ __forceinline__ void mma_tf32_16x8x8(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __noinline__ void tc_trailing_update(float *S, int lds, int R0, int nr, const float *panel) {
    constexpr int PP = 36;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
    const int nt = (nr + 31) / 32, ntiles = nt * (nt + 1) / 2;
    auto X = [&](int r, int l) -> float { return r < nr ? panel[r * PP + l] : 0.f; };
    for (int tb = warp; tb < ntiles; tb += kBWarps) {
        int I = (int)((sqrtf(8.f * tb + 1.f) - 1.f) * 0.5f);
        while (I * (I + 1) / 2 > tb) --I;
        while ((I + 1) * (I + 2) / 2 <= tb) ++I;
        const int J = tb - I * (I + 1) / 2;
        const int i0 = I * 32, j0 = J * 32;
        // the accumulators start as the tile of C, all 32 loads issued
        // before the MMAs so that their latency passes under them, and the
        // MMAs add (-X) X^T (the A fragments with the sign bit flipped)
        float acc[2][4][4];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int r = i0 + 16 * a + g + (q >= 2 ? 8 : 0);
                    const int c = j0 + 8 * b + 2 * t + (q & 1);
                    acc[a][b][q] = (r < nr && c < nr && r >= c) ? S[(R0 + r) + (int64_t)(R0 + c) * lds] : 0.f;
                }
#pragma unroll
        for (int k0 = 0; k0 < 32; k0 += 8) {
            uint32_t ah[2][4], al[2][4], bh[4][2], bl[4][2];
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const int ra = i0 + 16 * a + g;
                split_tf32(X(ra, k0 + t), ah[a][0], al[a][0]);
                split_tf32(X(ra + 8, k0 + t), ah[a][1], al[a][1]);
                split_tf32(X(ra, k0 + t + 4), ah[a][2], al[a][2]);
                split_tf32(X(ra + 8, k0 + t + 4), ah[a][3], al[a][3]);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    ah[a][q] ^= 0x80000000u;
                    al[a][q] ^= 0x80000000u;
                }
            }
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int cj = j0 + 8 * b + g;  // B(l, j) = X(j, l)
                split_tf32(X(cj, k0 + t), bh[b][0], bl[b][0]);
                split_tf32(X(cj, k0 + t + 4), bh[b][1], bl[b][1]);
            }
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    mma_tf32_16x8x8(acc[a][b], ah[a], bh[b]);
                    mma_tf32_16x8x8(acc[a][b], ah[a], bl[b]);
                    mma_tf32_16x8x8(acc[a][b], al[a], bh[b]);
                }
        }
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int r = i0 + 16 * a + g + (q >= 2 ? 8 : 0);
                    const int c = j0 + 8 * b + 2 * t + (q & 1);
                    if (r < nr && c < nr && r >= c) S[(R0 + r) + (int64_t)(R0 + c) * lds] = acc[a][b][q];
                }
    }
}

__device__ __forceinline__ double block_reduce_sum(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0) {
        for (int w = 0; w < kBWarps; ++w) t += sh[w];  // fixed order
        sh[0] = t;
    }
    __syncthreads();
    return sh[0];
}

__device__ __forceinline__ double block_reduce_max(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kBWarps; ++w) t = fmax(t, sh[w]);
        sh[0] = t;
    }
    __syncthreads();
    return sh[0];
}

__device__ __forceinline__ int block_reduce_isum(int v, int *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < kBWarps; ++w) t += sh[w];
        sh[0] = t;
    }
    __syncthreads();
    return sh[0];
}

__device__ __forceinline__ int block_reduce_imax(int v, int *sh) {
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = -1;
        for (int w = 0; w < kBWarps; ++w) t = max(t, sh[w]);
        sh[0] = t;
    }
    __syncthreads();
    return sh[0];
}

// Warp 0: factor the kb x kb (kb <= 32) diagonal block at (K, K) of S in
// registers (lane = row, the warp step of dense_block.cuh: the pivot chain
// by shuffles, no CTA barrier); L into S and into diag (diag[c * 65 + r]).
// Returns 0 or the 1-based column of the first non-positive pivot.
template <typename T>
__device__ __noinline__ int warp_factor_block(T *S, int lds, int K, int kb, T *diag, T (*col)[32]) {
    const int lane = threadIdx.x & 31;
    WarpCholL<T> s;
#pragma unroll
    for (int c = 0; c < 32; ++c)  // rows past kb hold the identity, so they factor to it and touch nothing
        s.a[c] = (lane < kb && c <= lane) ? S[(K + lane) + (int64_t)(K + c) * lds] : (c == lane ? T(1) : T(0));
    int bad = 0;
    warp_chol_step_l<T, 0>(s, col, lane, bad, __shfl_sync(0xffffffffu, s.a[0], 0));
#pragma unroll
    for (int c = 0; c < 32; ++c)
        if (lane < kb && c <= lane) {
            S[(K + lane) + (int64_t)(K + c) * lds] = s.a[c];
            diag[c * 65 + lane] = s.a[c];
        }
    return bad;
}

// G = A^T A on the tensor cores (MIXED precompute): one 64 x 64 lower tile
// per CTA and work item, 8 warps of 16 x 32, rows of A staged 32 at a time
// (pitch 72, so the fragment loads of a warp hit distinct banks);
// mma.sync m16n8k8 TF32 with the hi/lo split as in tc_trailing_update.
// A_mma(i, r) = A(r, r0 + i), B_mma(r, j) = A(r, c0 + j).
__global__ void __launch_bounds__(256)
    batch_gram_tc_kernel(const BatchProb *__restrict__ probs, const GramItem *__restrict__ items,
                         int32_t nitems) {
    constexpr int KC = 32, PT = 72;
    __shared__ __align__(16) float As[KC][PT];
    __shared__ __align__(16) float Bs[KC][PT];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 2, t = lane & 3;
    const int mi = (warp & 3) * 16, nj0 = (warp >> 2) * 32;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const GramItem w = items[it];
        const BatchProb P = probs[w.prob];
        const int n = P.n, m = P.m;
        const int r0 = w.I * 64, c0 = w.J * 64;
        float acc[4][4];
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[b][q] = 0.f;
        for (int k0 = 0; k0 < m; k0 += KC) {
            __syncthreads();
            for (int e = threadIdx.x; e < KC * 64; e += 256) {
                const int kk = e / 64, i = e % 64;
                const int row = k0 + kk;
                As[kk][i] = (row < m && r0 + i < n) ? P.A[(int64_t)row * n + r0 + i] : 0.f;
                Bs[kk][i] = (row < m && c0 + i < n) ? P.A[(int64_t)row * n + c0 + i] : 0.f;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < KC; kk += 8) {
                uint32_t ah[4], al[4];
                split_tf32(As[kk + t][mi + g], ah[0], al[0]);
                split_tf32(As[kk + t][mi + g + 8], ah[1], al[1]);
                split_tf32(As[kk + t + 4][mi + g], ah[2], al[2]);
                split_tf32(As[kk + t + 4][mi + g + 8], ah[3], al[3]);
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    uint32_t bh[2], bl[2];
                    split_tf32(Bs[kk + t][nj0 + 8 * b + g], bh[0], bl[0]);
                    split_tf32(Bs[kk + t + 4][nj0 + 8 * b + g], bh[1], bl[1]);
                    mma_tf32_16x8x8(acc[b], ah, bh);
                    mma_tf32_16x8x8(acc[b], ah, bl);
                    mma_tf32_16x8x8(acc[b], al, bh);
                }
            }
        }
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = r0 + mi + g + (q >= 2 ? 8 : 0);
                const int j = c0 + nj0 + 8 * b + 2 * t + (q & 1);
                if (i < n && j < n && i >= j) P.G[i + (int64_t)j * P.ld] = acc[b][q];
            }
    }
}

// In-CTA blocked right-looking Cholesky of the k x k lower matrix S (lds),
// panel width nb <= 64.  Returns 0 or 1 + the failing column.  With nb = 32
// warp 0 factors each diagonal block in registers; other widths factor it
// column by column with the whole CTA.
template <typename T>
__device__ int cta_cholesky(T *S, int k, int lds, int nb, T *panel, T *diag, int *sh_int) {
    __shared__ __align__(16) T col[2][32];
    const int tid = threadIdx.x;
    int info = 0;
    for (int K = 0; K < k; K += nb) {
        const int kb = min(nb, k - K);
        if (nb == 32) {
            if (tid < 32) {
                const int bad = warp_factor_block<T>(S, lds, K, kb, diag, col);
                if (tid == 0) sh_int[0] = (bad && !info) ? K + bad : info;
            }
            __syncthreads();
            info = sh_int[0];
        } else {
        // diagonal block in shared memory, factored column by column
        for (int e = tid; e < kb * kb; e += kBT) {
            const int c = e / kb, r = e % kb;
            if (r >= c) diag[c * 65 + r] = S[(K + r) + (int64_t)(K + c) * lds];
        }
        __syncthreads();
        for (int j = 0; j < kb; ++j) {
            if (tid == 0) {
                T d = diag[j * 65 + j];
                if (!(d > T(0))) {
                    if (!info) info = K + j + 1;
                    d = T(1);
                }
                diag[j * 65 + j] = sqrt(d);
                sh_int[0] = info;
            }
            __syncthreads();
            const T djj = diag[j * 65 + j];
            for (int i = j + 1 + tid; i < kb; i += kBT) diag[j * 65 + i] /= djj;
            __syncthreads();
            const int rem = kb - j - 1;
            for (int e = tid; e < rem * rem; e += kBT) {
                const int l = j + 1 + e / rem, i = j + 1 + e % rem;
                if (i >= l) diag[l * 65 + i] -= diag[j * 65 + i] * diag[j * 65 + l];
            }
            __syncthreads();
        }
        info = sh_int[0];
        for (int e = tid; e < kb * kb; e += kBT) {
            const int c = e / kb, r = e % kb;
            if (r >= c) S[(K + r) + (int64_t)(K + c) * lds] = diag[c * 65 + r];
        }
        }
        // panel: X L_KK^T = B for rows below, one thread per row, into smem
        // (pitch PP: 36 for the tensor-core update's fragment loads, whose rows
        // then fall on distinct banks; columns kb..nb of the last panel are 0)
        const int R0 = K + kb, nr = k - R0;
        const int PP = panel_pitch<T>(nb);
        // (the row's entries are loaded 16 at a time into registers, all 16 in
        // flight, then stored to the panel)
        if (nb == 32) {
            // the row in registers, L_KK read from shared memory (the same
            // entry for every lane: a broadcast)
            for (int r = tid; r < nr; r += kBT) {
                T xr[32];
#pragma unroll
                for (int c = 0; c < 32; ++c) xr[c] = c < kb ? S[(R0 + r) + (int64_t)(K + c) * lds] : T(0);
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    if (c < kb) {
                        T s = xr[c];
#pragma unroll
                        for (int l = 0; l < c; ++l) s -= xr[l] * diag[l * 65 + c];
                        xr[c] = s / diag[c * 65 + c];
                    }
                }
                if constexpr (sizeof(T) == 4) {
                    // 16-byte stores (pitch 36: rows 144 bytes apart, no bank conflict)
#pragma unroll
                    for (int c4 = 0; c4 < 8; ++c4) {
                        const T v4[4] = {xr[4 * c4], xr[4 * c4 + 1], xr[4 * c4 + 2], xr[4 * c4 + 3]};
                        st4(&panel[r * PP + 4 * c4], v4);
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < 32; ++c) panel[r * PP + c] = xr[c];
                }
#pragma unroll
                for (int c = 0; c < 32; ++c)
                    if (c < kb) S[(R0 + r) + (int64_t)(K + c) * lds] = xr[c];
            }
        } else {
        for (int r = tid; r < nr; r += kBT) {
            for (int c0 = 0; c0 < nb; c0 += 16) {
                T rowv[16];
#pragma unroll
                for (int u = 0; u < 16; ++u)
                    rowv[u] = c0 + u < kb ? S[(R0 + r) + (int64_t)(K + c0 + u) * lds] : T(0);
#pragma unroll
                for (int u = 0; u < 16; ++u)
                    if (c0 + u < nb) panel[r * PP + c0 + u] = rowv[u];
            }
            for (int c = 0; c < kb; ++c) {
                T s = panel[r * PP + c];
                for (int l = 0; l < c; ++l) s -= panel[r * PP + l] * diag[l * 65 + c];
                s /= diag[c * 65 + c];
                panel[r * PP + c] = s;
            }
            for (int c = 0; c < kb; ++c) S[(R0 + r) + (int64_t)(K + c) * lds] = panel[r * PP + c];
        }
        }
        __syncthreads();
        if constexpr (sizeof(T) == 4) {
            if (nb == 32 && nr > 0) {
                tc_trailing_update(S, lds, R0, nr, panel);
                __syncthreads();
                continue;
            }
        }
        // trailing update of the lower triangle, 4 x 4 register tiles over 64 x 64 tiles
        if (nr > 0) {
            const int t64 = (nr + 63) / 64;
            const int ntiles = t64 * (t64 + 1) / 2;
            // two 256-thread halves, one tile each; consecutive lanes take
            // consecutive rows, so the column-major read-modify-write of S
            // is coalesced
            const int sub = tid & 255, half = tid >> 8;
            const int tx = sub >> 4, ty = sub & 15;
            for (int tb = half; tb < ntiles; tb += 2) {
                int I = (int)((sqrtf(8.f * tb + 1.f) - 1.f) * 0.5f);
                while (I * (I + 1) / 2 > tb) --I;
                while ((I + 1) * (I + 2) / 2 <= tb) ++I;
                const int J = tb - I * (I + 1) / 2;
                const int ri = I * 64, cj = J * 64;
                T acc[4][4];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
                for (int l = 0; l < kb; ++l) {
                    T av[4], bv[4];
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        const int rr = ri + ty + 16 * a;
                        av[a] = rr < nr ? panel[rr * PP + l] : T(0);
                    }
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const int cc = cj + tx + 16 * b;
                        bv[b] = cc < nr ? panel[cc * PP + l] : T(0);
                    }
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b) acc[a][b] += av[a] * bv[b];
                }
                // all 16 loads of C before any store: the stores could alias
                // them as far as the compiler can tell, which would serialise
                // every read-modify-write on its memory latency
                T cv[4][4];
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const int rr = ri + ty + 16 * a;
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const int cc = cj + tx + 16 * b;
                        cv[a][b] = (rr < nr && cc < nr && rr >= cc) ? S[(R0 + rr) + (int64_t)(R0 + cc) * lds]
                                                                    : T(0);
                    }
                }
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const int rr = ri + ty + 16 * a;
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const int cc = cj + tx + 16 * b;
                        if (rr < nr && cc < nr && rr >= cc)
                            S[(R0 + rr) + (int64_t)(R0 + cc) * lds] = cv[a][b] - acc[a][b];
                    }
                }
            }
        }
        __syncthreads();
    }
    return info;
}

// Warp 0's solves with one 32 x 32 diagonal block of L at B0 (nb rows):
// lane = row (forward, L z = v) or column (backward, L^T w = v) of the block,
// its entries loaded before the serial shuffle steps.
template <typename T>
__device__ __forceinline__ void warp_diag_fwd(const T *L, int lds, int B0, int nb, T *rhs) {
    const int lane = threadIdx.x & 31;
    T l[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) l[c] = (c < nb && lane < nb) ? L[(B0 + lane) + (int64_t)(B0 + c) * lds] : T(0);
    const T inv = lane < nb ? T(1) / L[(B0 + lane) + (int64_t)(B0 + lane) * lds] : T(0);
    T v = lane < nb ? rhs[B0 + lane] : T(0);
#pragma unroll
    for (int c = 0; c < 32; ++c) {
        if (c < nb) {
            const T zc = __shfl_sync(0xffffffffu, v * inv, c);
            if (lane == c) v = zc;
            if (lane > c) v -= l[c] * zc;
        }
    }
    if (lane < nb) rhs[B0 + lane] = v;
}

template <typename T>
__device__ __forceinline__ void warp_diag_bwd(const T *L, int lds, int B0, int nb, T *rhs) {
    const int lane = threadIdx.x & 31;
    T lt[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) lt[c] = (c < nb && lane < nb) ? L[(B0 + c) + (int64_t)(B0 + lane) * lds] : T(0);
    const T inv = lane < nb ? T(1) / L[(B0 + lane) + (int64_t)(B0 + lane) * lds] : T(0);
    T v = lane < nb ? rhs[B0 + lane] : T(0);
#pragma unroll
    for (int c = 31; c >= 0; --c) {
        if (c < nb) {
            const T wc = __shfl_sync(0xffffffffu, v * inv, c);
            if (lane == c) v = wc;
            if (lane < c) v -= lt[c] * wc;
        }
    }
    if (lane < nb) rhs[B0 + lane] = v;
}

// rhs[r0 + q] -= sum_c L(B0 + c, r0 + q) w_c for the 32 rows r0 .. r0 + 31
// of L^T above the block at B0 (nb columns): lane c loads L(B0 + c, r) down
// the column r (one 128-byte line per load, 32 in flight) scaled by w_c =
// wl; five butterfly steps then leave in lane q the sum over c for row
// r0 + q (at each step a lane keeps the half of its partial sums selected
// by its own bit and adds its partner's).
template <typename T>
__device__ __forceinline__ void warp_bwd_tile(const T *L, int lds, int B0, int nb, int r0, T wl, T *rhs) {
    const int lane = threadIdx.x & 31;
    T v[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) v[q] = lane < nb ? L[(B0 + lane) + (int64_t)(r0 + q) * lds] * wl : T(0);
#pragma unroll
    for (int sft = 16; sft >= 1; sft >>= 1) {
        const bool upper = (lane & sft) != 0;
#pragma unroll
        for (int q = 0; q < sft; ++q) {
            const T send = upper ? v[q] : v[q + sft];
            const T keep = upper ? v[q + sft] : v[q];
            v[q] = keep + __shfl_xor_sync(0xffffffffu, send, sft);
        }
    }
    rhs[r0 + lane] -= v[0];
}

// rhs <- (L L^T)^{-1} rhs inside one CTA, by 32-row blocks with a look-ahead
// of one block: while warps 1.. apply block b's solution to the rows beyond
// block b + 1, warp 0 applies it to the 32 rows of block b + 1 and solves
// that block's diagonal system, so the serial shuffle chain of each diagonal
// block runs beside the bulk update instead of between two barriers.
template <typename T>
__device__ __noinline__ void cta_chol_solve(const T *L, int k, int lds, T *rhs) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (k <= 0) return;
    if (warp == 0) warp_diag_fwd<T>(L, lds, 0, min(32, k), rhs);  // L z = rhs
    __syncthreads();
    for (int B0 = 0; B0 + 32 < k; B0 += 32) {
        const int N0 = B0 + 32, nn = min(32, k - N0);  // the next block
        if (warp == 0) {
            if (lane < nn) {
                const int r = N0 + lane;
                T lv[32];
#pragma unroll
                for (int c = 0; c < 32; ++c) lv[c] = L[r + (int64_t)(B0 + c) * lds];
                T sum = T(0);
#pragma unroll
                for (int c = 0; c < 32; ++c) sum += lv[c] * rhs[B0 + c];
                rhs[r] -= sum;
            }
            __syncwarp();
            warp_diag_fwd<T>(L, lds, N0, nn, rhs);
        } else {
            for (int r = N0 + 32 + (tid - 32); r < k; r += kBT - 32) {
                T lv[32];
#pragma unroll
                for (int c = 0; c < 32; ++c) lv[c] = L[r + (int64_t)(B0 + c) * lds];
                T sum = T(0);
#pragma unroll
                for (int c = 0; c < 32; ++c) sum += lv[c] * rhs[B0 + c];
                rhs[r] -= sum;
            }
        }
        __syncthreads();
    }
    const int nblk = (k + 31) / 32;
    {  // L^T w = z
        const int B0 = (nblk - 1) * 32;
        if (warp == 0) warp_diag_bwd<T>(L, lds, B0, k - B0, rhs);
    }
    __syncthreads();
    for (int bi = nblk - 1; bi > 0; --bi) {
        const int B0 = bi * 32, nb = min(32, k - B0);
        const T wl = lane < nb ? rhs[B0 + lane] : T(0);
        if (warp == 0) {
            warp_bwd_tile<T>(L, lds, B0, nb, B0 - 32, wl, rhs);  // the rows of block bi - 1
            __syncwarp();
            warp_diag_bwd<T>(L, lds, B0 - 32, 32, rhs);
        } else {
            for (int t = warp - 1; t < bi - 1; t += kBWarps - 1) warp_bwd_tile<T>(L, lds, B0, nb, 32 * t, wl, rhs);
        }
        __syncthreads();
    }
}

// ---- FP64-accurate dense products on the FP32 pipes (mixed path) ---------
// GB300 issues FP64 at a small fraction of its FP32 rate, and the
// refinement's dense residual b - A_F x_F and A^T r would be bound by it.
// A is exactly FP32; an FP64 operand v is split into vh = (float)v and
// vl = (float)(v - vh) (v = vh + vl to about 2^-48 relative), the product
// a * vh is formed exactly as ph + pl (pl = fma(a, vh, -ph)), and the sum
// is carried as an unevaluated pair (h, l) with Knuth's two-sum: about 48
// significant bits instead of FP64's 53, enough for the refinement to reach
// the 1e-9 target with a residual floor near 1e-12.
__device__ __forceinline__ void ff_acc(float &h, float &l, float a, float vh, float vl) {
    const float ph = a * vh;
    const float pl = fmaf(a, vh, -ph);
    const float s = h + ph;
    const float bb = s - h;
    const float e = (h - (s - bb)) + (ph - bb);
    h = s;
    l += e + fmaf(a, vl, pl);
}
__device__ __forceinline__ void ff_add(float &h, float &l, float h2, float l2) {
    const float s = h + h2;
    const float bb = s - h;
    const float e = (h - (s - bb)) + (h2 - bb);
    h = s;
    l = (l + l2) + e;
}
__device__ __forceinline__ float2 ff_split(double v) {
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
}

// r = b - A_F x_F with the double-float products above, stored split into
// P.r.  One CTA streams all of A here, so what bounds it is the bytes it
// keeps in flight: x is scattered over all n columns (0 outside F) as hi /
// lo FP32 halves in shared memory, and a warp reads a whole row of A in
// 16-byte chunks, eight per lane issued before the first is used.  A row's
// chunks start at its first 16-byte boundary, h = 0..3 columns in; copy q of
// x is shifted by q columns (xq[t] = x[t + q]) so that every chunk finds its
// four x values in one aligned 16-byte shared load of copy h.  Columns
// before the boundary and after the last whole chunk are taken one by one.
// Without room for the four copies, lanes walk the F list instead.
__device__ __noinline__ void cta_residual_ff(const BatchProb &P, int k, void *scr, int scr_bytes) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n = P.n;
    const int np4 = (n + 7) & ~3;  // entries per copy: columns t + q < n for q <= 3
    float2 *rs = reinterpret_cast<float2 *>(P.r);
    if (32 * np4 <= scr_bytes) {
        float *xc = static_cast<float *>(scr);  // copy q: hi at xc[2q np4], lo at xc[(2q + 1) np4]
        for (int t = threadIdx.x; t < 8 * np4; t += kBT) xc[t] = 0.f;
        __syncthreads();
        for (int a = threadIdx.x; a < k; a += kBT) {
            const int j = P.F[a];
            const float2 v = ff_split(P.x[j]);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (j >= q) {
                    xc[2 * q * np4 + j - q] = v.x;
                    xc[(2 * q + 1) * np4 + j - q] = v.y;
                }
        }
        __syncthreads();
        constexpr int U = 8;
        for (int i = warp; i < P.m; i += kBWarps) {
            const float *row = P.A + (int64_t)i * n;
            const int h = min(n, (int)((16u - ((uint32_t)reinterpret_cast<uintptr_t>(row) & 15u)) & 15u) >> 2);
            const int nch = (n - h) >> 2;  // whole 16-byte chunks
            const float4 *r4 = reinterpret_cast<const float4 *>(row + h);
            const float4 *xh4 = reinterpret_cast<const float4 *>(xc + 2 * h * np4);
            const float4 *xl4 = reinterpret_cast<const float4 *>(xc + (2 * h + 1) * np4);
            float hs = 0.f, ls = 0.f;
            // the columns before the first boundary and after the last chunk
            const int tail0 = h + 4 * nch;
            if (lane < h) ff_acc(hs, ls, row[lane], xc[lane], xc[np4 + lane]);
            if (tail0 + lane < n) ff_acc(hs, ls, row[tail0 + lane], xc[tail0 + lane], xc[np4 + tail0 + lane]);
            for (int c0 = 0; c0 < nch; c0 += 32 * U) {
                float4 v[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int c = c0 + lane + 32 * u;
                    v[u] = c < nch ? __ldcg(r4 + c) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int c = c0 + lane + 32 * u;
                    if (c < nch) {
                        const float4 xh = xh4[c], xl = xl4[c];
                        ff_acc(hs, ls, v[u].x, xh.x, xl.x);
                        ff_acc(hs, ls, v[u].y, xh.y, xl.y);
                        ff_acc(hs, ls, v[u].z, xh.z, xl.z);
                        ff_acc(hs, ls, v[u].w, xh.w, xl.w);
                    }
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const float hh = __shfl_xor_sync(0xffffffffu, hs, o), ll = __shfl_xor_sync(0xffffffffu, ls, o);
                ff_add(hs, ls, hh, ll);
            }
            if (lane == 0) rs[i] = ff_split(P.b[i] - ((double)hs + (double)ls));
        }
        __syncthreads();
        return;
    }
    float2 *xs = reinterpret_cast<float2 *>(P.y);
    for (int a = threadIdx.x; a < k; a += kBT) xs[a] = ff_split(P.x[P.F[a]]);
    __syncthreads();
    for (int i = warp; i < P.m; i += kBWarps) {
        float hs = 0.f, ls = 0.f, h2 = 0.f, l2 = 0.f;
        const float *row = P.A + (int64_t)i * n;
        int a = lane;
        for (; a + 32 < k; a += 64) {  // two gathers in flight per lane
            const float2 v0 = xs[a], v1 = xs[a + 32];
            const float a0 = row[P.F[a]], a1 = row[P.F[a + 32]];
            ff_acc(hs, ls, a0, v0.x, v0.y);
            ff_acc(h2, l2, a1, v1.x, v1.y);
        }
        if (a < k) ff_acc(hs, ls, row[P.F[a]], xs[a].x, xs[a].y);
        ff_add(hs, ls, h2, l2);
        for (int o = 16; o > 0; o >>= 1) {
            const float hh = __shfl_xor_sync(0xffffffffu, hs, o), ll = __shfl_xor_sync(0xffffffffu, ls, o);
            ff_add(hs, ls, hh, ll);
        }
        if (lane == 0) rs[i] = ff_split(P.b[i] - ((double)hs + (double)ls));
    }
    __syncthreads();
}

// s_j = (A^T r)_j with r split in P.r (staged in shared memory when it
// fits); only the F columns unless all_cols.  Threads over columns (a
// warp's loads of one row are one 128-byte line), rows in groups of 16
// whose loads are all issued before the first product, in row order.
__device__ __noinline__ void cta_atr_ff(const BatchProb &P, bool all_cols, void *scr, int scr_bytes) {
    const bool staged = 8 * P.m <= scr_bytes;
    const float2 *rs = reinterpret_cast<const float2 *>(P.r);
    if (staged) {
        float2 *rsm = static_cast<float2 *>(scr);
        for (int i = threadIdx.x; i < P.m; i += kBT) rsm[i] = rs[i];
        __syncthreads();
        rs = rsm;
    }
    const int n = P.n, m = P.m;
    constexpr int R = 16;
    for (int j = threadIdx.x; j < n; j += kBT) {
        if (!all_cols && !P.inF[j]) continue;
        const float *col = P.A + j;
        float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;  // two chains, even and odd rows
        int i = 0;
        for (; i + R <= m; i += R) {
            float a[R];
#pragma unroll
            for (int u = 0; u < R; ++u) a[u] = __ldcg(col + (int64_t)(i + u) * n);
#pragma unroll
            for (int u = 0; u < R; u += 2) {
                const float2 v0 = rs[i + u], v1 = rs[i + u + 1];
                ff_acc(h0, l0, a[u], v0.x, v0.y);
                ff_acc(h1, l1, a[u + 1], v1.x, v1.y);
            }
        }
        for (; i < m; ++i) ff_acc(h0, l0, col[(int64_t)i * n], rs[i].x, rs[i].y);
        ff_add(h0, l0, h1, l1);
        P.s[j] = (double)h0 + (double)l0;
    }
    __syncthreads();
}

// r = b - A x (x zero outside F): warps over rows, lanes over the F list.
__device__ void cta_residual(const BatchProb &P, int k) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = warp; i < P.m; i += kBWarps) {
        double s = 0.0;
        const float *row = P.A + (int64_t)i * P.n;
        for (int a = lane; a < k; a += 32) {
            const int j = P.F[a];
            s += (double)row[j] * P.x[j];
        }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) P.r[i] = P.b[i] - s;
    }
    __syncthreads();
}

// s = A^T r for every column: threads over columns, rows in order.
__device__ void cta_atr(const BatchProb &P) {
    for (int j = threadIdx.x; j < P.n; j += kBT) {
        double s = 0.0;
        for (int i = 0; i < P.m; ++i) s += (double)P.A[(int64_t)i * P.n + j] * P.r[i];
        P.s[j] = s;
    }
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(kBT, 1)
    batch_bpp_kernel(const BatchProb *__restrict__ probs, int32_t count, int32_t *queue,
                     BatchParams prm, BatchOut *out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *diag = reinterpret_cast<T *>(smem_raw);                       // 64 x 65
    T *panel = reinterpret_cast<T *>(smem_raw + sizeof(T) * 64 * 65);  // up to 1024 x (nb+1)
    __shared__ double shd[kBWarps];
    __shared__ int shi[kBWarps];
    __shared__ int sh_p, sh_dec, sh_k, sh_big, sh_ninf;
    __shared__ int64_t sh_N, sh_Nprev;
    __shared__ int sh_pcount, sh_iters;
    const int tid = threadIdx.x;

    for (;;) {
        if (tid == 0) sh_p = atomicAdd(queue, 1);
        __syncthreads();
        const int p = sh_p;
        if (p >= count) return;
        const BatchProb P = probs[p];
        const int n = P.n;
        T *S = static_cast<T *>(P.S);
        T *rhs = static_cast<T *>(P.rhs);
        const T *Gsrc = prm.mixed ? reinterpret_cast<const T *>(P.G) : reinterpret_cast<const T *>(P.Gd);
        int status = TSNNLS_OK, refine = 0;
        double flops = 0.0;  // the same value in every thread
        // F = {}, x = 0, y = -A^T b
        for (int j = tid; j < n; j += kBT) {
            P.x[j] = 0.0;
            P.y[j] = -P.c[j];
            P.inF[j] = 0;
        }
        if (tid == 0) {
            sh_N = INT64_MAX;
            sh_pcount = prm.p_max;
            sh_iters = 0;
        }
        if (prm.mixed && prm.settle) {
            // the settle test's bound c = |A|^T (|A| 1); P.r serves as scratch
            // until the first residual
            const int lane = tid & 31, warp = tid >> 5;
            for (int i = warp; i < P.m; i += kBWarps) {
                double v = 0.0;
                for (int j = lane; j < n; j += 32) v += fabs((double)P.A[(int64_t)i * n + j]);
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) P.r[i] = v;
            }
            __syncthreads();
            for (int j = tid; j < n; j += kBT) {
                double v = 0.0;
                for (int i = 0; i < P.m; ++i) v += fabs((double)P.A[(int64_t)i * n + j]) * P.r[i];
                P.cb[j] = v;
            }
        }
        __syncthreads();
        int k = 0;
        bool open = false;    // the last pivot stopped refining once its signs were settled
        double last_dm = 0.0;  // its last correction
        // refinement of the current pivot's x_F on its factor (MIXED: FP32
        // solves, FP64-accurate residuals; FP64: only the residual for y_G).
        // allow_settle: before the last pivot only the signs matter (Section
        // 3), so the loop may stop once the contraction rho observed between
        // corrections bounds the error left (E = min(0.5, 20 rho) ||dx|| +
        // 1e-15 ||x_F||, c_j E on s_j) below every entry's distance to 0 and
        // +-zero_tol -- the rule of the single-problem path.  Returns 1 then,
        // 0 once converged to rel_tol, -1 on failure (status set).
        auto refine_loop = [&](bool allow_settle, double prev, int steps) -> int {
            const int lds = P.ld;
            bool conv = !prm.mixed || k == 0;
            bool check = false;
            double E = 0.0;
            for (;;) {
                if (prm.mixed) {
                    // in-loop steps need s on F only; a settle check and the
                    // last pass all of it (y_G)
                    cta_residual_ff(P, k, panel, prm.scratch_bytes);
                    cta_atr_ff(P, conv || check, panel, prm.scratch_bytes);
                    flops += 2.0 * P.m * ((double)k + (conv || check ? n : k));
                } else {
                    cta_residual(P, k);
                    cta_atr(P);
                    flops += 2.0 * P.m * ((double)k + n);
                }
                if (conv) return 0;
                if (check) {
                    int unsettled = 0;
                    for (int j = tid; j < n; j += kBT) {
                        const bool f = P.inF[j] != 0;
                        const double v = fabs(f ? P.x[j] : P.s[j]);
                        const double e = f ? E : P.cb[j] * E;
                        if (!(v >= prm.zero_tol + e || v + e < prm.zero_tol)) ++unsettled;
                    }
                    if (block_reduce_isum(unsettled, shi) == 0) return 1;
                    check = false;
                }
                for (int a = tid; a < k; a += kBT) rhs[a] = (T)P.s[P.F[a]];
                __syncthreads();
                cta_chol_solve<T>(S, k, lds, rhs);
                flops += 2.0 * (double)k * k;
                double dm = 0.0, xm = 0.0;
                for (int a = tid; a < k; a += kBT) {
                    const int j = P.F[a];
                    const double dd = (double)rhs[a];
                    const double xn = P.x[j] + dd;
                    P.x[j] = xn;
                    dm = fmax(dm, fabs(dd));
                    xm = fmax(xm, fabs(xn));
                }
                dm = block_reduce_max(dm, shd);
                xm = block_reduce_max(xm, shd);
                ++steps;
                ++refine;
                last_dm = dm;
                if (dm <= prm.rel_tol * xm) conv = true;
                else if (steps > 2 && dm > 0.5 * prev && dm <= 1e-9 * xm) conv = true;
                else if (steps >= prm.max_refine || (steps > 4 && dm > prev)) {
                    if (dm <= 1e-9 * xm) conv = true;
                    else { status = TSNNLS_ENOCONV; return -1; }
                } else if (allow_settle && dm <= 0.1 * prev) {
                    E = fmin(0.5, 20.0 * dm / prev) * dm + 1e-15 * xm;
                    check = true;
                }
                prev = dm;
            }
        };
        for (;;) {
            // zeroing (after the first pivot), infeasible count, largest index
            const bool zero = sh_iters > 0;
            int cnt = 0, largest = -1;
            for (int j = tid; j < n; j += kBT) {
                const uint8_t f = P.inF[j];
                double xv = P.x[j], yv = P.y[j];
                if (zero) {
                    if (f) {
                        if (fabs(xv) < prm.zero_tol) xv = 0.0;
                        yv = 0.0;
                    } else {
                        xv = 0.0;
                        if (fabs(yv) < prm.zero_tol) yv = 0.0;
                    }
                    P.x[j] = xv;
                    P.y[j] = yv;
                }
                if (f ? (xv < 0.0) : (yv < 0.0)) {
                    ++cnt;
                    largest = j;
                }
            }
            const int ninf = block_reduce_isum(cnt, shi);
            const int big = block_reduce_imax(largest, shi);
            if (tid == 0) {
                int d;
                sh_ninf = ninf;
                sh_Nprev = sh_N;
                if (ninf == 0) d = -1;
                else if (sh_iters >= prm.max_iter) d = -2;
                else if (ninf < sh_N) { sh_N = ninf; sh_pcount = prm.p_max; d = 0; }
                else if (sh_pcount > 0) { sh_pcount -= 1; d = 1; }
                else d = 2;
                sh_dec = d;
                sh_big = big;
            }
            __syncthreads();
            const int d = sh_dec;
            if (d == -1 && open) {
                // feasible: that was the last pivot, refined on to rel_tol now;
                // its decisions were settled, so the test passes again
                open = false;
                if (refine_loop(false, last_dm, 0) < 0) break;
                for (int j = tid; j < n; j += kBT) P.y[j] = P.inF[j] ? 0.0 : -P.s[j];
                __syncthreads();
                continue;
            }
            if (d == -1) break;
            if (d == -2) { status = TSNNLS_EMAXITER; break; }
            if (d == 2) {
                if (tid == 0 && TS_IN(sh_big, n)) P.inF[sh_big] ^= 1;
            } else {
                for (int j = tid; j < n; j += kBT)
                    if (P.inF[j] ? (P.x[j] < 0.0) : (P.y[j] < 0.0)) P.inF[j] ^= 1;
            }
            __syncthreads();
            // ascending F list (serial scan by warp 0 over n <= 1024 entries)
            if (tid < 32) {
                int base = 0;
                for (int j0 = 0; j0 < n; j0 += 32) {
                    const int j = j0 + tid;
                    const int v = j < n ? P.inF[j] : 0;
                    const unsigned bal = __ballot_sync(0xffffffffu, v);
                    const int pos = base + __popc(bal & ((1u << tid) - 1u));
                    if (v && TS_IN(pos, n)) P.F[pos] = j;
                    base += __popc(bal);
                }
                if (tid == 0) {
                    sh_k = base;
                    if (P.trace && sh_iters < P.trace_cap) {
                        int64_t *tr = P.trace + 6 * (int64_t)sh_iters;
                        tr[0] = sh_ninf;
                        tr[1] = sh_Nprev;
                        tr[2] = sh_pcount;
                        tr[3] = sh_dec;
                        tr[4] = base;
                        tr[5] = sh_dec == 2 ? sh_big : -1;
                    }
                    sh_iters += 1;
                }
            }
            for (int j = tid; j < n; j += kBT) P.x[j] = 0.0;
            __syncthreads();
            k = sh_k;
            const int lds = P.ld;
            if (k > 0) {
                // gather S = G_FF (lower): F staged in shared memory (the
                // panel area, free until the factorisation), warps over
                // columns, lanes over rows with four loads in flight
                {
                    int32_t *Fs = reinterpret_cast<int32_t *>(panel);
                    for (int a = tid; a < k; a += kBT) Fs[a] = P.F[a];
                    __syncthreads();
                    const int lane = tid & 31;
                    for (int bcol = tid >> 5; bcol < k; bcol += kBWarps) {
                        const T *gc = Gsrc + (int64_t)Fs[bcol] * P.ld;
                        T *sc = S + (int64_t)bcol * lds;
                        for (int a0 = bcol; a0 < k; a0 += 128) {
                            T v[4];
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                const int a = a0 + lane + 32 * u;
                                v[u] = a < k ? gc[Fs[a]] : T(0);
                            }
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                const int a = a0 + lane + 32 * u;
                                if (a < k) sc[a] = v[u];
                            }
                        }
                    }
                    __syncthreads();
                }
                const int info = cta_cholesky<T>(S, k, lds, P.nb, panel, diag, shi);
                if (info) { status = TSNNLS_ENOTPD; break; }
                for (int a = tid; a < k; a += kBT) rhs[a] = (T)P.c[P.F[a]];
                __syncthreads();
                cta_chol_solve<T>(S, k, lds, rhs);
                flops += (double)k * k * k / 3.0 + 2.0 * (double)k * k;
                for (int a = tid; a < k; a += kBT) P.x[P.F[a]] = (double)rhs[a];
                __syncthreads();
                ++refine;
            }
            // the first solve's correction is x_F itself
            double x0 = 0.0;
            for (int a = tid; a < k; a += kBT) x0 = fmax(x0, fabs(P.x[P.F[a]]));
            x0 = block_reduce_max(x0, shd);
            const int rr = refine_loop(prm.mixed && prm.settle, x0, 1);
            if (rr < 0) break;
            open = rr == 1;
            // Eq. 5: y_G = -s_G
            for (int j = tid; j < n; j += kBT) P.y[j] = P.inF[j] ? 0.0 : -P.s[j];
            __syncthreads();
        }
        if (tid == 0) {
            out[p].status = status;
            out[p].iters = sh_iters;
            out[p].refine = refine;
            out[p].nF = k;
            out[p].flops = flops;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// host side

// Panel width per problem-size bucket (n <= 64, 128, 256, 512, 1024), for
// MIXED (row 0) and FP64 (row 1).  tsnnls_batch_autotune overwrites it.
int g_batch_nb_table[2][5] = {{32, 32, 32, 32, 32}, {16, 16, 16, 16, 16}};

constexpr int kMaxNbMixed = 48;  // panel of 1024 x 49 floats fits shared memory
constexpr int kMaxNbFp64 = 16;   // 1024 x 17 doubles

static int size_bucket(int n) { return n <= 64 ? 0 : n <= 128 ? 1 : n <= 256 ? 2 : n <= 512 ? 3 : 4; }

static int pick_nb(int n, bool mixed) {
    const int nb = g_batch_nb_table[mixed ? 0 : 1][size_bucket(n)];
    return std::max(4, std::min(nb, mixed ? kMaxNbMixed : kMaxNbFp64));
}

size_t batch_smem_bytes(bool mixed, int max_nb) {
    const size_t t = mixed ? sizeof(float) : sizeof(double);
    const int pitch = std::max(max_nb + 1, mixed && max_nb >= 32 ? 36 : 0);
    return t * 64 * 65 + t * (size_t)kMaxPanelRows * pitch;
}

// The last call's graph and arena on a lane.  The graph's kernels read
// every per-problem pointer from the descriptor array in the arena, so a
// call with the same shape (count, precision, parameters, sizes and panel
// widths in queue order, trace capacity) only rewrites the descriptors and
// replays the graph; any other shape rebuilds both.
struct BatchGraphCache {
    std::vector<int64_t> key;
    char *arena = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;

    void release(cudaStream_t s) {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (arena) {
            cudaFreeAsync(arena, s);
            cudaStreamSynchronize(s);
        }
        key.clear();
        arena = nullptr;
        graph = nullptr;
        exec = nullptr;
    }
};

void batch_cache_release(Lane &l) {
    auto *c = static_cast<BatchGraphCache *>(l.batch_cache);
    if (!c) return;
    c->release(l.stream);
    delete c;
    l.batch_cache = nullptr;
}

int run_batch_dense(Context &ctx, Lane &lane, int count, const int32_t *m, const int32_t *n,
                    const float *const *a, const double *const *b, double *const *x,
                    const tsnnls_opts &o, int32_t *status_out, tsnnls_info *info,
                    const int *nb_override, int64_t *const *trace, int64_t trace_cap) {
    NvtxSolve range(lane, "tsnnls_solve_batch_dense");
    const bool mixed = o.precision == TSNNLS_MIXED;
    const size_t tsz = mixed ? sizeof(float) : sizeof(double);
    cudaStream_t s = lane.stream;
    // largest first
    std::vector<int> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int i, int j) { return n[i] > n[j]; });
    // arena layout
    std::vector<size_t> off(count);
    size_t total = 0;
    auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
    int max_nb = 0;
    std::vector<BatchProb> hp(count);
    for (int q = 0; q < count; ++q) {
        const int i = order[q];
        const int ld = (int)round_up(n[i], 4);
        size_t bytes = 0;
        bytes += up(sizeof(float) * (size_t)n[i] * ld);          // G (FP32)
        bytes += up(tsz * (size_t)n[i] * ld);                     // S
        if (!mixed) bytes += up(sizeof(double) * (size_t)n[i] * ld);  // Gd
        bytes += 3 * up(sizeof(double) * n[i]);                   // c, y, s
        if (mixed) bytes += up(sizeof(double) * n[i]);            // cb
        bytes += up(sizeof(double) * m[i]);                       // r
        bytes += up(tsz * n[i]);                                  // rhs
        bytes += up(sizeof(int32_t) * n[i]) + up(n[i]);           // F, inF
        if (trace) bytes += up(sizeof(int64_t) * 6 * (size_t)trace_cap);  // pivot trace
        off[q] = total;
        total += bytes;
        BatchProb &P = hp[q];
        P.m = m[i];
        P.n = n[i];
        P.ld = ld;
        P.nb = nb_override ? std::max(4, std::min(nb_override[i], mixed ? kMaxNbMixed : kMaxNbFp64))
                           : pick_nb(n[i], mixed);
        max_nb = std::max(max_nb, P.nb);
        P.A = a[i];
        P.b = b[i];
        P.x = x[i];
    }
    const size_t desc_bytes = up(sizeof(BatchProb) * count);
    const size_t out_bytes = up(sizeof(BatchOut) * count);
    std::vector<GramItem> items;
    for (int q = 0; q < count; ++q) {
        const int t = (hp[q].n + 63) / 64;
        for (int I = 0; I < t; ++I)
            for (int J = 0; J <= I; ++J) items.push_back({q, I, J});
    }
    const size_t item_bytes = up(sizeof(GramItem) * items.size());
    BatchParams prm{o.zero_tol, o.rel_tol, o.p_max,
                    o.max_iter > 0 ? o.max_iter : 0, o.max_refine, mixed ? 1 : 0,
                    (int32_t)(batch_smem_bytes(mixed, max_nb) - (mixed ? sizeof(float) : sizeof(double)) * 64 * 65),
                    mixed && o.full_refine == 0 ? 1 : 0};
    if (prm.max_iter == 0) {
        int nmax = 0;
        for (int q = 0; q < count; ++q) nmax = std::max(nmax, hp[q].n);
        prm.max_iter = 10 * nmax + 100;
    }
    // the shape the graph is built for (parameters are kernel arguments)
    std::vector<int64_t> key = {mixed ? 1 : 0, count, trace ? trace_cap : 0, prm.p_max, prm.max_iter,
                                prm.max_refine, prm.scratch_bytes, prm.settle};
    int64_t tb[2];
    std::memcpy(&tb[0], &prm.zero_tol, 8);
    std::memcpy(&tb[1], &prm.rel_tol, 8);
    key.push_back(tb[0]);
    key.push_back(tb[1]);
    for (int q = 0; q < count; ++q) {
        key.push_back(hp[q].m);
        key.push_back(hp[q].n);
        key.push_back(hp[q].nb);
    }
    auto *cache = static_cast<BatchGraphCache *>(lane.batch_cache);
    if (!cache) {
        cache = new (std::nothrow) BatchGraphCache;
        if (!cache) return TSNNLS_ENOMEM;
        lane.batch_cache = cache;
    }
    const bool hit = cache->exec != nullptr && cache->arena != nullptr && cache->key == key;
    cudaError_t e = cudaSuccess;
    if (!hit) {
        cache->release(s);
        e = cudaMallocAsync(reinterpret_cast<void **>(&cache->arena),
                            total + desc_bytes + out_bytes + item_bytes + 256, s);
        if (e != cudaSuccess) {
            cache->arena = nullptr;
            return status_from_cuda(e);
        }
    }
    char *arena = cache->arena;
    for (int q = 0; q < count; ++q) {
        char *pbase = arena + off[q];
        BatchProb &P = hp[q];
        auto take = [&](size_t sz) { char *r = pbase; pbase += up(sz); return r; };
        P.G = reinterpret_cast<float *>(take(sizeof(float) * (size_t)P.n * P.ld));
        P.S = take(tsz * (size_t)P.n * P.ld);
        P.Gd = mixed ? nullptr : reinterpret_cast<double *>(take(sizeof(double) * (size_t)P.n * P.ld));
        P.c = reinterpret_cast<double *>(take(sizeof(double) * P.n));
        P.y = reinterpret_cast<double *>(take(sizeof(double) * P.n));
        P.s = reinterpret_cast<double *>(take(sizeof(double) * P.n));
        P.cb = mixed ? reinterpret_cast<double *>(take(sizeof(double) * P.n)) : nullptr;
        P.r = reinterpret_cast<double *>(take(sizeof(double) * P.m));
        P.rhs = take(tsz * P.n);
        P.F = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * P.n));
        P.inF = reinterpret_cast<uint8_t *>(take(P.n));
        P.trace = trace ? reinterpret_cast<int64_t *>(take(sizeof(int64_t) * 6 * (size_t)trace_cap)) : nullptr;
        P.trace_cap = trace ? (int32_t)trace_cap : 0;
    }
    BatchProb *d_probs = reinterpret_cast<BatchProb *>(arena + total);
    BatchOut *d_out = reinterpret_cast<BatchOut *>(arena + total + desc_bytes);
    GramItem *d_items = reinterpret_cast<GramItem *>(arena + total + desc_bytes + out_bytes);
    int32_t *d_queue = reinterpret_cast<int32_t *>(arena + total + desc_bytes + out_bytes + item_bytes);
    std::vector<BatchOut> hout(count);
    int status = TSNNLS_OK;
    const size_t smem = batch_smem_bytes(mixed, max_nb);
    const int64_t launch0 = launches_so_far();
    do {
        e = cudaMemcpyAsync(d_probs, hp.data(), sizeof(BatchProb) * count, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) break;
        if (!hit && !items.empty())
            e = cudaMemcpyAsync(d_items, items.data(), sizeof(GramItem) * items.size(),
                                cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) break;
        if (trace)  // rows past a problem's last pivot read -1 (a real row has a count >= 1)
            for (int q = 0; q < count && e == cudaSuccess; ++q)
                e = cudaMemsetAsync(hp[q].trace, 0xFF, sizeof(int64_t) * 6 * (size_t)trace_cap, s);
        if (e != cudaSuccess) break;
        if (mixed)
            e = cudaFuncSetAttribute(batch_bpp_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        else
            e = cudaFuncSetAttribute(batch_bpp_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) break;
        // precompute + persistent kernel captured into one graph on the first
        // call of this shape, replayed as it stands by the next ones
        if (!hit) {
            e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) break;
            e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) break;
            cudaMemsetAsync(d_queue, 0, sizeof(int32_t), s);
            const int gitems = (int)items.size();
            const int ggrid = std::max(1, std::min(gitems, num_sms() * 8));
            if (mixed) batch_gram_tc_kernel<<<ggrid, 256, 0, s>>>(d_probs, d_items, gitems);
            else batch_gram64_kernel<<<ggrid, 256, 0, s>>>(d_probs, d_items, gitems);
            batch_atb_kernel<<<std::min(count, num_sms() * 8), 256, 0, s>>>(d_probs, count);
            const int pgrid = std::min(count, num_sms());
            if (mixed)
                batch_bpp_kernel<float><<<pgrid, kBT, smem, s>>>(d_probs, count, d_queue, prm, d_out);
            else
                batch_bpp_kernel<double><<<pgrid, kBT, smem, s>>>(d_probs, count, d_queue, prm, d_out);
            e = cudaStreamEndCapture(s, &cache->graph);
            if (e != cudaSuccess) break;
            e = cudaGraphInstantiate(&cache->exec, cache->graph, 0);
            if (e != cudaSuccess) break;
            cache->key = key;
        }
        note_launches(3);  // the graph's three kernels
        e = cudaEventRecord(lane.ev0, s);
        if (e != cudaSuccess) break;
        e = cudaGraphLaunch(cache->exec, s);
        if (e != cudaSuccess) break;
        e = cudaEventRecord(lane.ev1, s);
        if (e != cudaSuccess) break;
        e = cudaMemcpyAsync(hout.data(), d_out, sizeof(BatchOut) * count, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) break;
        if (trace) {
            for (int q = 0; q < count && e == cudaSuccess; ++q)
                if (trace[order[q]])
                    e = cudaMemcpyAsync(trace[order[q]], hp[q].trace, sizeof(int64_t) * 6 * (size_t)trace_cap,
                                        cudaMemcpyDeviceToHost, s);
            if (e != cudaSuccess) break;
        }
        e = cudaStreamSynchronize(s);
    } while (0);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(s);
        status = status_from_cuda(e);
    }
    float ms = 0.f;
    if (status == TSNNLS_OK) cudaEventElapsedTime(&ms, lane.ev0, lane.ev1);
    if (status != TSNNLS_OK) {
        // a failed capture or launch: nothing of this call is kept
        cudaGraph_t open_capture = nullptr;  // a capture left open ends here (an error otherwise, ignored)
        if (cudaStreamEndCapture(s, &open_capture) == cudaSuccess && open_capture) cudaGraphDestroy(open_capture);
        cudaGetLastError();
        cache->release(s);
    }
    if (check_collect(nullptr, 0) > 0 && status == TSNNLS_OK) status = TSNNLS_EBOUNDS;
    int32_t iters = 0, refine = 0;
    double flops = 0.0, bytes = 0.0;
    if (status == TSNNLS_OK) {
        for (int q = 0; q < count; ++q) {
            const int i = order[q];
            if (status_out) status_out[i] = hout[q].status;
            if (hout[q].status != TSNNLS_OK && status == TSNNLS_OK) status = hout[q].status;
            iters += hout[q].iters;
            refine += hout[q].refine;
            // precompute: lower A^T A and A^T b; then the pivot loop
            const double mq = hp[q].m, nq = hp[q].n;
            flops += mq * nq * (nq + 1.0) + 2.0 * mq * nq + hout[q].flops;
            bytes += 4.0 * mq * nq + (mixed ? 4.0 : 8.0) * nq * (nq + 1.0) / 2.0 + 8.0 * (mq + 2.0 * nq);
        }
        // the whole graph (precompute + persistent kernel) is accounted as
        // one FACTOR phase of the profiling API
        if (lane.prof) {
            tsnnls_phase_stat &ps = lane.stats[TSNNLS_PHASE_FACTOR];
            ps.ms += ms;
            ps.launches += launches_so_far() - launch0;
            ps.flops += flops;
            ps.bytes += bytes;
        }
    }
    if (info) {
        std::memset(info, 0, sizeof(*info));
        info->status = status;
        info->iters = iters;
        info->refine_steps = refine;
        info->time_ms = ms;
        info->path_used = TSNNLS_PATH_FACTOR;
        info->precision_used = o.precision;
        info->kernel_launches = launches_so_far() - launch0;
    }
    return status;
}

}  // namespace tsnnls

namespace tsnnls {

// Autotuner: for every size bucket, time the batched solve of a synthetic
// batch (FP32 N(0,1)-like entries from a counter hash, m = 1.5 n, b = A 1 +
// perturbation) with each candidate panel width and keep the fastest.
__global__ void autotune_fill_kernel(float *A, double *b, int m, int n, uint32_t seed) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)m * n;
         e += (int64_t)gridDim.x * blockDim.x) {
        uint32_t h = (uint32_t)e * 2654435761u ^ seed;
        h ^= h >> 16; h *= 0x7feb352du; h ^= h >> 15; h *= 0x846ca68bu; h ^= h >> 16;
        uint32_t g = h * 747796405u + 2891336453u;
        g ^= g >> 13; g *= 0x5bd1e995u; g ^= g >> 15;
        // sum of two uniforms, centred: a cheap bell-shaped value in (-1, 1)
        A[e] = ((h >> 8) * (1.0f / 16777216.0f)) + ((g >> 8) * (1.0f / 16777216.0f)) - 1.0f;
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
        b[i] = (double)((i * 37) % 11) * 0.1 - 0.3;
}

int batch_autotune(Context &ctx, Lane &lane, bool mixed, int per_bucket) {
    const int sizes[5] = {48, 96, 192, 384, 768};
    const int cands_mixed[] = {8, 16, 32, 48};
    const int cands_fp64[] = {8, 16};
    const int *cands = mixed ? cands_mixed : cands_fp64;
    const int ncand = mixed ? 4 : 2;
    tsnnls_opts o;
    tsnnls_opts_default(&o);
    o.precision = mixed ? TSNNLS_MIXED : TSNNLS_FP64;
    cudaStream_t s = lane.stream;
    for (int bkt = 0; bkt < 5; ++bkt) {
        const int n = sizes[bkt], m = (3 * n) / 2;
        const int cnt = std::max(4, std::min(per_bucket, (int)(4e8 / ((double)n * n * n) + 4)));
        float *A = nullptr;
        double *bx = nullptr;
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&A), sizeof(float) * (size_t)m * n * cnt, s);
        if (e == cudaSuccess)
            e = cudaMallocAsync(reinterpret_cast<void **>(&bx), sizeof(double) * (size_t)(m + n) * cnt, s);
        if (e != cudaSuccess) return status_from_cuda(e);
        std::vector<int32_t> mv(cnt, m), nv(cnt, n), nbv(cnt);
        std::vector<const float *> av(cnt);
        std::vector<const double *> bv(cnt);
        std::vector<double *> xv(cnt);
        for (int i = 0; i < cnt; ++i) {
            av[i] = A + (size_t)m * n * i;
            bv[i] = bx + (size_t)(m + n) * i;
            xv[i] = bx + (size_t)(m + n) * i + m;
            autotune_fill_kernel<<<64, 256, 0, s>>>(A + (size_t)m * n * i, bx + (size_t)(m + n) * i, m,
                                                     n, 0x9e3779b9u * (uint32_t)(i + 1) + bkt);
        }
        float best_ms = 1e30f;
        int best = cands[0];
        for (int c = 0; c < ncand; ++c) {
            std::fill(nbv.begin(), nbv.end(), cands[c]);
            float total = 0.f;
            bool ok = true;
            for (int rep = 0; rep < 2 && ok; ++rep) {
                tsnnls_info info;
                int st = run_batch_dense(ctx, lane, cnt, mv.data(), nv.data(), av.data(), bv.data(),
                                         xv.data(), o, nullptr, &info, nbv.data(), nullptr, 0);
                ok = st == TSNNLS_OK;
                if (rep == 1) total = (float)info.time_ms;
            }
            if (ok && total < best_ms) {
                best_ms = total;
                best = cands[c];
            }
        }
        g_batch_nb_table[mixed ? 0 : 1][bkt] = best;
        cudaFreeAsync(A, s);
        cudaFreeAsync(bx, s);
        cudaStreamSynchronize(s);
    }
    return TSNNLS_OK;
}

}  // namespace tsnnls

TSNNLS_CHECK_UNIT("batch")
