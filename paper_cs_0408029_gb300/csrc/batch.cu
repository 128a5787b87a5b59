// Batched dense solves: many small or uneven NNLS problems at once.
//
// Each problem i has a dense FP32 A_i (m_i x n_i, row-major), FP64 b_i and x_i.
// The work is two kernels, captured once into a CUDA graph and replayed:
//   1. batched precompute (Section 3): G_i = A_i^T A_i (lower tiles, FP32
//      accumulate) and c_i = A_i^T b_i (FP64), over one flat list of
//      (problem, tile) work items;
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
#include <numeric>
#include <vector>

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
    void *rhs;       // n (factor type)
    int32_t *F;
    uint8_t *inF;
    int32_t m, n, ld, nb;
};

struct BatchOut {
    int32_t status, iters, refine, nF;
    double flops;  // algorithmic flops of the pivot loop (factors, solves, residuals)
};

struct BatchParams {
    double zero_tol, rel_tol;
    int32_t p_max, max_iter, max_refine, mixed;
    int32_t scratch_bytes;  // bytes of the panel area free outside the factorisation
};

// ---------------------------------------------------------------------------
// 1. precompute: G = A^T A lower 64 x 64 tiles, FP32; c = A^T b in FP64.

struct GramItem {
    int32_t prob, I, J;
};

__global__ void __launch_bounds__(256)
    batch_gram_kernel(const BatchProb *__restrict__ probs, const GramItem *__restrict__ items,
                      int32_t nitems) {
    __shared__ float As[16][68];
    __shared__ float Bs[16][68];
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const GramItem w = items[it];
        const BatchProb P = probs[w.prob];
        const int n = P.n, m = P.m;
        const int r0 = w.I * 64, c0 = w.J * 64;
        const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
        float acc[4][4] = {};
        for (int k0 = 0; k0 < m; k0 += 16) {
            for (int e = threadIdx.x; e < 16 * 64; e += 256) {
                const int kk = e / 64, i = e % 64;
                const int row = k0 + kk;
                As[kk][i] = (row < m && r0 + i < n) ? P.A[(int64_t)row * n + r0 + i] : 0.f;
                Bs[kk][i] = (row < m && c0 + i < n) ? P.A[(int64_t)row * n + c0 + i] : 0.f;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) {
                float a[4], bb[4];
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
                if (i < n && j < n && i >= j) P.G[i + (int64_t)j * P.ld] = acc[q][t];
            }
        }
    }
}

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

template <typename T>
struct BSmem {
    // panel rows staged for the trailing update: P[row][l], padded
    static constexpr size_t panel_bytes(int nb) { return sizeof(T) * (size_t)kMaxPanelRows * (nb + 1); }
};

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

// In-CTA blocked right-looking Cholesky of the k x k lower matrix S (lds),
// panel width nb <= 64.  Returns 0 or 1 + the failing column.
template <typename T>
__device__ int cta_cholesky(T *S, int k, int lds, int nb, T *panel, T *diag, int *sh_int) {
    const int tid = threadIdx.x;
    int info = 0;
    for (int K = 0; K < k; K += nb) {
        const int kb = min(nb, k - K);
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
        // panel: X L_KK^T = B for rows below, one thread per row, into smem
        const int R0 = K + kb, nr = k - R0;
        // (the row's kb entries are loaded into the panel first, all in flight)
        for (int r = tid; r < nr; r += kBT) {
            for (int c = 0; c < kb; ++c) panel[r * (nb + 1) + c] = S[(R0 + r) + (int64_t)(K + c) * lds];
            for (int c = 0; c < kb; ++c) {
                T s = panel[r * (nb + 1) + c];
                for (int l = 0; l < c; ++l) s -= panel[r * (nb + 1) + l] * diag[l * 65 + c];
                s /= diag[c * 65 + c];
                panel[r * (nb + 1) + c] = s;
            }
            for (int c = 0; c < kb; ++c) S[(R0 + r) + (int64_t)(K + c) * lds] = panel[r * (nb + 1) + c];
        }
        __syncthreads();
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
                        av[a] = rr < nr ? panel[rr * (nb + 1) + l] : T(0);
                    }
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const int cc = cj + tx + 16 * b;
                        bv[b] = cc < nr ? panel[cc * (nb + 1) + l] : T(0);
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

// rhs <- (L L^T)^{-1} rhs inside one CTA: 32-row blocks, the diagonal block
// solved by warp 0 with shuffles, the rest of the column updated by all threads.
template <typename T>
__device__ void cta_chol_solve(const T *L, int k, int lds, T *rhs) {
    const int tid = threadIdx.x, lane = tid & 31;
    for (int B0 = 0; B0 < k; B0 += 32) {  // L z = rhs
        const int nb = min(32, k - B0);
        if (tid < 32) {
            // lane = row of the 32 x 32 diagonal block, loaded before the
            // serial steps (l[c] = L(B0 + lane, B0 + c)); d = its diagonal entry
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
        __syncthreads();
        for (int r = B0 + nb + tid; r < k; r += kBT) {
            T lv[32];
#pragma unroll
            for (int c = 0; c < 32; ++c) lv[c] = c < nb ? L[r + (int64_t)(B0 + c) * lds] : T(0);
            T s = T(0);
#pragma unroll
            for (int c = 0; c < 32; ++c) s += lv[c] * rhs[B0 + c];
            rhs[r] -= s;
        }
        __syncthreads();
    }
    const int nblk = (k + 31) / 32;
    for (int bi = nblk - 1; bi >= 0; --bi) {  // L^T w = z
        const int B0 = bi * 32, nb = min(32, k - B0);
        if (tid < 32) {
            // lane = column of the block: lt[c] = L(B0 + c, B0 + lane)
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
        __syncthreads();
        // rows above: rhs[r] -= sum_c L(B0 + c, r) w_c for r < B0 (L^T row r)
        for (int r = tid; r < B0; r += kBT) {
            T lv[32];
#pragma unroll
            for (int c = 0; c < 32; ++c) lv[c] = c < nb ? L[(B0 + c) + (int64_t)r * lds] : T(0);
            T s = T(0);
#pragma unroll
            for (int c = 0; c < 32; ++c) s += lv[c] * rhs[B0 + c];
            rhs[r] -= s;
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

// r = b - A_F x_F with the double-float products above; x_F (split) and F
// are staged in shared memory (the factorisation's panel area, free here)
// when they fit, and r is stored split into P.r.
__device__ void cta_residual_ff(const BatchProb &P, int k, void *scr, int scr_bytes) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool staged = 12 * k <= scr_bytes;
    float2 *xs = staged ? static_cast<float2 *>(scr) : reinterpret_cast<float2 *>(P.y);
    const int32_t *F = P.F;
    if (staged) {
        int32_t *Fs = reinterpret_cast<int32_t *>(static_cast<float2 *>(scr) + k);
        for (int a = threadIdx.x; a < k; a += kBT) {
            const int j = P.F[a];
            Fs[a] = j;
            xs[a] = ff_split(P.x[j]);
        }
        F = Fs;
    } else {
        for (int a = threadIdx.x; a < k; a += kBT) xs[a] = ff_split(P.x[P.F[a]]);
    }
    __syncthreads();
    float2 *rs = reinterpret_cast<float2 *>(P.r);
    for (int i = warp; i < P.m; i += kBWarps) {
        float h = 0.f, l = 0.f, h2 = 0.f, l2 = 0.f;
        const float *row = P.A + (int64_t)i * P.n;
        int a = lane;
        for (; a + 32 < k; a += 64) {  // two gathers in flight per lane
            const float2 v0 = xs[a], v1 = xs[a + 32];
            const float a0 = row[F[a]], a1 = row[F[a + 32]];
            ff_acc(h, l, a0, v0.x, v0.y);
            ff_acc(h2, l2, a1, v1.x, v1.y);
        }
        if (a < k) ff_acc(h, l, row[F[a]], xs[a].x, xs[a].y);
        ff_add(h, l, h2, l2);
        for (int o = 16; o > 0; o >>= 1) {
            const float hh = __shfl_xor_sync(0xffffffffu, h, o), ll = __shfl_xor_sync(0xffffffffu, l, o);
            ff_add(h, l, hh, ll);
        }
        if (lane == 0) rs[i] = ff_split(P.b[i] - ((double)h + (double)l));
    }
    __syncthreads();
}

// s_j = (A^T r)_j with r split in P.r (staged in shared memory when it
// fits); only the F columns unless all_cols.
__device__ void cta_atr_ff(const BatchProb &P, bool all_cols, void *scr, int scr_bytes) {
    const bool staged = 8 * P.m <= scr_bytes;
    const float2 *rs = reinterpret_cast<const float2 *>(P.r);
    if (staged) {
        float2 *rsm = static_cast<float2 *>(scr);
        for (int i = threadIdx.x; i < P.m; i += kBT) rsm[i] = rs[i];
        __syncthreads();
        rs = rsm;
    }
    for (int j = threadIdx.x; j < P.n; j += kBT) {
        if (!all_cols && !P.inF[j]) continue;
        float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;  // two chains for ILP
        int i = 0;
        for (; i + 1 < P.m; i += 2) {
            const float2 v0 = rs[i], v1 = rs[i + 1];
            ff_acc(h0, l0, P.A[(int64_t)i * P.n + j], v0.x, v0.y);
            ff_acc(h1, l1, P.A[(int64_t)(i + 1) * P.n + j], v1.x, v1.y);
        }
        if (i < P.m) ff_acc(h0, l0, P.A[(int64_t)i * P.n + j], rs[i].x, rs[i].y);
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
    __shared__ int sh_p, sh_dec, sh_k, sh_big;
    __shared__ int64_t sh_N;
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
        __syncthreads();
        int k = 0;
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
            if (d == -1) break;
            if (d == -2) { status = TSNNLS_EMAXITER; break; }
            if (d == 2) {
                if (tid == 0) P.inF[sh_big] ^= 1;
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
                    if (v) P.F[base + __popc(bal & ((1u << tid) - 1u))] = j;
                    base += __popc(bal);
                }
                if (tid == 0) {
                    sh_k = base;
                    sh_iters += 1;
                }
            }
            for (int j = tid; j < n; j += kBT) P.x[j] = 0.0;
            __syncthreads();
            k = sh_k;
            const int lds = P.ld;
            if (k > 0) {
                // gather S = G_FF (lower)
                for (int e = tid; e < k * k; e += kBT) {
                    const int bcol = e / k, a = e % k;
                    if (a >= bcol) S[a + (int64_t)bcol * lds] = Gsrc[P.F[a] + (int64_t)P.F[bcol] * P.ld];
                }
                __syncthreads();
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
            double prev = 0.0;
            bool conv = !prm.mixed || k == 0;
            int steps = 1;
            for (;;) {
                if (prm.mixed) {
                    // in-loop steps need s on F only; the last pass all of it (y_G)
                    cta_residual_ff(P, k, panel, prm.scratch_bytes);
                    cta_atr_ff(P, conv, panel, prm.scratch_bytes);
                    flops += 2.0 * P.m * ((double)k + (conv ? n : k));
                } else {
                    cta_residual(P, k);
                    cta_atr(P);
                    flops += 2.0 * P.m * ((double)k + n);
                }
                if (conv) break;
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
                if (dm <= prm.rel_tol * xm) conv = true;
                else if (steps > 2 && dm > 0.5 * prev && dm <= 1e-9 * xm) conv = true;
                else if (steps >= prm.max_refine || (steps > 4 && dm > prev)) {
                    if (dm <= 1e-9 * xm) conv = true;
                    else { status = TSNNLS_ENOCONV; break; }
                }
                prev = dm;
            }
            if (status != TSNNLS_OK) break;
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
    return t * 64 * 65 + t * (size_t)kMaxPanelRows * (max_nb + 1);
}

int run_batch_dense(Context &ctx, Lane &lane, int count, const int32_t *m, const int32_t *n,
                    const float *const *a, const double *const *b, double *const *x,
                    const tsnnls_opts &o, int32_t *status_out, tsnnls_info *info,
                    const int *nb_override) {
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
        bytes += up(sizeof(double) * m[i]);                       // r
        bytes += up(tsz * n[i]);                                  // rhs
        bytes += up(sizeof(int32_t) * n[i]) + up(n[i]);           // F, inF
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
    char *arena = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&arena),
                                    total + desc_bytes + out_bytes + item_bytes + 256, s);
    if (e != cudaSuccess) return status_from_cuda(e);
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
        P.r = reinterpret_cast<double *>(take(sizeof(double) * P.m));
        P.rhs = take(tsz * P.n);
        P.F = reinterpret_cast<int32_t *>(take(sizeof(int32_t) * P.n));
        P.inF = reinterpret_cast<uint8_t *>(take(P.n));
    }
    BatchProb *d_probs = reinterpret_cast<BatchProb *>(arena + total);
    BatchOut *d_out = reinterpret_cast<BatchOut *>(arena + total + desc_bytes);
    GramItem *d_items = reinterpret_cast<GramItem *>(arena + total + desc_bytes + out_bytes);
    int32_t *d_queue = reinterpret_cast<int32_t *>(arena + total + desc_bytes + out_bytes + item_bytes);
    std::vector<BatchOut> hout(count);
    BatchParams prm{o.zero_tol, o.rel_tol, o.p_max,
                    o.max_iter > 0 ? o.max_iter : 0, o.max_refine, mixed ? 1 : 0,
                    (int32_t)((mixed ? sizeof(float) : sizeof(double)) * (size_t)kMaxPanelRows * (max_nb + 1))};
    int status = TSNNLS_OK;
    const size_t smem = batch_smem_bytes(mixed, max_nb);
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const int64_t launch0 = launches_so_far();
    do {
        e = cudaMemcpyAsync(d_probs, hp.data(), sizeof(BatchProb) * count, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) break;
        if (!items.empty())
            e = cudaMemcpyAsync(d_items, items.data(), sizeof(GramItem) * items.size(),
                                cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) break;
        if (prm.max_iter == 0) {
            int nmax = 0;
            for (int q = 0; q < count; ++q) nmax = std::max(nmax, hp[q].n);
            prm.max_iter = 10 * nmax + 100;
        }
        if (mixed)
            e = cudaFuncSetAttribute(batch_bpp_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        else
            e = cudaFuncSetAttribute(batch_bpp_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) break;
        // capture precompute + persistent kernel into one graph and replay it
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) break;
        e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) break;
        cudaMemsetAsync(d_queue, 0, sizeof(int32_t), s);
        const int gitems = (int)items.size();
        const int ggrid = std::max(1, std::min(gitems, num_sms() * 8));
        if (mixed) batch_gram_kernel<<<ggrid, 256, 0, s>>>(d_probs, d_items, gitems);
        else batch_gram64_kernel<<<ggrid, 256, 0, s>>>(d_probs, d_items, gitems);
        note_launches(1);
        batch_atb_kernel<<<std::min(count, num_sms() * 8), 256, 0, s>>>(d_probs, count);
        note_launches(1);
        const int pgrid = std::min(count, num_sms());
        if (mixed)
            batch_bpp_kernel<float><<<pgrid, kBT, smem, s>>>(d_probs, count, d_queue, prm, d_out);
        else
            batch_bpp_kernel<double><<<pgrid, kBT, smem, s>>>(d_probs, count, d_queue, prm, d_out);
        note_launches(1);
        e = cudaStreamEndCapture(s, &graph);
        if (e != cudaSuccess) break;
        e = cudaGraphInstantiate(&exec, graph, 0);
        if (e != cudaSuccess) break;
        e = cudaEventRecord(lane.ev0, s);
        if (e != cudaSuccess) break;
        e = cudaGraphLaunch(exec, s);
        if (e != cudaSuccess) break;
        e = cudaEventRecord(lane.ev1, s);
        if (e != cudaSuccess) break;
        e = cudaMemcpyAsync(hout.data(), d_out, sizeof(BatchOut) * count, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) break;
        e = cudaStreamSynchronize(s);
    } while (0);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(s);
        status = status_from_cuda(e);
    }
    float ms = 0.f;
    if (status == TSNNLS_OK) cudaEventElapsedTime(&ms, lane.ev0, lane.ev1);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    cudaFreeAsync(arena, s);
    cudaStreamSynchronize(s);
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
                                         xv.data(), o, nullptr, &info, nbv.data());
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

