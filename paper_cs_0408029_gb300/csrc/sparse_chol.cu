// Supernodal sparse Cholesky of the cached normal equations on the GPU
// (Section 3: TAUCS factors A^T A as a sparse matrix when it is sparse).
// The structure comes from sparse_sym.cpp, analysed once per problem; every
// pivot factors
//     G' = P (A^T A)_{FF} P^T  (+ the identity on the variables in G)
// so one structure serves every F: a variable outside F keeps a unit column,
// and its entry of every solve is 0.
//
// Factor (multifrontal): one persistent kernel, one CTA per SM.  CTAs take
// supernodes by ticket in order of height in the supernodal tree (leaves
// first); a supernode waits (bounded) until its children are done -- CTAs
// holding smaller tickets, so running or finished.  It then
//   - clears its panel (rows x width) and its update matrix (rows below
//     squared), assembles the entries of G' in its columns, and adds its
//     children's update matrices, child by child in ascending order, through
//     the precomputed positions of their rows among its own;
//   - factors and inverts its diagonal block in shared memory with the dense
//     block code of the blocked factorisation (dense_block.cuh) and forms
//     the rows below as X = B W^T, 32 rows at a time;
//   - subtracts X X^T from its update matrix and publishes a done flag.
// Solves: forward in the factor's order (a supernode adds its children's
// update vectors, applies W, and leaves the update vector of its rows below
// for its parent), backward by depth, roots first (it gathers the solved
// entries of its rows below from the supernodes above, then applies W^T).  Every sum
// runs in a fixed order, so results are reproducible.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cuda/atomic>
#include <vector>

#include "check.cuh"
#include "common.cuh"
#include "dense_block.cuh"
#include "sparse_sym.h"
#include "sparse_chol.h"

namespace tsnnls {

namespace {

__device__ __forceinline__ int sp_flag_load(const int32_t *p) {
    cuda::atomic_ref<const int32_t, cuda::thread_scope_device> a(*p);
    return a.load(cuda::memory_order_acquire);
}
__device__ __forceinline__ void sp_flag_store(int32_t *p, int v) {
    cuda::atomic_ref<int32_t, cuda::thread_scope_device> a(*p);
    a.store(v, cuda::memory_order_release);
}

// Thread 0 waits until flags[list[b..e)] are all set (bounded); the CTA
// learns whether it may go on.
__device__ bool sp_wait_all(const SpDev &D, const int32_t *flags, const int32_t *list, int64_t b, int64_t e,
                            DevStatus *st, int *ok_sh) {
    if (threadIdx.x == 0) {
        int ok = 1;
        for (int64_t i = b; i < e && ok; ++i) {
            const int32_t *f = flags + list[i];
            int spins = 0;
            while (sp_flag_load(f) == 0) {
                if (sp_flag_load(D.abort) != 0) { ok = 0; break; }
                if (++spins > kSpinLimit) {
                    sp_flag_store(D.abort, 1);
                    st->timeout = 1;
                    ok = 0;
                    break;
                }
                if (spins > 8) __nanosleep(32);
            }
        }
        *ok_sh = ok;
    }
    __syncthreads();
    return *ok_sh != 0;
}

// G = A^T A on its pattern: one thread per stored entry, a merge of the two
// sorted columns of A (rows ascending), summed in row order.
__global__ void sp_gram_values_kernel(int64_t nnzg, const int32_t *__restrict__ orow, const int32_t *__restrict__ ocol,
                                      const int64_t *__restrict__ col_ptr, const int32_t *__restrict__ row_idx,
                                      const double *__restrict__ cval, double *__restrict__ gval) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnzg; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = orow[e], j = ocol[e];
        int64_t p = col_ptr[i], pe = col_ptr[i + 1], q = col_ptr[j], qe = col_ptr[j + 1];
        double s = 0.0;
        while (p < pe && q < qe) {
            const int32_t a = row_idx[p], b = row_idx[q];
            if (a < b) {
                ++p;
            } else if (a > b) {
                ++q;
            } else {
                s += cval[p] * cval[q];
                ++p;
                ++q;
            }
        }
        gval[e] = s;
    }
}

__global__ void sp_permF_kernel(int64_t n, const int32_t *__restrict__ perm, const uint8_t *__restrict__ inF,
                                int32_t *__restrict__ permF) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t j = perm[p];
        permF[p] = TS_IN(j, n) && inF[j] ? j : -1;
    }
}

// Extend-add of a child's update matrix Uc (hc x hc lower, leading dimension
// lduc) into this supernode's panel P (rows h, leading dimension ld, w
// columns) and update matrix U (leading dimension ldu): child row i lands on
// row rel[i] (increasing in i).  Child columns j0 .. j1 - 1: a warp takes a
// column j of Uc, its lanes the rows i >= j, eight at a time with every load
// issued before the stores (the targets of distinct (i, j) are distinct, so
// the reordering is safe).
template <typename T>
__device__ __noinline__ void sp_extend_add(const T *__restrict__ Uc, int64_t lduc, int64_t hc,
                                           const int32_t *__restrict__ rel, T *P, int64_t ld, T *U,
                                           int64_t ldu, int w, int64_t h, int64_t j0, int64_t j1) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t j = j0 + warp; j < j1; j += 8) {
        const int32_t lj = rel[j];
        if (!TS_IN(lj, h)) continue;
        // target column, indexed by li - roff
        T *dst = lj < w ? P + (int64_t)lj * ld : U + (int64_t)(lj - w) * ldu;
        const int roff = lj < w ? 0 : w;
        const T *src = Uc + j * lduc;
        for (int64_t i0 = j + lane; i0 < hc; i0 += 256) {
            int32_t li[8];
            T v[8], old[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int64_t i = i0 + 32 * u;
                li[u] = -1;
                if (i < hc) {
                    const int32_t r = rel[i];  // r >= lj: rows keep their order
                    if (TS_IN(r, h) && TS_IN(r - lj, h - lj)) {
                        li[u] = r;
                        v[u] = __ldcg(src + i);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (li[u] >= 0) old[u] = dst[li[u] - roff];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (li[u] >= 0) dst[li[u] - roff] = old[u] + v[u];
        }
    }
}

// FP32: block (I, J) (I >= J) of U -= X X^T on the lower triangle (X: hu
// rows x w <= 64 columns, leading dimension ld; U leading dimension ldu;
// blocks of 128 x 128): the block's row and column panels of X are staged
// in shared memory (sm: two 64 x 132 panels, k-major) and each thread
// accumulates an 8 x 8 register tile over all w columns, then loads its 64
// entries of U before storing any.  A block then costs 128 x 128 x w FMAs
// from shared memory instead of 8 global loads per 16 FMAs.  Called by all
// 256 threads.
__device__ __noinline__ void sp_syrk_block(const float *X, int64_t ld, int64_t hu, int w, float *U, int64_t ldu,
                                           float *sm, int64_t I, int64_t J) {
    constexpr int BM = 128, P = BM + 4;
    float(*Xa)[P] = reinterpret_cast<float(*)[P]>(sm);            // Xa[k][i] = X(I0 + i, k)
    float(*Xb)[P] = reinterpret_cast<float(*)[P]>(sm + 64 * P);   // Xb[k][j] = X(J0 + j, k)
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t I0 = I * BM, J0 = J * BM;
    __syncthreads();
    // eight elements of each panel per thread in flight
    for (int e0 = tid; e0 < w * BM; e0 += 256 * 8) {
        float va[8], vb[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = e0 + 256 * u, k = e / BM, i = e % BM;
            va[u] = (e < w * BM && I0 + i < hu) ? X[(int64_t)k * ld + I0 + i] : 0.f;
            vb[u] = (e < w * BM && J0 + i < hu) ? X[(int64_t)k * ld + J0 + i] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = e0 + 256 * u, k = e / BM, i = e % BM;
            if (e < w * BM) {
                Xa[k][i] = va[u];
                Xb[k][i] = vb[u];
            }
        }
    }
    __syncthreads();
    // thread (tx, ty): rows I0 + 4 tx .. + 3 and I0 + 64 + 4 tx .. + 3 (16
    // lanes run down a column of U: 16-byte accesses), columns likewise
    // from ty
    float acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
    for (int k = 0; k < w; ++k) {
        const float4 a0 = *reinterpret_cast<const float4 *>(&Xa[k][tx * 4]);
        const float4 a1 = *reinterpret_cast<const float4 *>(&Xa[k][64 + tx * 4]);
        const float4 b0 = *reinterpret_cast<const float4 *>(&Xb[k][ty * 4]);
        const float4 b1 = *reinterpret_cast<const float4 *>(&Xb[k][64 + ty * 4]);
        const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int b = 0; b < 8; ++b) acc[a][b] += av[a] * bv[b];
    }
    // U's entries: a whole 4-row group with one 16-byte load when it
    // lies inside the lower triangle (ldu, the offsets and the row
    // start are multiples of 4), entry by entry otherwise; every load
    // before the first store
    float cv[8][8];
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const int64_t j = J0 + (b < 4 ? ty * 4 + b : 64 + ty * 4 + b - 4);
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            const int64_t i4 = I0 + 64 * hh + tx * 4;
            if (j < hu && i4 + 3 < hu && i4 >= j) {
                const float4 u4 = *reinterpret_cast<const float4 *>(&U[j * ldu + i4]);
                cv[4 * hh][b] = u4.x;
                cv[4 * hh + 1][b] = u4.y;
                cv[4 * hh + 2][b] = u4.z;
                cv[4 * hh + 3][b] = u4.w;
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int64_t i = i4 + q;
                    cv[4 * hh + q][b] = (i < hu && j < hu && i >= j) ? U[j * ldu + i] : 0.f;
                }
            }
        }
    }
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const int64_t j = J0 + (b < 4 ? ty * 4 + b : 64 + ty * 4 + b - 4);
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            const int64_t i4 = I0 + 64 * hh + tx * 4;
            if (j < hu && i4 + 3 < hu && i4 >= j) {
                *reinterpret_cast<float4 *>(&U[j * ldu + i4]) =
                    make_float4(cv[4 * hh][b] - acc[4 * hh][b], cv[4 * hh + 1][b] - acc[4 * hh + 1][b],
                                cv[4 * hh + 2][b] - acc[4 * hh + 2][b], cv[4 * hh + 3][b] - acc[4 * hh + 3][b]);
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int64_t i = i4 + q;
                    if (i < hu && j < hu && i >= j) U[j * ldu + i] = cv[4 * hh + q][b] - acc[4 * hh + q][b];
                }
            }
        }
    }
}

// All blocks of one update matrix by this CTA alone.
__device__ __noinline__ void sp_syrk_tiled(const float *X, int64_t ld, int64_t hu, int w, float *U, int64_t ldu,
                                           float *sm) {
    const int64_t nb = (hu + 127) / 128;
    for (int64_t I = 0; I < nb; ++I)
        for (int64_t J = 0; J <= I; ++J) sp_syrk_block(X, ld, hu, w, U, ldu, sm, I, J);
}

// U -= X X^T on the lower triangle (X: hu rows x w columns, leading dimension
// ld; U leading dimension ldu), one 4 x 4 tile per thread and turn; the
// tile's 16 entries of U are loaded before the products so that their
// latency passes under them.
template <typename T>
__device__ __noinline__ void sp_syrk(const T *X, int64_t ld, int64_t hu, int w, T *U, int64_t ldu) {
    const int64_t nt = (hu + 3) / 4;
    for (int64_t tile = threadIdx.x; tile < nt * nt; tile += 256) {
        const int64_t tr = tile % nt, tc = tile / nt;
        if (tr < tc) continue;
        const int64_t i0 = 4 * tr, j0 = 4 * tc;
        T cv[4][4];
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int64_t i = i0 + a, j = j0 + b;
                cv[a][b] = (i < hu && j < hu && i >= j) ? U[j * ldu + i] : T(0);
            }
        T acc[4][4] = {};
        for (int k = 0; k < w; ++k) {
            const T *xk = X + (int64_t)k * ld;
            T xi[4], xj[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                xi[u] = i0 + u < hu ? xk[i0 + u] : T(0);
                xj[u] = j0 + u < hu ? xk[j0 + u] : T(0);
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] += xi[a] * xj[b];
        }
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int64_t i = i0 + a, j = j0 + b;
                if (i < hu && j < hu && i >= j) U[j * ldu + i] = cv[a][b] - acc[a][b];
            }
    }
}

// ---- shared jobs (FP32 factor) -----------------------------------------------
// Near the root the factor's critical path is a chain of tall supernodes,
// while most CTAs wait for children.  The owner of a tall supernode posts
// three of its steps as jobs in its CTA's two slots: the extend-add of its
// children by 64-column blocks of its own rows (a block gathers, child by
// child in ascending order, every child column that lands in it, so each
// entry receives its additions in the sequential order; the owner adds the
// first block, its panel, itself, and the others, which touch the update
// matrix only, run beside its diagonal block and its rows below), the rows
// below X = B W^T by 128-row blocks, and the update matrix by 128 x 128
// blocks.  CTAs that wait for children take blocks meanwhile (a
// compare-and-swap on the slot's word, which carries the kind, the
// supernode and the block count, so a stale read never claims a block of a
// job that is not posted); the owner takes blocks too, waits (bounded) until
// every block is done and frees the slot.  A block waits on nothing once
// claimed, so every claimed block completes.
//
// Word: kind << 62 | (supernode + 1) << 40 | blocks << 20 | next block.

// kinds: the update matrix, the rows below, the extend-add (all blocks) and
// the extend-add's blocks from the second on (the update matrix only)
constexpr int kSpJobSyrk = 0, kSpJobTrsm = 1, kSpJobExtend = 2, kSpJobExtendRest = 3;
constexpr int64_t kSpJobMinBlocks = 3;  // share a step of at least three blocks
constexpr int64_t kSpMaxJobSupernodes = (1ll << 22) - 1;

__device__ __forceinline__ unsigned long long sp_word_load(unsigned long long *p) {
    cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> a(*p);
    return a.load(cuda::memory_order_acquire);
}
__device__ __forceinline__ void sp_word_store(unsigned long long *p, unsigned long long v) {
    cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> a(*p);
    a.store(v, cuda::memory_order_release);
}
__device__ __forceinline__ bool sp_word_open(unsigned long long w) {
    return (w >> 40) != 0 && (w & 0xFFFFFull) < ((w >> 20) & 0xFFFFFull);
}
__device__ __forceinline__ unsigned long long sp_word(int kind, int64_t s, int64_t nblk) {
    return ((unsigned long long)kind << 62) | ((unsigned long long)(s + 1) << 40) | ((unsigned long long)nblk << 20);
}

// One thread: claim the next block of the job in slot sl, starting from the
// word value w.  Returns the claimed word (its low field is the block), or
// 0 once the job has no block left.  A failed swap means that another CTA
// claimed a block (or the job is gone), so the loop ends after at most as
// many turns as the job has blocks.
__device__ __forceinline__ unsigned long long sp_claim_slot(const SpDev &D, int sl, unsigned long long w) {
    while (sp_word_open(w)) {
        const unsigned long long prev = atomicCAS(D.job_word + sl, w, w + 1);
        if (prev == w) {
            __threadfence();  // the owner's data, published before its word, is visible from here on
            return w;
        }
        w = prev;
    }
    return 0ull;
}

// Warp 0: claim one block of any open job, the slots scanned by the lanes
// from `first` round robin.  Returns the claimed word and its slot, or 0.
// Uniform across the warp.
__device__ unsigned long long sp_claim_any(const SpDev &D, int first, int *slot) {
    const int lane = threadIdx.x & 31;
    constexpr int kRounds = 8;  // slot words a lane reads before the first is looked at
    for (int base0 = 0; base0 < D.njobs; base0 += 32 * kRounds) {
        unsigned long long ws[kRounds];
#pragma unroll
        for (int q = 0; q < kRounds; ++q) {
            const int k = base0 + 32 * q + lane;
            ws[q] = k < D.njobs ? sp_word_load(D.job_word + (first + k) % D.njobs) : 0ull;
        }
#pragma unroll
        for (int q = 0; q < kRounds; ++q) {
            const int sl = (first + base0 + 32 * q + lane) % D.njobs;
            unsigned m = __ballot_sync(0xffffffffu, sp_word_open(ws[q]));
            while (m) {
                const int src = __ffs(m) - 1;
                const int slw = __shfl_sync(0xffffffffu, sl, src);
                const unsigned long long ww = __shfl_sync(0xffffffffu, ws[q], src);
                unsigned long long got = 0;
                if (lane == 0) got = sp_claim_slot(D, slw, ww);
                got = __shfl_sync(0xffffffffu, got, 0);
                if (got != 0) {
                    *slot = slw;
                    return got;
                }
                m &= m - 1;
            }
        }
    }
    return 0ull;
}

__device__ __forceinline__ void sp_block_ij(int64_t b, int64_t &I, int64_t &J) {
    int64_t i = (int64_t)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
    while (i * (i + 1) / 2 > b) --i;
    while ((i + 1) * (i + 2) / 2 <= b) ++i;
    I = i;
    J = b - i * (i + 1) / 2;
}

// Rows r_begin .. r_end - 1 (>= w) of X = B W^T in place over the panel P of
// a supernode of w columns and h rows (leading dimension ld), W = the
// inverse of its diagonal block from Ws (W(r, c) at Ws[c w + r]), 32 rows at
// a time through shared memory (sm: W as Wt[t][c] = W(c, t), then the rows).
// All 256 threads.
__device__ void sp_trsm_rows(float *P, int64_t ld, int64_t h, int w, const float *Ws, float *sm,
                             int64_t r_begin, int64_t r_end) {
    const int tid = threadIdx.x;
    float *Wt = sm;                                                 // [t][c], w x w
    float(*Bs)[36] = reinterpret_cast<float(*)[36]>(sm + 64 * 64);  // Bs[t][r]
    __syncthreads();
    for (int e = tid; e < w * w; e += 256) Wt[e] = Ws[e];  // Ws[t w + c] = W(c, t)
    for (int64_t r0 = r_begin; r0 < r_end; r0 += 32) {
        __syncthreads();
        {  // all of this thread's loads (at most eight) before the stores
            float bv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = tid + 256 * u, t = e / 32, rr = e % 32;
                bv[u] = (e < w * 32 && r0 + rr < r_end) ? P[(int64_t)t * ld + r0 + rr] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = tid + 256 * u;
                if (e < w * 32) Bs[e / 32][e % 32] = bv[u];
            }
        }
        __syncthreads();
        for (int e = tid; e < w * 32; e += 256) {
            const int c = e / 32, rr = e % 32;
            float acc = 0.f;
            for (int t = 0; t <= c; ++t) acc += Bs[t][rr] * Wt[t * w + c];  // W(c, t), zero for t > c
            if (r0 + rr < r_end) P[(int64_t)c * ld + r0 + rr] = acc;
        }
    }
    __syncthreads();
}

// Number of entries of rel[0 .. n) (increasing) below lo and below hi, for
// all 256 threads (red: 16 ints of shared scratch).
__device__ void sp_count_below(const int32_t *rel, int64_t n, int32_t lo, int32_t hi, int *red, int64_t *c_lo,
                               int64_t *c_hi) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int a = 0, b = 0;
    for (int64_t j = tid; j < n; j += 256) {
        const int32_t r = rel[j];
        a += r < lo;
        b += r < hi;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    __syncthreads();
    if (lane == 0) {
        red[warp] = a;
        red[8 + warp] = b;
    }
    __syncthreads();
    int64_t sa = 0, sb = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        sa += red[q];
        sb += red[8 + q];
    }
    *c_lo = sa;
    *c_hi = sb;
}

// Block b of a posted job (all 256 threads).
__device__ void sp_job_block(const SpDev &D, float *L, const float *Wa, float *Ua, float *sm, int *red,
                             unsigned long long word) {
    const int kind = (int)(word >> 62);
    const int64_t s = (int64_t)((word >> 40) & 0x3FFFFFull) - 1, b = (int64_t)(word & 0xFFFFFull);
    if (!TS_IN(s, D.ns)) return;
    const int32_t w = D.sn_first[s + 1] - D.sn_first[s];
    const int64_t h = D.rows_off[s + 1] - D.rows_off[s], ld = (h + 3) / 4 * 4;
    const int64_t hu = h - w, ldu = (hu + 3) / 4 * 4;
    float *P = L + D.L_off[s];
    if (kind == kSpJobSyrk) {
        int64_t I, J;
        sp_block_ij(b, I, J);
        sp_syrk_block(P + w, ld, hu, w, Ua + D.U_off[s], ldu, sm, I, J);
    } else if (kind == kSpJobTrsm) {
        const int64_t r0 = w + 128 * b;
        sp_trsm_rows(P, ld, h, w, Wa + D.W_off[s], sm, r0, min(h, r0 + 128));
    } else {
        // this supernode's rows [64 bb, 64 bb + 64) as columns: every child
        // column landing there, child by child in ascending order
        const int64_t bb = kind == kSpJobExtendRest ? b + 1 : b;
        const int32_t lo = (int32_t)(64 * bb), hi = (int32_t)min(h, 64 * bb + 64);
        for (int64_t ci = D.c_off[s]; ci < D.c_off[s + 1]; ++ci) {
            const int32_t c = D.clist[ci];
            const int32_t wc = D.sn_first[c + 1] - D.sn_first[c];
            const int64_t hc = D.rows_off[c + 1] - D.rows_off[c] - wc, lduc = (hc + 3) / 4 * 4;
            const int32_t *rel = D.rel + D.u_off[c];
            int64_t j0, j1;
            sp_count_below(rel, hc, lo, hi, red, &j0, &j1);
            if (j1 > j0)
                sp_extend_add<float>(Ua + D.U_off[c], lduc, hc, rel, P, ld, Ua + D.U_off[s], ldu, w, h, j0, j1);
            __syncthreads();
        }
    }
}

// The factor's wait for flags[list[b..e)]: bounded, and taking blocks of
// open jobs meanwhile.  Uniform across the CTA; false on abort or timeout.
__device__ bool sp_wait_help(const SpDev &D, const int32_t *list, int64_t b, int64_t e, float *L, const float *Wa,
                             float *Ua, float *sm, int *red, DevStatus *st, long long *sh) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int idle = 0;
    for (;;) {
        if (warp == 0) {
            bool notready = false;
            for (int64_t i = b + lane; i < e; i += 32) notready |= sp_flag_load(D.flags + list[i]) == 0;
            long long cmd = 0;  // 0: ready, 1: a claimed block, 2: nothing to take, 3: abort
            unsigned long long got = 0;
            int slot = 0;
            if (__any_sync(0xffffffffu, notready)) {
                if (sp_flag_load(D.abort) != 0) {
                    cmd = 3;
                } else {
                    got = sp_claim_any(D, (int)((blockIdx.x + 1) % max(D.njobs, 1)), &slot);
                    cmd = got != 0 ? 1 : 2;
                }
            }
            if (lane == 0) {
                sh[0] = cmd;
                sh[1] = (long long)got;
                sh[2] = slot;
            }
        }
        __syncthreads();
        const long long cmd = sh[0];
        const unsigned long long word = (unsigned long long)sh[1];
        const int slot = (int)sh[2];
        __syncthreads();
        if (cmd == 0) return true;
        if (cmd == 3) return false;
        if (cmd == 2) {
            if (++idle > kSpinLimit) {
                if (tid == 0) {
                    sp_flag_store(D.abort, 1);
                    st->timeout = 1;
                }
                return false;
            }
            if (tid == 0 && idle > 8) __nanosleep(32);
            continue;
        }
        idle = 0;
        sp_job_block(D, L, Wa, Ua, sm, red, word);
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            atomicAdd(D.job_done + slot, 1);
        }
    }
}

// The owner's side of a job in slot `slot` (one of its CTA's two): post it
// (everything the blocks read is written and fenced before the word) ...
__device__ void sp_post_job(const SpDev &D, int slot, int kind, int64_t s, int64_t nblk) {
    __syncthreads();
    if (threadIdx.x == 0) {
        D.job_done[slot] = 0;
        __threadfence();
        sp_word_store(D.job_word + slot, sp_word(kind, s, nblk));
    }
    __syncthreads();
}

// ... then take blocks until none is left, wait (bounded) until the blocks
// other CTAs took are done and free the slot.  Uniform across the CTA;
// false on abort or timeout.
__device__ bool sp_finish_job(const SpDev &D, int slot, int64_t nblk, float *L, const float *Wa, float *Ua,
                              float *sm, int *red, DevStatus *st, long long *sh) {
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) sh[0] = (long long)sp_claim_slot(D, slot, sp_word_load(D.job_word + slot));
        __syncthreads();
        const unsigned long long got = (unsigned long long)sh[0];
        __syncthreads();
        if (got == 0) break;
        sp_job_block(D, L, Wa, Ua, sm, red, got);
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            atomicAdd(D.job_done + slot, 1);
        }
    }
    if (tid == 0) {
        int ok = 1, spins = 0;
        cuda::atomic_ref<int32_t, cuda::thread_scope_device> dn(D.job_done[slot]);
        while (dn.load(cuda::memory_order_acquire) < (int32_t)nblk) {
            if (sp_flag_load(D.abort) != 0) { ok = 0; break; }
            if (++spins > kSpinLimit) {
                sp_flag_store(D.abort, 1);
                st->timeout = 1;
                ok = 0;
                break;
            }
            if (spins > 8) __nanosleep(32);
        }
        if (ok) sp_word_store(D.job_word + slot, 0ull);
        sh[1] = ok;
    }
    __syncthreads();
    return sh[1] != 0;
}

__device__ bool sp_run_job(const SpDev &D, int slot, int kind, int64_t s, int64_t nblk, float *L, const float *Wa,
                           float *Ua, float *sm, int *red, DevStatus *st, long long *sh) {
    sp_post_job(D, slot, kind, s, nblk);
    return sp_finish_job(D, slot, nblk, L, Wa, Ua, sm, red, st, sh);
}

__device__ __forceinline__ bool sp_share(const SpDev &D, int64_t nblk) {
    return nblk >= kSpJobMinBlocks && 2 * (int)blockIdx.x + 1 < D.njobs && nblk < (1 << 20);
}

template <typename T, int NB>
struct SpSmem {
    static constexpr int P = NB + 4;
    static constexpr size_t core = sizeof(T) * (2 * (size_t)NB * P + (size_t)NB * 36);
    // the FP32 update matrix's two staged operand panels (sp_syrk_block),
    // more than a shared panel solve's W and rows (25 KB) need
    static constexpr size_t tiled = sizeof(T) == 4 ? sizeof(float) * 2 * 64 * 132 : 0;
    static constexpr size_t bytes = core > tiled ? core : tiled;
};

template <typename T, int NB>
__global__ void __launch_bounds__(256, 1)
    sp_factor_kernel(SpDev D, const uint8_t *__restrict__ inF, T *__restrict__ L, T *__restrict__ Wa,
                     T *__restrict__ Ua, DevStatus *st) {
    using SM = SpSmem<T, NB>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T(*A)[NB + 4] = reinterpret_cast<T(*)[NB + 4]>(smem_raw);
    T(*W)[NB + 4] = reinterpret_cast<T(*)[NB + 4]>(smem_raw + sizeof(T) * NB * SM::P);
    // the same memory viewed as 32 x 32 blocks, for supernodes of at most 32 columns
    T(*A32)[36] = reinterpret_cast<T(*)[36]>(smem_raw);
    T(*W32)[36] = reinterpret_cast<T(*)[36]>(smem_raw + sizeof(T) * NB * SM::P);
    T(*Bs)[36] = reinterpret_cast<T(*)[36]>(smem_raw + 2 * sizeof(T) * NB * SM::P);  // Bs[t][r]
    __shared__ int sh_s, ok_sh, bad_sh;
    __shared__ long long job_sh[3];
    __shared__ int red_sh[16];
    __shared__ __align__(16) T col[2][32];
    const int tid = threadIdx.x;
    constexpr bool kF32 = sizeof(T) == 4;
    float *Lf = reinterpret_cast<float *>(L);
    float *Uf = reinterpret_cast<float *>(Ua);
    const float *Wf = reinterpret_cast<const float *>(Wa);
    float *smf = reinterpret_cast<float *>(smem_raw);
    for (;;) {
        if (tid == 0) sh_s = atomicAdd(D.ticket, 1);
        __syncthreads();
        if (sh_s >= D.ns) return;
        const int64_t s = D.order_up[sh_s];
        const int32_t f = D.sn_first[s], w = D.sn_first[s + 1] - f;
        const int64_t h = D.rows_off[s + 1] - D.rows_off[s], ld = (h + 3) / 4 * 4;
        const int64_t hu = h - w, ldu = (hu + 3) / 4 * 4;
        T *P = L + D.L_off[s];
        T *U = Ua + D.U_off[s];
        // clear the panel and the update matrix before waiting: nothing else
        // touches them until this supernode's children are done
        for (int64_t e = tid; e < ld * w; e += 256) P[e] = T(0);
        for (int64_t e = tid; e < ldu * hu; e += 256) U[e] = T(0);
        if constexpr (kF32) {
            if (!sp_wait_help(D, D.clist, D.c_off[s], D.c_off[s + 1], Lf, Wf, Uf, smf, red_sh, st, job_sh)) return;
        } else {
            __syncthreads();
            if (!sp_wait_all(D, D.flags, D.clist, D.c_off[s], D.c_off[s + 1], st, &ok_sh)) return;
        }
        // G' in this supernode's columns
        for (int64_t p = D.gptr[f] + tid; p < D.gptr[f + w]; p += 256) {
            const int32_t io = D.grow_orig[p], jo = D.gcol_orig[p];
            if (!TS_IN(io, D.n) || !TS_IN(jo, D.n) || !TS_IN(D.gpos[p] - D.L_off[s], ld * w)) continue;
            const T v = (inF[io] && inF[jo]) ? (T)D.gval[p] : (io == jo ? T(1) : T(0));
            L[D.gpos[p]] = v;
        }
        __syncthreads();
        // children's update matrices (extend-add), or one child after
        // another.  Shared: the owner adds the first 64 of this supernode's
        // rows (its whole panel: w <= 64) itself, while the blocks from the
        // second on, which touch the update matrix only, go out as a job
        // that runs beside the diagonal block and the rows below and is
        // finished before the update matrix is
        const int slot_a = 2 * (int)blockIdx.x, slot_b = slot_a + 1;
        const int64_t nbe = (h + 63) / 64;
        const bool ext_shared = kF32 && sp_share(D, nbe - 1) && D.c_off[s + 1] > D.c_off[s];
        if (ext_shared) {
            sp_post_job(D, slot_a, kSpJobExtendRest, s, nbe - 1);
            sp_job_block(D, Lf, Wf, Uf, smf, red_sh, sp_word(kSpJobExtend, s, 1));  // block 0
            __syncthreads();
        } else {
            for (int64_t ci = D.c_off[s]; ci < D.c_off[s + 1]; ++ci) {
                const int32_t c = D.clist[ci];
                const int32_t wc = D.sn_first[c + 1] - D.sn_first[c];
                const int64_t hc = D.rows_off[c + 1] - D.rows_off[c] - wc, lduc = (hc + 3) / 4 * 4;
                const T *Uc = Ua + D.U_off[c];
                const int32_t *rel = D.rel + D.u_off[c];
                sp_extend_add<T>(Uc, lduc, hc, rel, P, ld, U, ldu, w, h, 0, hc);
                __syncthreads();
            }
        }
        // the diagonal block: factor and inverse in shared memory
        if (tid == 0) bad_sh = 0;
        if (w <= 32) {
            for (int e = tid; e < 32 * 32; e += 256) {
                const int c = e / 32, r = e % 32;
                T v = T(0);
                if (r < w && c < w) v = r >= c ? P[(int64_t)c * ld + r] : T(0);
                else if (r == c) v = T(1);
                A32[c][r] = v;
                W32[c][r] = T(0);
            }
            __syncthreads();
            diag_block_core<T, 32>(A32, W32, col, &bad_sh);
        } else {
            for (int e = tid; e < NB * NB; e += 256) {
                const int c = e / NB, r = e % NB;
                T v = T(0);
                if (r < w && c < w) v = r >= c ? P[(int64_t)c * ld + r] : T(0);
                else if (r == c) v = T(1);
                A[c][r] = v;
                W[c][r] = T(0);
            }
            __syncthreads();
            diag_block_core<T, NB>(A, W, col, &bad_sh);
        }
        if (tid == 0 && bad_sh && bad_sh <= w) atomicCAS(&st->chol_info, 0, (int32_t)(f + bad_sh));
        auto Lsm = [&](int c, int r) -> T { return w <= 32 ? A32[c][r] : A[c][r]; };
        auto Wsm = [&](int c, int r) -> T { return w <= 32 ? W32[c][r] : W[c][r]; };  // W(r, c)
        T *Ws = Wa + D.W_off[s];
        for (int e = tid; e < w * w; e += 256) {
            const int c = e / w, r = e % w;
            if (r >= c) P[(int64_t)c * ld + r] = Lsm(c, r);
            Ws[e] = Wsm(c, r);  // W(r, c), column-major, w x w
        }
        // rows below: X = B W^T, shared by 128-row blocks, or 32 rows at a
        // time through shared memory (Bs lies after both views of A and W)
        if (kF32 && sp_share(D, (hu + 127) / 128)) {
            if (!sp_run_job(D, slot_b, kSpJobTrsm, s, (hu + 127) / 128, Lf, Wf, Uf, smf, red_sh, st, job_sh))
                return;
        } else {
            for (int64_t r0 = w; r0 < h; r0 += 32) {
                __syncthreads();
                {  // all of this thread's loads (at most eight) before the stores
                    T bv[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int e = tid + 256 * u, t = e / 32, rr = e % 32;
                        bv[u] = (e < w * 32 && r0 + rr < h) ? P[(int64_t)t * ld + r0 + rr] : T(0);
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int e = tid + 256 * u;
                        if (e < w * 32) Bs[e / 32][e % 32] = bv[u];
                    }
                }
                __syncthreads();
                for (int e = tid; e < w * 32; e += 256) {
                    const int c = e / 32, rr = e % 32;
                    T acc = T(0);
                    for (int t = 0; t <= c; ++t) acc += Bs[t][rr] * Wsm(t, c);  // W(c, t), zero for t > c
                    if (r0 + rr < h) P[(int64_t)c * ld + r0 + rr] = acc;
                }
            }
        }
        __syncthreads();
        // the rest of the extend-add, before the update matrix takes X X^T
        if (ext_shared && !sp_finish_job(D, slot_a, nbe - 1, Lf, Wf, Uf, smf, red_sh, st, job_sh)) return;
        // update matrix: U -= X X^T on its lower triangle, X = rows below (hu x w)
        if constexpr (kF32) {
            const int64_t nbu = (hu + 127) / 128, nblk = nbu * (nbu + 1) / 2;
            if (sp_share(D, nblk)) {
                if (!sp_run_job(D, slot_a, kSpJobSyrk, s, nblk, Lf, Wf, Uf, smf, red_sh, st, job_sh)) return;
            } else {
                sp_syrk_tiled(P + w, ld, hu, w, U, ldu, smf);
            }
        } else {
            sp_syrk<T>(P + w, ld, hu, w, U, ldu);
        }
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            sp_flag_store(D.flags + s, 1);
        }
    }
}

constexpr int kSpT = 256;  // threads of a solve CTA

template <typename T>
__global__ void __launch_bounds__(kSpT)
    sp_fwd_kernel(SpDev D, const T *__restrict__ L, const T *__restrict__ Wa, T *__restrict__ ua, T *v,
                  DevStatus *st) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *a = reinterpret_cast<T *>(smem_raw);  // max_height entries
    __shared__ T y_sh[64];
    __shared__ int sh_s, ok_sh;
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) sh_s = atomicAdd(D.ticket, 1);
        __syncthreads();
        if (sh_s >= D.ns) return;
        const int64_t s = D.order_up[sh_s];
        if (!sp_wait_all(D, D.flags, D.clist, D.c_off[s], D.c_off[s + 1], st, &ok_sh)) return;
        const int32_t f = D.sn_first[s], w = D.sn_first[s + 1] - f;
        const int64_t h = D.rows_off[s + 1] - D.rows_off[s], ld = (h + 3) / 4 * 4;
        for (int64_t i = tid; i < h; i += kSpT) a[i] = i < w ? v[f + i] : T(0);
        __syncthreads();
        for (int64_t ci = D.c_off[s]; ci < D.c_off[s + 1]; ++ci) {
            const int32_t c = D.clist[ci];
            const int32_t wc = D.sn_first[c + 1] - D.sn_first[c];
            const int64_t hc = D.rows_off[c + 1] - D.rows_off[c] - wc;
            const T *uc = ua + D.u_off[c];
            const int32_t *rel = D.rel + D.u_off[c];
#pragma unroll 4
            for (int64_t i = tid; i < hc; i += kSpT) {
                const int32_t r = rel[i];
                if (TS_IN(r, h)) a[r] -= __ldcg(uc + i);
            }
            __syncthreads();
        }
        const T *Ws = Wa + D.W_off[s];
        if (tid < w) {
            T y = T(0);
#pragma unroll 8
            for (int c = 0; c <= tid; ++c) y += Ws[(int64_t)c * w + tid] * a[c];  // W(r, c), c <= r
            y_sh[tid] = y;
            v[f + tid] = y;
        }
        __syncthreads();
        // update vector of the rows below, what the parent subtracts: L_below y
        // plus the children's updates passed through (a_below holds minus
        // those).  A thread takes four rows at a time with 16-byte loads down
        // the panel's columns (a column starts 16-byte aligned: ld and the
        // panel offsets are multiples of 4), from the group holding row w.
        const T *Ls = L + D.L_off[s];
        for (int64_t q = w / 4 + tid; q < (h + 3) / 4; q += kSpT) {
            T acc[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int64_t r = 4 * q + j;
                acc[j] = (r >= w && r < h) ? -a[r] : T(0);
            }
#pragma unroll 16
            for (int k = 0; k < w; ++k) {
                T l4[4];
                ld4(Ls + (int64_t)k * ld + 4 * q, l4);
                const T yk = y_sh[k];
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[j] += l4[j] * yk;
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int64_t r = 4 * q + j;
                if (r >= w && r < h) ua[D.u_off[s] + r - w] = acc[j];
            }
        }
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            sp_flag_store(D.flags + s, 1);
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kSpT)
    sp_bwd_kernel(SpDev D, const T *__restrict__ L, const T *__restrict__ Wa, T *v, DevStatus *st) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *xb = reinterpret_cast<T *>(smem_raw);  // max_height entries: x at the rows below
    __shared__ T t_sh[128];
    __shared__ int sh_s, ok_sh;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (;;) {
        if (tid == 0) sh_s = atomicAdd(D.ticket, 1);
        __syncthreads();
        if (sh_s >= D.ns) return;
        const int64_t s = D.order_down[sh_s];
        if (!sp_wait_all(D, D.flags, D.alist, D.a_off[s], D.a_off[s + 1], st, &ok_sh)) return;
        const int32_t f = D.sn_first[s], w = D.sn_first[s + 1] - f;
        const int32_t *rows = D.rows + D.rows_off[s];
        const int64_t h = D.rows_off[s + 1] - D.rows_off[s], ld = (h + 3) / 4 * 4, hu = h - w;
        const T *Ls = L + D.L_off[s];
        // x at the rows below, gathered once (independent loads)
        for (int64_t p = tid; p < hu; p += kSpT) {
            const int32_t r = rows[w + p];
            xb[p] = TS_IN(r, D.n) ? __ldcg(v + r) : T(0);
        }
        __syncthreads();
        // t_c = y_c - sum_{p >= w} L(p, c) x(rows[p]): a warp takes four
        // adjacent columns at a time, its lanes down them by groups of four
        // rows with 16-byte loads (from the group holding row w; rows outside
        // [w, h) count zero), four independent sums, each in a fixed order
        constexpr int kWarps = kSpT / 32;
        for (int c0 = 4 * warp; c0 < w; c0 += 4 * kWarps) {
            T acc[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll 2
            for (int64_t q = w / 4 + lane; q < (h + 3) / 4; q += 32) {
                T xv[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int64_t r = 4 * q + j;
                    xv[j] = (r >= w && r < h) ? xb[r - w] : T(0);
                }
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) {
                    if (c0 + cc < w) {
                        T l4[4];
                        ld4(Ls + (int64_t)(c0 + cc) * ld + 4 * q, l4);
#pragma unroll
                        for (int j = 0; j < 4; ++j) acc[cc] += l4[j] * xv[j];
                    }
                }
            }
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc[cc] += __shfl_xor_sync(0xffffffffu, acc[cc], o);
                if (lane == 0 && c0 + cc < w) t_sh[c0 + cc] = __ldcg(v + f + c0 + cc) - acc[cc];
            }
        }
        __syncthreads();
        const T *Ws = Wa + D.W_off[s];
        T x = T(0);
        if (tid < w) {
#pragma unroll 8
            for (int cc = tid; cc < w; ++cc) x += Ws[(int64_t)tid * w + cc] * t_sh[cc];  // W(cc, r), cc >= r
        }
        if (tid < w) v[f + tid] = x;
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            sp_flag_store(D.flags + s, 1);
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// host side

template <typename T>
int SparseChol<T>::nb() {
    return kSpNB;
}

template <typename T>
size_t SparseChol<T>::device_bytes(const SparseSym &S, int /*ctas*/) {
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t ns = (size_t)S.ns, n = (size_t)S.n, ng = S.grow.size(), nu = (size_t)S.u_off[S.ns];
    size_t b = 0;
    b += up(4 * (ns + 1)) + up(8 * (ns + 1)) + up(4 * S.rows.size() + 4);  // sn_first, rows_off, rows
    b += 6 * up(8 * (ns + 1));                                           // L, W, U, u, c, a offsets
    b += up(4 * S.clist.size() + 4) + up(4 * S.alist.size() + 4) + up(4 * nu + 4);  // clist, alist, rel
    b += up(4 * n) + up(8 * (n + 1)) + 2 * up(4 * ng) + up(8 * ng) + up(8 * ng);  // perm, gptr, rows/cols, gpos, gval
    b += up(sizeof(T) * (size_t)S.L_off[ns]) + up(sizeof(T) * (size_t)S.W_off[ns]);
    b += up(sizeof(T) * (size_t)S.U_off[ns]) + up(sizeof(T) * nu + 4);   // update matrices and vectors
    b += up(4 * ns) + up(16) + up(4 * n);                                // flags, ticket / abort, permF
    b += 2 * up(4 * ns);                                                 // ticket orders
    b += up(8 * (size_t)kSpJobSlots) + up(4 * (size_t)kSpJobSlots);      // job words and counts
    return b + 256;
}

template <typename T>
cudaError_t SparseChol<T>::setup(const SparseSym &S, void *mem, cudaStream_t s, const int64_t *col_ptr,
                                 const int32_t *row_idx, const double *cval) {
    ctas = std::max(1, num_sms());
    max_height = S.max_height;
    char *p = static_cast<char *>(mem);
    auto take = [&](size_t b) {
        p = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(p) + 255) / 256 * 256);
        char *q = p;
        p += std::max<size_t>(b, 1);
        return q;
    };
    const size_t ns = (size_t)S.ns, n = (size_t)S.n, ng = S.grow.size(), nu = (size_t)S.u_off[S.ns];
    D.n = S.n;
    D.ns = S.ns;
    int32_t *sn_first = (int32_t *)take(4 * (ns + 1));
    int64_t *rows_off = (int64_t *)take(8 * (ns + 1));
    int32_t *rows = (int32_t *)take(4 * S.rows.size() + 4);
    int64_t *L_off = (int64_t *)take(8 * (ns + 1));
    int64_t *W_off = (int64_t *)take(8 * (ns + 1));
    int64_t *U_off = (int64_t *)take(8 * (ns + 1));
    int64_t *u_off = (int64_t *)take(8 * (ns + 1));
    int64_t *c_off = (int64_t *)take(8 * (ns + 1));
    int64_t *a_off = (int64_t *)take(8 * (ns + 1));
    int32_t *clist = (int32_t *)take(4 * S.clist.size() + 4);
    int32_t *alist = (int32_t *)take(4 * S.alist.size() + 4);
    int32_t *rel = (int32_t *)take(4 * nu + 4);
    int32_t *perm = (int32_t *)take(4 * n);
    int64_t *gptr = (int64_t *)take(8 * (n + 1));
    int32_t *grow_orig = (int32_t *)take(4 * ng);
    int32_t *gcol_orig = (int32_t *)take(4 * ng);
    int64_t *gpos = (int64_t *)take(8 * ng);
    double *gval = (double *)take(8 * ng);
    Lmem = (T *)take(sizeof(T) * (size_t)S.L_off[ns]);
    Wmem = (T *)take(sizeof(T) * (size_t)S.W_off[ns]);
    Umem = (T *)take(sizeof(T) * (size_t)S.U_off[ns]);
    umem = (T *)take(sizeof(T) * nu + 4);
    int32_t *flags = (int32_t *)take(4 * ns);
    int32_t *ctl = (int32_t *)take(16);
    permF = (int32_t *)take(4 * n);
    int32_t *order_up = (int32_t *)take(4 * ns);
    int32_t *order_down = (int32_t *)take(4 * ns);
    D.job_word = (unsigned long long *)take(8 * (size_t)kSpJobSlots);
    D.job_done = (int32_t *)take(4 * (size_t)kSpJobSlots);
    D.njobs = (2 * ctas <= kSpJobSlots && S.ns < kSpMaxJobSupernodes) ? 2 * ctas : 0;  // two slots per CTA
    // per-entry original column of the lower pattern
    std::vector<int32_t> gcol(ng);
    for (int64_t j = 0; j < S.n; ++j)
        for (int64_t q = S.gptr[j]; q < S.gptr[j + 1]; ++q) gcol[q] = S.perm[j];
    cudaError_t e = cudaSuccess;
    auto up = [&](void *dst, const void *src, size_t bytes) {
        if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
    };
    up(sn_first, S.sn_first.data(), 4 * (ns + 1));
    up(rows_off, S.rows_off.data(), 8 * (ns + 1));
    up(rows, S.rows.data(), 4 * S.rows.size());
    up(L_off, S.L_off.data(), 8 * (ns + 1));
    up(W_off, S.W_off.data(), 8 * (ns + 1));
    up(U_off, S.U_off.data(), 8 * (ns + 1));
    up(u_off, S.u_off.data(), 8 * (ns + 1));
    up(c_off, S.c_off.data(), 8 * (ns + 1));
    up(a_off, S.a_off.data(), 8 * (ns + 1));
    up(clist, S.clist.data(), 4 * S.clist.size());
    up(alist, S.alist.data(), 4 * S.alist.size());
    up(rel, S.rel.data(), 4 * nu);
    up(perm, S.perm.data(), 4 * n);
    up(gptr, S.gptr.data(), 8 * (n + 1));
    up(grow_orig, S.gpair_orig_row.data(), 4 * ng);
    up(gcol_orig, gcol.data(), 4 * ng);
    up(gpos, S.gpos.data(), 8 * ng);
    up(order_up, S.order_up.data(), 4 * ns);
    up(order_down, S.order_down.data(), 4 * ns);
    if (e != cudaSuccess) return e;
    // the host vectors must outlive the copies: wait for them here (setup runs once per problem)
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    D.sn_first = sn_first;
    D.rows_off = rows_off;
    D.rows = rows;
    D.L_off = L_off;
    D.W_off = W_off;
    D.U_off = U_off;
    D.u_off = u_off;
    D.c_off = c_off;
    D.a_off = a_off;
    D.clist = clist;
    D.alist = alist;
    D.rel = rel;
    D.perm = perm;
    D.gptr = gptr;
    D.grow_orig = grow_orig;
    D.gcol_orig = gcol_orig;
    D.gpos = gpos;
    D.gval = gval;
    D.order_up = order_up;
    D.order_down = order_down;
    D.flags = flags;
    D.ticket = ctl;
    D.abort = ctl + 1;
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv((int64_t)ng, 256), (int64_t)num_sms() * 8));
    sp_gram_values_kernel<<<g, 256, 0, s>>>((int64_t)ng, grow_orig, gcol_orig, col_ptr, row_idx, cval, gval);
    note_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t SparseChol<T>::reset(cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(D.flags, 0, sizeof(int32_t) * (size_t)D.ns, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(D.ticket, 0, 16, s);
    return e;
}

template <typename T>
cudaError_t SparseChol<T>::factor(cudaStream_t s, const uint8_t *inF, DevStatus *st) {
    constexpr int NB = kSpNB;
    const size_t smem = SpSmem<T, NB>::bytes;
    cudaError_t e = cudaFuncSetAttribute(sp_factor_kernel<T, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e == cudaSuccess) e = reset(s);
    if (e == cudaSuccess && sizeof(T) == 4)  // no job is open (an aborted factor may have left one)
        e = cudaMemsetAsync(D.job_word, 0, sizeof(unsigned long long) * kSpJobSlots, s);
    if (e != cudaSuccess) return e;
    sp_factor_kernel<T, NB><<<ctas, 256, smem, s>>>(D, inF, Lmem, Wmem, Umem, st);
    note_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t SparseChol<T>::perm_list(cudaStream_t s, const uint8_t *inF) {
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(D.n, 256), (int64_t)num_sms() * 8));
    sp_permF_kernel<<<g, 256, 0, s>>>(D.n, D.perm, inF, permF);
    note_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t SparseChol<T>::solve(cudaStream_t s, T *v, DevStatus *st) {
    const int g = std::max(1, num_sms() * 4);
    const size_t smem = sizeof(T) * (size_t)std::max<int64_t>(max_height, 1);
    cudaError_t e = cudaFuncSetAttribute(sp_fwd_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sp_bwd_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = reset(s);
    if (e != cudaSuccess) return e;
    sp_fwd_kernel<T><<<g, kSpT, smem, s>>>(D, Lmem, Wmem, umem, v, st);
    e = reset(s);
    if (e != cudaSuccess) return e;
    sp_bwd_kernel<T><<<g, kSpT, smem, s>>>(D, Lmem, Wmem, v, st);
    note_launches(2);
    return cudaGetLastError();
}

template struct SparseChol<float>;
template struct SparseChol<double>;

}  // namespace tsnnls

TSNNLS_CHECK_UNIT("sparse_chol")
