// Dense building blocks shared by the blocked Cholesky of the gathered
// normal-equations block and the supernodal sparse Cholesky (Section 2,
// "normal equations solver"): 4-vector shared-memory access, the warp-level
// 32 x 32 factor + inverse, CTA-level small products, and the factor +
// inverse of one NB x NB diagonal block held in shared memory.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tsnnls {

// ---------------------------------------------------------------------------
// ---- 4-element vector access (16-byte aligned) --------------------------------
__device__ __forceinline__ void ld4(const float *p, float (&v)[4]) {
    const float4 f = *reinterpret_cast<const float4 *>(p);
    v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
}
__device__ __forceinline__ void ld4(const double *p, double (&v)[4]) {
    const double2 f = *reinterpret_cast<const double2 *>(p);
    const double2 g = *reinterpret_cast<const double2 *>(p + 2);
    v[0] = f.x; v[1] = f.y; v[2] = g.x; v[3] = g.y;
}
__device__ __forceinline__ void ld2(const float *p, float (&v)[2]) {
    const float2 a = *reinterpret_cast<const float2 *>(p);
    v[0] = a.x;
    v[1] = a.y;
}
__device__ __forceinline__ void ld2(const double *p, double (&v)[2]) {
    const double2 a = *reinterpret_cast<const double2 *>(p);
    v[0] = a.x;
    v[1] = a.y;
}
__device__ __forceinline__ void st4(float *p, const float (&v)[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double *p, const double (&v)[4]) {
    *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
    *reinterpret_cast<double2 *>(p + 2) = make_double2(v[2], v[3]);
}

// ---- warp-level 32 x 32 factor + inverse -------------------------------------
// Lane i holds row i of the block (a[32]) and column i of W = L^-1 (w[32]);
// step J, fully unrolled through template recursion so that every register
// index is a compile-time constant:
//   L(J, J) = sqrt(a_J[J]),  L(i, J) = a_i[J] / L(J, J),
//   a_i[l] -= L(i, J) L(l, J)                      for J < l <= i;
// the same column J drives the inverse by forward substitution, w[l]
// (l > J) accumulating sum_{t <= J} L(l, t) W(t, c) until step l:
//   W(J, c) = (delta_Jc - w[J]) / L(J, J),  w[l] += L(l, J) W(J, c).
// Column J reaches every lane through a 32-entry shared buffer (one store
// per lane, broadcast vector loads), double-buffered by the parity of J.
template <typename T>
struct WarpChol {
    T a[32], w[32];
};

__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }

template <typename T, int J>
__device__ __forceinline__ void warp_chol_step(WarpChol<T> &s, T (*col)[32], int lane, int &bad, int base,
                                               T d) {
    if (!(d > T(0))) {
        if (!bad) bad = base + J + 1;
        d = T(1);
    }
    const T inv = rsqrt_t(d);
    const T lij = (lane > J) ? s.a[J] * inv : (lane == J ? d * inv : s.a[J]);
    s.a[J] = lij;
    const T wj = (J >= lane) ? (((J == lane) ? T(1) : T(0)) - s.w[J]) * inv : T(0);
    s.w[J] = wj;
    if constexpr (J + 1 < 32) {
        // the next pivot first: lane J + 1 finishes its diagonal entry with its
        // own L(J + 1, J), so the pivot chain skips the shared-memory broadcast
        const T dn = __shfl_sync(0xffffffffu, s.a[J + 1] - lij * lij, J + 1);
        col[J & 1][lane] = lij;
        __syncwarp();
#pragma unroll
        for (int g = (J + 1) / 4; g < 8; ++g) {
            T v[4];
            ld4(&col[J & 1][4 * g], v);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int l = 4 * g + u;
                if (l > J) {
                    // rows above l (lane < l) update entries above the
                    // diagonal, which are never read as L: no predicate
                    s.a[l] -= lij * v[u];
                    s.w[l] += v[u] * wj;
                }
            }
        }
        warp_chol_step<T, J + 1>(s, col, lane, bad, base, dn);
    }
}

// The same step without the inverse (L only, half the registers), for
// callers that solve with L directly.
template <typename T>
struct WarpCholL {
    T a[32];
};

template <typename T, int J>
__device__ __forceinline__ void warp_chol_step_l(WarpCholL<T> &s, T (*col)[32], int lane, int &bad, T d) {
    if (!(d > T(0))) {
        if (!bad) bad = J + 1;
        d = T(1);
    }
    const T inv = rsqrt_t(d);
    const T lij = (lane > J) ? s.a[J] * inv : (lane == J ? d * inv : s.a[J]);
    s.a[J] = lij;
    if constexpr (J + 1 < 32) {
        const T dn = __shfl_sync(0xffffffffu, s.a[J + 1] - lij * lij, J + 1);
        col[J & 1][lane] = lij;
        __syncwarp();
#pragma unroll
        for (int g = (J + 1) / 4; g < 8; ++g) {
            T v[4];
            ld4(&col[J & 1][4 * g], v);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int l = 4 * g + u;
                if (l > J) s.a[l] -= lij * v[u];
            }
        }
        warp_chol_step_l<T, J + 1>(s, col, lane, bad, dn);
    }
}

// Factor A(j0.., j0..) (32 x 32, lower) in place and write its inverse to W
// (W[col][row]) and, transposed, to the strict upper triangle of the block
// in A.  col: 2 x 32 shared scratch, 16-byte aligned.
template <typename T, int NB>
__device__ __forceinline__ void warp_chol_inv(T (*A)[NB + 4], T (*W)[NB + 4], T (*col)[32], int j0,
                                              int lane, int &bad) {
    WarpChol<T> s;
#pragma unroll
    for (int c = 0; c < 32; ++c) {
        s.a[c] = c <= lane ? A[j0 + c][j0 + lane] : T(0);
        s.w[c] = T(0);
    }
    warp_chol_step<T, 0>(s, col, lane, bad, j0, __shfl_sync(0xffffffffu, s.a[0], 0));
#pragma unroll
    for (int c = 0; c < 32; ++c) {
        A[j0 + c][j0 + lane] = c <= lane ? s.a[c] : s.w[c];  // L, and W(c, lane) above the diagonal
        W[j0 + lane][j0 + c] = s.w[c];  // column `lane` of W, rows c (0 above the diagonal)
    }
}

// ---- CTA-level small products on shared-memory blocks -------------------------
// For each of nb independent products:  out(r, c) = sum_{t < K} X(r, t) Y(t, c),
// r < M, c < N (multiples of 4), in 4 x 4 register tiles, one per thread and
// wave of 256.  fx(b, r0, t, x) loads X(r0..r0+3, t), fy(b, t, c0, y) loads
// Y(t, c0..c0+3), fo(b, r0, c0, acc) stores the tile, fr(b, r0, c0, t0, t1)
// may narrow the sum to t0 <= t < t1 (zeros of a triangular factor).  tri: only the lower
// tiles (row block >= column block) of a square output.  All reads of a wave
// happen before the barrier and all writes after it, so an output that fits
// in one wave may overwrite a source.
struct FullRange {
    __device__ void operator()(int, int, int, int &, int &) const {}
};

template <typename T, typename FX, typename FY, typename FO, typename FR = FullRange>
__device__ __forceinline__ void cta_prod(int nb, int M, int N, int K, bool tri, FX fx, FY fy, FO fo,
                                         FR fr = FR()) {
    const int tid = threadIdx.x;
    const int nt_r = M / 4, nt_c = N / 4;
    const int per = tri ? nt_r * (nt_r + 1) / 2 : nt_r * nt_c;
    const int ntiles = nb * per;
    for (int base = 0; base < ntiles; base += 256) {
        const int tile = base + tid;
        const bool active = tile < ntiles;
        T acc[4][4] = {};
        int bi = 0, tr = 0, tc = 0;
        if (active) {
            bi = tile / per;
            const int lt = tile - bi * per;
            if (tri) {
                int i = (int)((sqrtf(8.f * lt + 1.f) - 1.f) * 0.5f);
                while (i * (i + 1) / 2 > lt) --i;
                while ((i + 1) * (i + 2) / 2 <= lt) ++i;
                tr = i;
                tc = lt - i * (i + 1) / 2;
            } else {
                tr = lt % nt_r;
                tc = lt / nt_r;
            }
            int t0 = 0, t1 = K;
            fr(bi, tr * 4, tc * 4, t0, t1);  // narrower t-range where a factor is triangular
#pragma unroll 4
            for (int t = t0; t < t1; ++t) {
                T x[4], y[4];
                fx(bi, tr * 4, t, x);
                fy(bi, t, tc * 4, y);
#pragma unroll
                for (int p = 0; p < 4; ++p)
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[p][q] += x[p] * y[q];
            }
        }
        __syncthreads();
        if (active) fo(bi, tr * 4, tc * 4, acc);
        __syncthreads();
    }
}

// ---- factor + invert an NB x NB block in shared memory (256 threads)
// A[col][row] holds the block (lower triangle, identity beyond the block's
// true size), W[col][row] starts at 0.  On return A's lower triangle holds L
// and its strict upper triangle W^T, W = L^-1 (W[col][row] = W(row, col)),
// and *bad_sh (initially 0) the 1-based column of the first non-positive
// pivot, if any.  For each 32-column block jb: warp 0 factors and inverts the
// 32 x 32 diagonal block, the CTA forms X = B W_jj^T for the rows below it
// (in place) and subtracts X X^T from the trailing lower triangle.  The
// off-diagonal blocks of W follow level by level: for sibling blocks a, b of
// size sz, W_ba = -W_bb (L_ba W_aa).  Called by all 256 threads after a
// barrier; ends with a barrier.
template <typename T, int NB>
__device__ __forceinline__ void diag_block_core(T (*A)[NB + 4], T (*W)[NB + 4], T (*col)[32], int *bad_sh) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NBB = NB / 32;
    for (int jb = 0; jb < NBB; ++jb) {
        const int j0 = jb * 32;
        if (warp == 0) {
            int bad = 0;
            warp_chol_inv<T, NB>(A, W, col, j0, lane, bad);
            if (lane == 0 && bad && !*bad_sh) *bad_sh = bad;
        }
        __syncthreads();
        const int R = NB - j0 - 32;
        if (R > 0) {
            // rows below: X = B W_jj^T, in place over B
            cta_prod<T>(
                1, R, 32, 32, false,
                [&](int, int r0, int t, T(&x)[4]) { ld4(&A[j0 + t][j0 + 32 + r0], x); },
                [&](int, int t, int c0, T(&y)[4]) { ld4(&W[j0 + t][j0 + c0], y); },  // W_jj(c, t)
                [&](int, int r0, int c0, T(&acc)[4][4]) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const T o[4] = {acc[0][q], acc[1][q], acc[2][q], acc[3][q]};
                        st4(&A[j0 + c0 + q][j0 + 32 + r0], o);
                    }
                },
                [](int, int, int c0, int &, int &t1) { t1 = c0 + 4; });  // W_jj(c, t) = 0 for t > c
            // trailing update: A(r, c) -= sum_t X(r, t) X(c, t) on the lower part
            cta_prod<T>(
                1, R, R, 32, true,
                [&](int, int r0, int t, T(&x)[4]) { ld4(&A[j0 + t][j0 + 32 + r0], x); },
                [&](int, int t, int c0, T(&y)[4]) { ld4(&A[j0 + t][j0 + 32 + c0], y); },
                [&](int, int r0, int c0, T(&acc)[4][4]) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        T *col = &A[j0 + 32 + c0 + q][j0 + 32 + r0];
                        T o[4];
                        ld4(col, o);
#pragma unroll
                        for (int p = 0; p < 4; ++p)
                            if (r0 + p >= c0 + q) o[p] -= acc[p][q];
                        st4(col, o);
                    }
                });
        }
    }
    // off-diagonal blocks of W = L^-1, level by level, all pairs of a level
    // at once: T1 = L_ba W_aa goes to the free upper block (rows a, columns
    // b) of W, then W_ba = -W_bb T1, then the scratch is cleared (it lies in
    // the upper triangle of the next level's diagonal blocks).
    for (int sz = 32; sz < NB; sz *= 2) {
        const int npair = NB / (2 * sz);
        cta_prod<T>(
            npair, sz, sz, sz, false,
            [&](int p, int r0, int t, T(&x)[4]) {  // L_ba(r, t)
                const int a0 = 2 * sz * p, b0 = a0 + sz;
                ld4(&A[a0 + t][b0 + r0], x);
            },
            [&](int p, int t, int c0, T(&y)[4]) {  // W_aa(t, c)
                const int a0 = 2 * sz * p;
#pragma unroll
                for (int q = 0; q < 4; ++q) y[q] = W[a0 + c0 + q][a0 + t];
            },
            [&](int p, int r0, int c0, T(&acc)[4][4]) {  // T1(r, c) at W[b0 + r][a0 + c]
                const int a0 = 2 * sz * p, b0 = a0 + sz;
#pragma unroll
                for (int pp = 0; pp < 4; ++pp) st4(&W[b0 + r0 + pp][a0 + c0], acc[pp]);
            },
            [](int, int, int c0, int &t0, int &) { t0 = c0; });  // W_aa(t, c) = 0 for t < c
        cta_prod<T>(
            npair, sz, sz, sz, false,
            [&](int p, int r0, int t, T(&x)[4]) {  // W_bb(r, t)
                const int b0 = 2 * sz * p + sz;
                ld4(&W[b0 + t][b0 + r0], x);
            },
            [&](int p, int t, int c0, T(&y)[4]) {  // T1(t, c)
                const int a0 = 2 * sz * p, b0 = a0 + sz;
                ld4(&W[b0 + t][a0 + c0], y);
            },
            [&](int p, int r0, int c0, T(&acc)[4][4]) {  // W_ba(r, c) at W[a0 + c][b0 + r]
                const int a0 = 2 * sz * p, b0 = a0 + sz;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const T o[4] = {-acc[0][q], -acc[1][q], -acc[2][q], -acc[3][q]};
                    st4(&W[a0 + c0 + q][b0 + r0], o);
                }
                // and transposed into the strict upper triangle of A: S(a0 + c, b0 + r)
#pragma unroll
                for (int pp = 0; pp < 4; ++pp) {
                    const T o[4] = {-acc[pp][0], -acc[pp][1], -acc[pp][2], -acc[pp][3]};
                    st4(&A[b0 + r0 + pp][a0 + c0], o);
                }
            },
            [](int, int r0, int, int &, int &t1) { t1 = r0 + 4; });  // W_bb(r, t) = 0 for t > r
        for (int e = tid; e < npair * sz * sz / 4; e += 256) {
            const int p = e / (sz * sz / 4), f = e % (sz * sz / 4);
            const int a0 = 2 * sz * p, b0 = a0 + sz;
            const T z[4] = {T(0), T(0), T(0), T(0)};
            st4(&W[b0 + f / (sz / 4)][a0 + (f % (sz / 4)) * 4], z);
        }
        __syncthreads();
    }
}

}  // namespace tsnnls
