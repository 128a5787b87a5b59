// Reuse of one Cholesky factor across pivots.  The paper refactors the
// normal-equations matrix at every pivot (Section 2 box, Section 3); when only
// a few variables move, this instead keeps the factor L of G_BB for an earlier
// set B and solves over U = B + A (A: variables added since) with the rows
// and columns of R (variables of B removed since) held at zero:
//
//   H = G_UU = [[G_BB, G_BA], [G_AB, G_AA]] = L_U L_U^T,
//   L_U = [[L, 0], [P, Q]],  P^T = L^-1 G_BA,  Q Q^T = G_AA - P P^T,
//
// and, with Z = H^-1 E_R and C = Z_R (the R rows of Z, = (H^-1)_RR, SPD),
//   z = H^-1 w - Z C^-1 (H^-1 w)_R
// solves H z + E_R mu = w, z_R = 0: its F' = U \ R part solves
// G_F'F' z_F' = w_F' (block elimination with a bordered factor, and the
// capacitance form of deleting rows and columns).  The long vectors and
// their triangular solves run in the factor's precision, the a x a and r x r
// factors in FP64; the FP64 refinement of the solve takes the result to full
// accuracy exactly as with a fresh factor.  The setup's triangular solves run
// side by side (one launch for the a columns of P^T, two for the r of Z).
#include <cuda_runtime.h>
#include <stdint.h>

#include "check.cuh"
#include "common.cuh"

namespace tsnnls {

constexpr int kBThreads = 1024;

// A = {j : F'_j and not B_j} ascending, R = {p < kb : B[p] not in F'}
// ascending, U = B with R entries set to -1, then A.  Lists hold at most
// kBorderMax entries; the counts are exact (st->border_a / border_r).
__global__ void __launch_bounds__(kBThreads)
    border_diff_kernel(int64_t n, const uint8_t *__restrict__ inF, const uint8_t *__restrict__ inB,
                       const int32_t *__restrict__ Bl, int64_t kb, int32_t *__restrict__ Ul,
                       int32_t *__restrict__ Al, int32_t *__restrict__ Rpos, DevStatus *st) {
    __shared__ int32_t wsum[32];
    __shared__ int64_t carry;
    __shared__ int32_t al[kBorderMax];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // one ballot-and-scan compaction pass over [0, N)
    auto compact = [&](int64_t N, auto pred, auto emit) -> int64_t {
        if (tid == 0) carry = 0;
        __syncthreads();
        for (int64_t base = 0; base < N; base += kBThreads) {
            const int64_t i = base + tid;
            const int v = (i < N) ? (int)pred(i) : 0;
            const unsigned bal = __ballot_sync(0xffffffffu, v);
            const int before = __popc(bal & ((1u << lane) - 1u));
            if (lane == 0) wsum[warp] = __popc(bal);
            __syncthreads();
            if (warp == 0) {
                int w = wsum[lane];
                for (int o = 1; o < 32; o <<= 1) {
                    const int t = __shfl_up_sync(0xffffffffu, w, o);
                    if (lane >= o) w += t;
                }
                wsum[lane] = w;  // inclusive prefix over warps
            }
            __syncthreads();
            if (v) emit(carry + (warp > 0 ? wsum[warp - 1] : 0) + before, i);
            __syncthreads();
            if (tid == 0) carry += wsum[31];
            __syncthreads();
        }
        return carry;
    };
    const int64_t a = compact(
        n, [&](int64_t j) { return inF[j] != 0 && inB[j] == 0; },
        [&](int64_t pos, int64_t j) {
            if (pos < kBorderMax) {
                Al[pos] = (int32_t)j;
                al[pos] = (int32_t)j;
            }
        });
    const int64_t r = compact(
        kb, [&](int64_t p) { return TS_IN(Bl[p], n) && inF[Bl[p]] == 0; },
        [&](int64_t pos, int64_t p) {
            if (pos < kBorderMax) Rpos[pos] = (int32_t)p;
        });
    for (int64_t p = tid; p < kb; p += kBThreads) Ul[p] = TS_IN(Bl[p], n) && inF[Bl[p]] ? Bl[p] : -1;
    if (tid < kBorderMax && tid < a) Ul[kb + tid] = al[tid];
    if (tid == 0) {
        st->border_a = (int32_t)min(a, (int64_t)INT32_MAX);
        st->border_r = (int32_t)min(r, (int64_t)INT32_MAX);
    }
}

// Counts only: st->border_a = |F' \ B|, st->border_r = |B \ F'| (integer
// sums, so the order of the CTAs does not matter).
__global__ void border_count_kernel(int64_t n, const uint8_t *__restrict__ inF, const uint8_t *__restrict__ inB,
                                    DevStatus *st) {
    int a = 0, r = 0;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const bool f = inF[j] != 0, b = inB[j] != 0;
        a += f && !b;
        r += b && !f;
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        r += __shfl_xor_sync(0xffffffffu, r, o);
    }
    if ((threadIdx.x & 31) == 0 && (a | r)) {
        atomicAdd(&st->border_a, a);
        atomicAdd(&st->border_r, r);
    }
}

// Pt(p, al) = G(B[p], A[al]) for p < kb; GAA(al, be) = G(A[al], A[be]).
// G holds the lower triangle of the cached A^T A (leading dimension ldg).
template <typename T>
__global__ void border_gather_kernel(const T *__restrict__ G, int64_t ldg, const int32_t *__restrict__ Bl,
                                     int64_t kb, const int32_t *__restrict__ Al, int a, T *__restrict__ Pt,
                                     int64_t ldp, double *__restrict__ GAA) {
    const int64_t rows = kb + a;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < rows * a;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % rows;
        const int al = (int)(e / rows);
        const int64_t ri = i < kb ? Bl[i] : Al[i - kb], cj = Al[al];
        const T v = TS_IN(ri, ldg) && TS_IN(cj, ldg) ? (ri >= cj ? G[ri + cj * ldg] : G[cj + ri * ldg]) : T(0);
        if (i < kb) Pt[i + al * ldp] = v;
        else GAA[(i - kb) + al * kBorderMax] = (double)v;
    }
}

// SA(al, be) = GAA(al, be) - sum_p Pt(p, al) Pt(p, be) for be <= al (FP64
// sums in a fixed order), one CTA per entry.
template <typename T>
__global__ void __launch_bounds__(256)
    border_schur_kernel(const T *__restrict__ Pt, int64_t ldp, int64_t kb, int a, const double *__restrict__ GAA,
                        double *__restrict__ SA) {
    __shared__ double sh[8];
    const int al = blockIdx.x % a, be = blockIdx.x / a;
    if (be > al) return;
    double t = 0.0;
    for (int64_t p = threadIdx.x; p < kb; p += 256) t += (double)Pt[p + al * ldp] * (double)Pt[p + be * ldp];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += sh[w];
        SA[al + be * kBorderMax] = GAA[al + be * kBorderMax] - s;
    }
}

// In-place Cholesky of the a x a lower triangle of M (leading dimension
// kBorderMax, FP64) by one warp, lane i holding row i; the strict upper part
// is set to zero.  *bad = 1 on a non-positive pivot.
__device__ __forceinline__ void warp_small_chol(double *M, int a, int32_t *bad) {
    const int lane = threadIdx.x & 31;
    double m[kBorderMax];
#pragma unroll
    for (int c = 0; c < kBorderMax; ++c) m[c] = (lane < a && c < a && c <= lane) ? M[lane + c * kBorderMax] : 0.0;
    int fail = 0;
#pragma unroll
    for (int j = 0; j < kBorderMax; ++j) {
        if (j < a) {
            double d = __shfl_sync(0xffffffffu, m[j], j);
            if (!(d > 0.0)) {
                fail = 1;
                d = 1.0;
            }
            const double inv = rsqrt(d);
            const double l = lane > j ? m[j] * inv : (lane == j ? d * inv : 0.0);
            m[j] = l;
#pragma unroll
            for (int c = j + 1; c < kBorderMax; ++c) {
                const double v = __shfl_sync(0xffffffffu, l, c);
                if (c < a && lane >= c) m[c] -= l * v;
            }
        }
    }
    if (lane < a) {
#pragma unroll
        for (int c = 0; c < kBorderMax; ++c)
            if (c < a) M[lane + c * kBorderMax] = c <= lane ? m[c] : 0.0;
    }
    if (lane == 0 && fail) *bad = 1;
}

__global__ void border_chol_kernel(double *M, int a, int32_t *bad) {
    if (threadIdx.x < 32) warp_small_chol(M, a, bad);
}

// v <- (L L^T)^-1 v for the a x a factor L (leading dimension kBorderMax) by
// one warp; v[i] lives in lane i.
__device__ __forceinline__ double warp_small_solve(const double *L, int a, double v) {
    const int lane = threadIdx.x & 31;
    for (int j = 0; j < a; ++j) {  // L y = v
        if (lane == j) v /= L[j + j * kBorderMax];
        const double vj = __shfl_sync(0xffffffffu, v, j);
        if (lane > j && lane < a) v -= L[lane + j * kBorderMax] * vj;
    }
    for (int j = a - 1; j >= 0; --j) {  // L^T x = y
        if (lane == j) v /= L[j + j * kBorderMax];
        const double vj = __shfl_sync(0xffffffffu, v, j);
        if (lane < j) v -= L[j + lane * kBorderMax] * vj;
    }
    return v;
}

// Middle of H^-1 w, after the forward solve with L on z[0, kb):
// t = z_A - P z_B, z_A <- Q^-T Q^-1 t, z_B <- z_B - P^T z_A.  One CTA.  The
// long dot products run in the factor's precision T (GB300 issues FP64 at a
// small fraction of the FP32 rate); only the a x a solve is FP64.
constexpr int kMidThreads = 512;

template <typename T>
__global__ void __launch_bounds__(kMidThreads)
    border_mid_kernel(T *__restrict__ z, int64_t kb, int a, const T *__restrict__ Pt, int64_t ldp,
                      const double *__restrict__ Lq, int64_t zld) {
    z += (int64_t)blockIdx.y * zld;  // one vector per grid row
    __shared__ T red[kMidThreads / 32];
    __shared__ double tv[kBorderMax];
    __shared__ T za[kBorderMax];
    __shared__ double Ls[kBorderMax * kBorderMax];  // the sequential solve reads the factor from here
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int e = tid; e < kBorderMax * kBorderMax; e += kMidThreads) Ls[e] = Lq[e];
    for (int al = 0; al < a; ++al) {
        const T *pc = Pt + (int64_t)al * ldp;
        T acc = T(0);
        for (int64_t p = tid; p < kb; p += kMidThreads) acc += pc[p] * z[p];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) red[warp] = acc;
        __syncthreads();
        if (tid == 0) {
            T t = T(0);
            for (int w = 0; w < kMidThreads / 32; ++w) t += red[w];
            tv[al] = (double)z[kb + al] - (double)t;
        }
        __syncthreads();
    }
    if (warp == 0) {
        double t = lane < a ? tv[lane] : 0.0;
        t = warp_small_solve(Ls, a, t);
        if (lane < a) {
            za[lane] = (T)t;
            z[kb + lane] = (T)t;
        }
    }
    __syncthreads();
    for (int64_t p = tid; p < kb; p += kMidThreads) {
        T s = T(0);
        for (int al = 0; al < a; ++al) s += Pt[p + (int64_t)al * ldp] * za[al];
        z[p] -= s;
    }
}

// mu = C^-1 z_R (one warp), then z <- z - Z mu over all u rows.
template <typename T>
__global__ void border_cap_mu_kernel(const T *__restrict__ z, int r, const int32_t *__restrict__ Rpos,
                                     const double *__restrict__ Lc, double *__restrict__ mu) {
    __shared__ double Ls[kBorderMax * kBorderMax];
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int e = lane; e < kBorderMax * kBorderMax; e += 32) Ls[e] = Lc[e];
    __syncwarp();
    double g = 0.0;
    if (lane < r) g = (double)z[Rpos[lane]];
    g = warp_small_solve(Ls, r, g);
    if (lane < r) mu[lane] = g;
}

template <typename T>
__global__ void border_cap_apply_kernel(T *__restrict__ z, int64_t u, int r, const T *__restrict__ Z, int64_t ldz,
                                        const double *__restrict__ mu) {
    __shared__ T m[kBorderMax];
    if (threadIdx.x < kBorderMax) m[threadIdx.x] = threadIdx.x < r ? (T)mu[threadIdx.x] : T(0);
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < u; i += (int64_t)gridDim.x * blockDim.x) {
        T s = T(0);
        for (int q = 0; q < r; ++q) s += Z[i + q * ldz] * m[q];
        z[i] -= s;
    }
}

// Z(:, q) = e_{Rpos[q]} over u rows
template <typename T>
__global__ void border_unit_kernel(T *__restrict__ Z, int64_t u, int64_t ldz, int r, const int32_t *__restrict__ Rpos) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < u * r; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % u;
        const int q = (int)(e / u);
        Z[i + q * ldz] = (i == Rpos[q]) ? T(1) : T(0);
    }
}

// C(q, s) = (Z(Rpos[q], s) + Z(Rpos[s], q)) / 2 for s <= q, then its Cholesky.
template <typename T>
__global__ void border_cap_factor_kernel(const T *__restrict__ Z, int64_t ldz, int r, const int32_t *__restrict__ Rpos,
                                         double *__restrict__ C, int32_t *bad) {
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
        const int q = e % r, s = e / r;
        if (s <= q)
            C[q + s * kBorderMax] = 0.5 * ((double)Z[Rpos[q] + s * ldz] + (double)Z[Rpos[s] + q * ldz]);
    }
    __syncthreads();
    if (threadIdx.x < 32) warp_small_chol(C, r, bad);
}

// ---------------------------------------------------------------------------

size_t border_bytes(int64_t n, size_t elem) {
    const int64_t u = n + kBorderMax;
    return (size_t)round_up(4 * n, 256) + (size_t)round_up(n, 256)   // base list, base flags
           + (size_t)round_up(4 * u, 256) + 2 * 256                  // U list, A list, R positions
           + (size_t)round_up((int64_t)elem * n * kBorderMax, 256)   // P^T
           + (size_t)round_up((int64_t)elem * u * kBorderMax, 256)   // Z
           + 4 * (size_t)round_up(8 * kBorderMax * kBorderMax, 256)  // G_AA, Q, C, spare
           + 256 + 256                                               // mu, flag
           + trsv_multi_scratch_bytes(n, elem, kBorderMax);          // simultaneous solves
}

BorderBuffers border_carve(void *base, int64_t n, size_t elem) {
    BorderBuffers b{};
    char *p = static_cast<char *>(base);
    auto take = [&](size_t bytes) {
        char *q = p;
        p += round_up((int64_t)bytes, 256);
        return q;
    };
    const int64_t u = n + kBorderMax;
    b.Bl = reinterpret_cast<int32_t *>(take(4 * n));
    b.inB = reinterpret_cast<uint8_t *>(take(n));
    b.Ul = reinterpret_cast<int32_t *>(take(4 * u));
    b.Al = reinterpret_cast<int32_t *>(take(4 * kBorderMax));
    b.Rpos = reinterpret_cast<int32_t *>(take(4 * kBorderMax));
    b.Pt = take(elem * n * kBorderMax);
    b.Z = take(elem * u * kBorderMax);
    b.GAA = reinterpret_cast<double *>(take(8 * kBorderMax * kBorderMax));
    b.Lq = reinterpret_cast<double *>(take(8 * kBorderMax * kBorderMax));
    b.Lc = reinterpret_cast<double *>(take(8 * kBorderMax * kBorderMax));
    take(8 * kBorderMax * kBorderMax);
    b.mu = reinterpret_cast<double *>(take(8 * kBorderMax));
    b.bad = reinterpret_cast<int32_t *>(take(4));
    b.multi = take(trsv_multi_scratch_bytes(n, elem, kBorderMax));
    b.ldp = n;
    b.ldz = u;
    return b;
}

cudaError_t launch_border_count(cudaStream_t s, int64_t n, const uint8_t *inF, const BorderBuffers &b,
                                DevStatus *st) {
    static_assert(offsetof(DevStatus, border_r) == offsetof(DevStatus, border_a) + sizeof(int32_t), "adjacent");
    cudaError_t e = cudaMemsetAsync(&st->border_a, 0, 2 * sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(n, 256), num_sms()));
    border_count_kernel<<<g, 256, 0, s>>>(n, inF, b.inB, st);
    note_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_border_diff(cudaStream_t s, int64_t n, const uint8_t *inF, const BorderBuffers &b, int64_t kb,
                               DevStatus *st) {
    border_diff_kernel<<<1, kBThreads, 0, s>>>(n, inF, b.inB, b.Bl, kb, b.Ul, b.Al, b.Rpos, st);
    note_launches(1);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_border_setup(cudaStream_t s, const T *G, int64_t ldg, const T *L, int64_t kb, int64_t lds,
                                int a, int r, const BorderBuffers &b, DevStatus *st) {
    T *Pt = static_cast<T *>(b.Pt);
    T *Z = static_cast<T *>(b.Z);
    const int64_t u = kb + a;
    cudaError_t e = cudaMemsetAsync(b.bad, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    if (a > 0) {
        const int64_t work = (kb + a) * a;
        const int g = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(work, 256), num_sms() * 8));
        border_gather_kernel<T><<<g, 256, 0, s>>>(G, ldg, b.Bl, kb, b.Al, a, Pt, b.ldp, b.GAA);
        note_launches(1);
        e = launch_trsv_multi<T>(s, L, kb, lds, Pt, b.ldp, a, b.multi, st, 1);
        if (e != cudaSuccess) return e;
        border_schur_kernel<T><<<a * a, 256, 0, s>>>(Pt, b.ldp, kb, a, b.GAA, b.Lq);
        border_chol_kernel<<<1, 32, 0, s>>>(b.Lq, a, b.bad);
        note_launches(2);
    }
    if (r > 0) {
        const int g = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(u * r, 256), num_sms() * 8));
        border_unit_kernel<T><<<g, 256, 0, s>>>(Z, u, b.ldz, r, b.Rpos);
        note_launches(1);
        // the r columns of Z side by side: forward, border step, backward
        e = launch_trsv_multi<T>(s, L, kb, lds, Z, b.ldz, r, b.multi, st, 1);
        if (e == cudaSuccess && a > 0) {
            border_mid_kernel<T><<<dim3(1, (unsigned)r), kMidThreads, 0, s>>>(Z, kb, a, Pt, b.ldp, b.Lq, b.ldz);
            note_launches(1);
        }
        if (e == cudaSuccess) e = launch_trsv_multi<T>(s, L, kb, lds, Z, b.ldz, r, b.multi, st, 2);
        if (e != cudaSuccess) return e;
        border_cap_factor_kernel<T><<<1, 256, 0, s>>>(Z, b.ldz, r, b.Rpos, b.Lc, b.bad);
        note_launches(1);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_border_solve(cudaStream_t s, const T *L, int64_t kb, int64_t lds, int a, int r,
                                const BorderBuffers &b, T *z, void *trsv_scratch, DevStatus *st) {
    const int64_t u = kb + a;
    cudaError_t e = launch_trsv_fwd<T>(s, L, kb, lds, z, trsv_scratch, st);
    if (e == cudaSuccess && a > 0) {
        border_mid_kernel<T><<<1, kMidThreads, 0, s>>>(z, kb, a, static_cast<const T *>(b.Pt), b.ldp, b.Lq, 0);
        note_launches(1);
    }
    if (e == cudaSuccess) e = launch_trsv_bwd<T>(s, L, kb, lds, z, trsv_scratch, st);
    if (e == cudaSuccess && r > 0) {
        border_cap_mu_kernel<T><<<1, 32, 0, s>>>(z, r, b.Rpos, b.Lc, b.mu);
        const int g = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(u, 256), num_sms() * 2));
        border_cap_apply_kernel<T><<<g, 256, 0, s>>>(z, u, r, static_cast<const T *>(b.Z), b.ldz, b.mu);
        note_launches(2);
    }
    return e == cudaSuccess ? cudaGetLastError() : e;
}

template cudaError_t launch_border_setup<float>(cudaStream_t, const float *, int64_t, const float *, int64_t,
                                                int64_t, int, int, const BorderBuffers &, DevStatus *);
template cudaError_t launch_border_setup<double>(cudaStream_t, const double *, int64_t, const double *, int64_t,
                                                 int64_t, int, int, const BorderBuffers &, DevStatus *);
template cudaError_t launch_border_solve<float>(cudaStream_t, const float *, int64_t, int64_t, int, int,
                                                const BorderBuffers &, float *, void *, DevStatus *);
template cudaError_t launch_border_solve<double>(cudaStream_t, const double *, int64_t, int64_t, int, int,
                                                 const BorderBuffers &, double *, void *, DevStatus *);

}  // namespace tsnnls

TSNNLS_CHECK_UNIT("border")
