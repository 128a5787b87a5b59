// Supernodal sparse Cholesky of the cached normal equations on the GPU
// (Section 3: TAUCS factors A^T A as a sparse matrix when it is sparse).
// The structure comes from sparse_sym.cpp, analysed once per problem; every
// pivot factors
//     G' = P (A^T A)_{FF} P^T  (+ the identity on the variables in G)
// so one structure serves every F: a variable outside F keeps a unit column,
// and its entry of every solve is 0.
//
// Factor: one persistent kernel, one CTA per SM.  CTAs take supernodes in
// postorder by ticket; a supernode waits (bounded) until every earlier
// supernode that updates it is done, which is always a CTA that took a
// smaller ticket and so is running or finished.  It then
//   - clears its panel (rows x width, column-major) and assembles the
//     entries of G' in its columns;
//   - subtracts, descendant by descendant in ascending order, L_d(R, :)
//     L_d(C, :)^T for the descendant's rows R at or below its first column
//     and C inside its columns (scattered through a row -> panel-row map);
//   - factors and inverts its diagonal block in shared memory with the dense
//     block code of the blocked factorisation (dense_block.cuh), and forms
//     the rows below as X = B W^T, 32 rows at a time;
//   - publishes a done flag (release).
// Solves: the same ticketing, forward in postorder (a supernode gathers the
// updates of its descendants, then applies W), backward in reverse
// postorder (it gathers the solved entries of its rows below, then W^T).
// Every sum runs in a fixed order, so results are reproducible.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cuda/atomic>
#include <vector>

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

// first p in [lo, hi) with rows[p] >= v
__device__ __forceinline__ int64_t sp_lower_bound(const int32_t *rows, int64_t lo, int64_t hi, int32_t v) {
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (rows[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
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
        permF[p] = inF[j] ? j : -1;
    }
}

template <typename T, int NB>
struct SpSmem {
    static constexpr int P = NB + 4;
    static constexpr size_t bytes = sizeof(T) * (2 * (size_t)NB * P + (size_t)NB * 36);
};

template <typename T, int NB>
__global__ void __launch_bounds__(256, 1)
    sp_factor_kernel(SpDev D, const uint8_t *__restrict__ inF, T *__restrict__ L, T *__restrict__ Wa, DevStatus *st) {
    using SM = SpSmem<T, NB>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T(*A)[NB + 4] = reinterpret_cast<T(*)[NB + 4]>(smem_raw);
    T(*W)[NB + 4] = reinterpret_cast<T(*)[NB + 4]>(smem_raw + sizeof(T) * NB * SM::P);
    T(*Bs)[36] = reinterpret_cast<T(*)[36]>(smem_raw + 2 * sizeof(T) * NB * SM::P);  // Bs[t][r]
    __shared__ int sh_s, ok_sh, bad_sh;
    __shared__ __align__(16) T col[2][32];
    const int tid = threadIdx.x;
    int32_t *map = D.map + (int64_t)blockIdx.x * D.n;
    for (;;) {
        if (tid == 0) sh_s = atomicAdd(D.ticket, 1);
        __syncthreads();
        const int64_t s = sh_s;
        if (s >= D.ns) return;
        if (!sp_wait_all(D, D.flags, D.dlist, D.d_off[s], D.d_off[s + 1], st, &ok_sh)) return;
        const int32_t f = D.sn_first[s], w = D.sn_first[s + 1] - f;
        const int32_t *rows = D.rows + D.rows_off[s];
        const int64_t h = D.rows_off[s + 1] - D.rows_off[s], ld = (h + 3) / 4 * 4;
        T *P = L + D.L_off[s];
        for (int64_t i = tid; i < h; i += 256) map[rows[i]] = (int32_t)i;
        for (int64_t e = tid; e < ld * w; e += 256) P[e] = T(0);
        __syncthreads();
        // G' in this supernode's columns
        for (int64_t p = D.gptr[f] + tid; p < D.gptr[f + w]; p += 256) {
            const int32_t io = D.grow_orig[p], jo = D.gcol_orig[p];
            const T v = (inF[io] && inF[jo]) ? (T)D.gval[p] : (io == jo ? T(1) : T(0));
            L[D.gpos[p]] = v;
        }
        __syncthreads();
        // updates from the descendants, one after another
        for (int64_t di = D.d_off[s]; di < D.d_off[s + 1]; ++di) {
            const int32_t d = D.dlist[di];
            const int32_t wd = D.sn_first[d + 1] - D.sn_first[d];
            const int64_t rb = D.rows_off[d], hd = D.rows_off[d + 1] - rb, ldd = (hd + 3) / 4 * 4;
            const int32_t *rd = D.rows + rb;
            const T *Ld = L + D.L_off[d];
            const int64_t p0 = sp_lower_bound(rd, wd, hd, f), p1 = sp_lower_bound(rd, p0, hd, f + w);
            const int64_t M = hd - p0, N = p1 - p0;
            const int64_t mt = (M + 3) / 4, nt = (N + 3) / 4;
            for (int64_t tile = tid; tile < mt * nt; tile += 256) {
                const int64_t tr = tile % mt, tc = tile / mt;
                const int64_t pa = p0 + 4 * tr, qa = p0 + 4 * tc;
                if (pa + 3 < qa) continue;  // above the diagonal of the target
                T acc[4][4] = {};
                for (int k = 0; k < wd; ++k) {
                    const T *lk = Ld + (int64_t)k * ldd;
                    T x[4], y[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        x[u] = pa + u < hd ? lk[pa + u] : T(0);
                        y[u] = qa + u < p1 ? lk[qa + u] : T(0);
                    }
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b) acc[a][b] += x[a] * y[b];
                }
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int64_t q = qa + b;
                    if (q >= p1) break;
                    T *pc = P + (int64_t)(rd[q] - f) * ld;
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        const int64_t p = pa + a;
                        if (p < hd && p >= q) {
                            // rows of a descendant at or below this supernode's first
                            // column are rows of this supernode (elimination tree)
                            const int32_t loc = map[rd[p]];
                            if (loc >= 0 && loc < h) pc[loc] -= acc[a][b];
                        }
                    }
                }
            }
            __syncthreads();
        }
        // the diagonal block: factor and inverse in shared memory
        if (tid == 0) bad_sh = 0;
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
        if (tid == 0 && bad_sh && bad_sh <= w) atomicCAS(&st->chol_info, 0, (int32_t)(f + bad_sh));
        T *Ws = Wa + D.W_off[s];
        for (int e = tid; e < w * w; e += 256) {
            const int c = e / w, r = e % w;
            if (r >= c) P[(int64_t)c * ld + r] = A[c][r];
            Ws[e] = W[c][r];  // W(r, c), column-major, w x w
        }
        // rows below: X = B W^T, 32 rows at a time through shared memory
        for (int64_t r0 = w; r0 < h; r0 += 32) {
            __syncthreads();
            for (int e = tid; e < w * 32; e += 256) {
                const int t = e / 32, rr = e % 32;
                Bs[t][rr] = r0 + rr < h ? P[(int64_t)t * ld + r0 + rr] : T(0);
            }
            __syncthreads();
            for (int e = tid; e < w * 32; e += 256) {
                const int c = e / 32, rr = e % 32;
                T acc = T(0);
                for (int t = 0; t <= c; ++t) acc += Bs[t][rr] * W[t][c];  // W(c, t), zero for t > c
                if (r0 + rr < h) P[(int64_t)c * ld + r0 + rr] = acc;
            }
        }
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            sp_flag_store(D.flags + s, 1);
        }
    }
}

constexpr int kSpT = 128;  // threads of a solve CTA

template <typename T>
__global__ void __launch_bounds__(kSpT)
    sp_fwd_kernel(SpDev D, const T *__restrict__ L, const T *__restrict__ Wa, T *v, DevStatus *st) {
    __shared__ T t_sh[128];
    __shared__ int sh_s, ok_sh;
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) sh_s = atomicAdd(D.ticket, 1);
        __syncthreads();
        const int64_t s = sh_s;
        if (s >= D.ns) return;
        if (!sp_wait_all(D, D.flags, D.dlist, D.d_off[s], D.d_off[s + 1], st, &ok_sh)) return;
        const int32_t f = D.sn_first[s], w = D.sn_first[s + 1] - f;
        if (tid < w) t_sh[tid] = __ldcg(v + f + tid);
        __syncthreads();
        for (int64_t di = D.d_off[s]; di < D.d_off[s + 1]; ++di) {
            const int32_t d = D.dlist[di];
            const int32_t fd = D.sn_first[d], wd = D.sn_first[d + 1] - fd;
            const int64_t rb = D.rows_off[d], hd = D.rows_off[d + 1] - rb, ldd = (hd + 3) / 4 * 4;
            const int32_t *rd = D.rows + rb;
            const T *Ld = L + D.L_off[d];
            const int64_t p0 = sp_lower_bound(rd, wd, hd, f), p1 = sp_lower_bound(rd, p0, hd, f + w);
            for (int64_t q = p0 + tid; q < p1; q += kSpT) {
                T acc = T(0);
                for (int k = 0; k < wd; ++k) acc += Ld[(int64_t)k * ldd + q] * __ldcg(v + fd + k);
                t_sh[rd[q] - f] -= acc;
            }
            __syncthreads();
        }
        const T *Ws = Wa + D.W_off[s];
        T y = T(0);
        if (tid < w)
            for (int c = 0; c <= tid; ++c) y += Ws[(int64_t)c * w + tid] * t_sh[c];  // W(r, c), c <= r
        if (tid < w) v[f + tid] = y;
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
    __shared__ T t_sh[128];
    __shared__ T part[kSpT];
    __shared__ int sh_s, ok_sh;
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) sh_s = atomicAdd(D.ticket, 1);
        __syncthreads();
        if (sh_s >= D.ns) return;
        const int64_t s = D.ns - 1 - sh_s;  // reverse postorder
        if (!sp_wait_all(D, D.flags, D.alist, D.a_off[s], D.a_off[s + 1], st, &ok_sh)) return;
        const int32_t f = D.sn_first[s], w = D.sn_first[s + 1] - f;
        const int32_t *rows = D.rows + D.rows_off[s];
        const int64_t h = D.rows_off[s + 1] - D.rows_off[s], ld = (h + 3) / 4 * 4;
        const T *Ls = L + D.L_off[s];
        // t_c = y_c - sum_{p >= w} L(p, c) x(rows[p]): G groups of threads per
        // column share the rows below, partial sums added in group order
        const int G = max(1, kSpT / w);
        const int c = tid % w, g = tid / w;
        T acc = T(0);
        if (g < G)
            for (int64_t p = w + g; p < h; p += G) acc += Ls[(int64_t)c * ld + p] * __ldcg(v + rows[p]);
        part[tid] = acc;
        __syncthreads();
        if (tid < w) {
            T t = __ldcg(v + f + tid);
            for (int q = 0; q < G; ++q) t -= part[q * w + tid];
            t_sh[tid] = t;
        }
        __syncthreads();
        const T *Ws = Wa + D.W_off[s];
        T x = T(0);
        if (tid < w)
            for (int cc = tid; cc < w; ++cc) x += Ws[(int64_t)tid * w + cc] * t_sh[cc];  // W(cc, r), cc >= r
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
size_t SparseChol<T>::device_bytes(const SparseSym &S, int ctas) {
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t ns = (size_t)S.ns, n = (size_t)S.n, ng = S.grow.size();
    size_t b = 0;
    b += up(4 * (ns + 1)) + up(8 * (ns + 1)) + up(4 * S.rows.size()) + 4 * up(8 * (ns + 1));
    b += up(4 * S.dlist.size() + 4) + up(4 * S.alist.size() + 4);
    b += up(4 * n) + up(8 * (n + 1)) + 2 * up(4 * ng) + up(8 * ng) + up(8 * ng);  // perm, gptr, rows/cols, gpos, gval
    b += up(sizeof(T) * (size_t)S.L_off[ns]) + up(sizeof(T) * (size_t)S.W_off[ns]);
    b += up(4 * n * (size_t)ctas) + up(4 * ns) + up(16) + up(4 * n) + up(sizeof(T) * n);
    return b + 256;
}

template <typename T>
cudaError_t SparseChol<T>::setup(const SparseSym &S, void *mem, cudaStream_t s, const int64_t *col_ptr,
                                 const int32_t *row_idx, const double *cval) {
    ctas = std::max(1, num_sms());
    char *p = static_cast<char *>(mem);
    auto take = [&](size_t b) {
        p = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(p) + 255) / 256 * 256);
        char *q = p;
        p += std::max<size_t>(b, 1);
        return q;
    };
    const size_t ns = (size_t)S.ns, n = (size_t)S.n, ng = S.grow.size();
    D.n = S.n;
    D.ns = S.ns;
    int32_t *sn_first = (int32_t *)take(4 * (ns + 1));
    int64_t *rows_off = (int64_t *)take(8 * (ns + 1));
    int32_t *rows = (int32_t *)take(4 * S.rows.size());
    int64_t *L_off = (int64_t *)take(8 * (ns + 1));
    int64_t *W_off = (int64_t *)take(8 * (ns + 1));
    int64_t *d_off = (int64_t *)take(8 * (ns + 1));
    int64_t *a_off = (int64_t *)take(8 * (ns + 1));
    int32_t *dlist = (int32_t *)take(4 * S.dlist.size() + 4);
    int32_t *alist = (int32_t *)take(4 * S.alist.size() + 4);
    int32_t *perm = (int32_t *)take(4 * n);
    int64_t *gptr = (int64_t *)take(8 * (n + 1));
    int32_t *grow_orig = (int32_t *)take(4 * ng);
    int32_t *gcol_orig = (int32_t *)take(4 * ng);
    int64_t *gpos = (int64_t *)take(8 * ng);
    double *gval = (double *)take(8 * ng);
    Lmem = (T *)take(sizeof(T) * (size_t)S.L_off[ns]);
    Wmem = (T *)take(sizeof(T) * (size_t)S.W_off[ns]);
    int32_t *map = (int32_t *)take(4 * n * (size_t)ctas);
    int32_t *flags = (int32_t *)take(4 * ns);
    int32_t *ctl = (int32_t *)take(16);
    permF = (int32_t *)take(4 * n);
    vec = (T *)take(sizeof(T) * n);
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
    up(d_off, S.d_off.data(), 8 * (ns + 1));
    up(a_off, S.a_off.data(), 8 * (ns + 1));
    up(dlist, S.dlist.data(), 4 * S.dlist.size());
    up(alist, S.alist.data(), 4 * S.alist.size());
    up(perm, S.perm.data(), 4 * n);
    up(gptr, S.gptr.data(), 8 * (n + 1));
    up(grow_orig, S.gpair_orig_row.data(), 4 * ng);
    up(gcol_orig, gcol.data(), 4 * ng);
    up(gpos, S.gpos.data(), 8 * ng);
    if (e != cudaSuccess) return e;
    // the host vectors must outlive the copies: wait for them here (setup runs once per problem)
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    D.sn_first = sn_first;
    D.rows_off = rows_off;
    D.rows = rows;
    D.L_off = L_off;
    D.W_off = W_off;
    D.d_off = d_off;
    D.a_off = a_off;
    D.dlist = dlist;
    D.alist = alist;
    D.perm = perm;
    D.gptr = gptr;
    D.grow_orig = grow_orig;
    D.gcol_orig = gcol_orig;
    D.gpos = gpos;
    D.gval = gval;
    D.map = map;
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
    if (e != cudaSuccess) return e;
    sp_factor_kernel<T, NB><<<ctas, 256, smem, s>>>(D, inF, Lmem, Wmem, st);
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
    cudaError_t e = reset(s);
    if (e != cudaSuccess) return e;
    sp_fwd_kernel<T><<<g, kSpT, 0, s>>>(D, Lmem, Wmem, v, st);
    e = reset(s);
    if (e != cudaSuccess) return e;
    sp_bwd_kernel<T><<<g, kSpT, 0, s>>>(D, Lmem, Wmem, v, st);
    note_launches(2);
    return cudaGetLastError();
}

template struct SparseChol<float>;
template struct SparseChol<double>;

}  // namespace tsnnls
