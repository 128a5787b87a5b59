// Sparse kernels: CSR -> CSC transpose, the A^T A / A^T b precompute of
// Section 3 ("A^T A_ij is the dot product of the i-th and j-th columns",
// formed once and cached), and the FP64 CSR mat-vec used for Eq. 5 and for
// the refinement residuals.
//
// All sums run in a fixed order, so every output is bit-reproducible from
// run to run and independent of what else shares the GPU.
#include <cuda_runtime.h>
#include <stdint.h>

#include "check.cuh"
#include "common.cuh"

namespace tsnnls {

// ---------------------------------------------------------------------------
// CSR -> CSC

__global__ void csc_count_kernel(int64_t nnz, int64_t n, const int32_t *__restrict__ col,
                                 int32_t *__restrict__ cnt) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t j = col[e];
        if (TS_IN(j, n)) atomicAdd(&cnt[j], 1);
    }
}

// Exclusive scan of cnt[0..n) into ptr[0..n] (ptr[n] = total) by one CTA of
// 1024 threads walking the array in tiles; next[] receives a copy of ptr.
__global__ void __launch_bounds__(1024) csc_scan_kernel(int64_t n, const int32_t *__restrict__ cnt,
                                                        int64_t *__restrict__ ptr,
                                                        int64_t *__restrict__ next) {
    __shared__ int64_t warp_sums[32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t base = 0; base < n; base += 1024) {
        int64_t i = base + threadIdx.x;
        int64_t v = i < n ? cnt[i] : 0;
        int64_t incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) warp_sums[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int64_t w = warp_sums[lane];
            for (int o = 1; o < 32; o <<= 1) {
                int64_t t = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += t;
            }
            warp_sums[lane] = w;
        }
        __syncthreads();
        int64_t excl = carry + incl - v + (warp > 0 ? warp_sums[warp - 1] : 0);
        if (i < n) {
            ptr[i] = excl;
            next[i] = excl;
        }
        __syncthreads();
        if (threadIdx.x == 1023) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        ptr[n] = carry;
        next[n] = carry;
    }
}

__global__ void csc_fill_kernel(int64_t m, int64_t n, int64_t nnz, const int64_t *__restrict__ row_ptr,
                                const int32_t *__restrict__ col, const double *__restrict__ val,
                                int64_t *__restrict__ next, int32_t *__restrict__ row_idx,
                                double *__restrict__ cval) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m;
         r += (int64_t)gridDim.x * blockDim.x) {
        for (int64_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e) {
            const int32_t j = col[e];
            if (!TS_IN(j, n)) continue;
            unsigned long long p = atomicAdd((unsigned long long *)&next[j], 1ull);
            if (!TS_IN(p, nnz)) continue;
            row_idx[p] = (int32_t)r;
            cval[p] = val[e];
        }
    }
}

// The fill above leaves each column's entries in arrival order.  Put them in
// ascending row order: every entry's final slot is its rank among the
// column's (distinct) rows.  One CTA per column; long columns are ranked
// straight from global memory.
constexpr int kSortCap = 2048;

__global__ void __launch_bounds__(256) csc_sort_kernel(int64_t n, const int64_t *__restrict__ ptr,
                                                       int32_t *__restrict__ row_idx,
                                                       double *__restrict__ cval) {
    __shared__ int32_t rows[kSortCap];
    __shared__ double vals[kSortCap];
    for (int64_t j = blockIdx.x; j < n; j += gridDim.x) {
        const int64_t a = ptr[j];
        const int64_t len = ptr[j + 1] - a;
        if (len <= 1) continue;
        if (len <= kSortCap) {
            for (int64_t q = threadIdx.x; q < len; q += blockDim.x) {
                rows[q] = row_idx[a + q];
                vals[q] = cval[a + q];
            }
            __syncthreads();
            for (int64_t q = threadIdx.x; q < len; q += blockDim.x) {
                const int32_t r = rows[q];
                int64_t rank = 0;
                for (int64_t t = 0; t < len; ++t) rank += rows[t] < r;
                row_idx[a + rank] = r;
                cval[a + rank] = vals[q];
            }
            __syncthreads();
        } else if (threadIdx.x == 0) {
            // insertion sort in place (rare: columns longer than kSortCap)
            for (int64_t q = 1; q < len; ++q) {
                const int32_t r = row_idx[a + q];
                const double v = cval[a + q];
                int64_t t = q - 1;
                while (t >= 0 && row_idx[a + t] > r) {
                    row_idx[a + t + 1] = row_idx[a + t];
                    cval[a + t + 1] = cval[a + t];
                    --t;
                }
                row_idx[a + t + 1] = r;
                cval[a + t + 1] = v;
            }
        }
        __syncthreads();
    }
}

cudaError_t launch_csr_to_csc(cudaStream_t s, int64_t m, int64_t n, int64_t nnz,
                              const int64_t *row_ptr, const int32_t *col, const double *val,
                              int64_t *col_ptr, int32_t *row_idx, double *cval, int32_t *work,
                              int64_t *scan_work) {
    cudaError_t e = cudaMemsetAsync(work, 0, sizeof(int32_t) * (size_t)(n + 1), s);
    if (e != cudaSuccess) return e;
    if (nnz > 0) {
        int g = (int)std::min<int64_t>(cdiv(nnz, 256), num_sms() * 16);
        csc_count_kernel<<<g, 256, 0, s>>>(nnz, n, col, work);
        note_launches(1);
    }
    csc_scan_kernel<<<1, 1024, 0, s>>>(n, work, col_ptr, scan_work);
    note_launches(1);
    if (nnz > 0) {
        int g = (int)std::min<int64_t>(cdiv(m, 128), num_sms() * 16);
        csc_fill_kernel<<<g, 128, 0, s>>>(m, n, nnz, row_ptr, col, val, scan_work, row_idx, cval);
        note_launches(1);
        int gs = (int)std::min<int64_t>(n, num_sms() * 8);
        csc_sort_kernel<<<gs, 256, 0, s>>>(n, col_ptr, row_idx, cval);
        note_launches(1);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Section 3 precompute: G = A^T A (lower triangle), c = A^T b.
//
// G(:, j) = sum over the rows r holding a_rj of a_rj * A(r, :).  One CTA owns
// output column j restricted to a chunk of rows [i0, i1) with i0 >= j.  It
// stages the (i, a_rj * a_ri) contributions of up to 256 rows r at a time in
// shared memory, then a single warp adds them into an FP64 accumulator row
// by row, in ascending r: the entries of one CSR row hit distinct i, so the
// warp's lanes never collide and every G_ij is summed in the same order on
// every run.  The accumulator is written once, coalesced, as T.

constexpr int kGramThreads = 256;
constexpr int kGramChunk = 2048;   // output rows per CTA (FP64 accumulator: 16 KB)
constexpr int kGramPairs = 1024;   // staged contributions per window

template <typename T>
__global__ void __launch_bounds__(kGramThreads)
    gram_kernel(int64_t n, const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                const double *__restrict__ val, const int64_t *__restrict__ col_ptr,
                const int32_t *__restrict__ row_idx, const double *__restrict__ cval,
                const double *__restrict__ b, T *__restrict__ G, int64_t ldg,
                double *__restrict__ c) {
    __shared__ double acc[kGramChunk];
    __shared__ int32_t pr_i[kGramPairs];
    __shared__ double pr_v[kGramPairs];
    __shared__ int64_t q_start[kGramThreads];
    __shared__ int32_t q_cnt[kGramThreads];
    __shared__ int64_t q_off[kGramThreads + 1];
    __shared__ double q_v[kGramThreads];
    __shared__ double red[kGramThreads];

    const int64_t j = blockIdx.x;
    const int64_t i0 = j + (int64_t)blockIdx.y * kGramChunk;
    if (i0 >= n) return;
    const int64_t i1 = min(n, i0 + (int64_t)kGramChunk);
    const int tid = threadIdx.x;
    for (int t = tid; t < kGramChunk; t += kGramThreads) acc[t] = 0.0;

    const int64_t qa = col_ptr[j], qe = col_ptr[j + 1];
    double csum = 0.0;  // thread 0 only: c_j in ascending row order
    for (int64_t qb = qa; qb < qe; qb += kGramThreads) {
        const int64_t nq = min((int64_t)kGramThreads, qe - qb);
        // phase A: locate the part of each row r_q that falls in [i0, i1)
        if (tid < nq) {
            const int32_t r = row_idx[qb + tid];
            const double v = cval[qb + tid];
            int64_t lo = row_ptr[r], hi = row_ptr[r + 1];
            int64_t a = lo, z = hi;  // first entry with col >= i0
            while (a < z) {
                int64_t mid = (a + z) >> 1;
                if (col[mid] < i0) a = mid + 1; else z = mid;
            }
            int64_t e = a, z2 = hi;  // first entry with col >= i1
            while (e < z2) {
                int64_t mid = (e + z2) >> 1;
                if (col[mid] < i1) e = mid + 1; else z2 = mid;
            }
            q_start[tid] = a;
            q_cnt[tid] = (int32_t)(e - a);
            q_v[tid] = v;
            red[tid] = (blockIdx.y == 0) ? v * b[r] : 0.0;
        }
        __syncthreads();
        if (tid == 0) {
            int64_t o = 0;
            for (int q = 0; q < nq; ++q) {
                q_off[q] = o;
                o += q_cnt[q];
                csum += red[q];
            }
            q_off[nq] = o;
        }
        __syncthreads();
        const int64_t total = q_off[nq];
        // phases B/C over windows of staged pairs, in (q, entry) order
        for (int64_t w0 = 0; w0 < total; w0 += kGramPairs) {
            const int64_t wn = min((int64_t)kGramPairs, total - w0);
            for (int64_t p = tid; p < wn; p += kGramThreads) {
                const int64_t gp = w0 + p;
                int a = 0, z = (int)nq - 1;  // q with q_off[q] <= gp < q_off[q+1]
                while (a < z) {
                    int mid = (a + z + 1) >> 1;
                    if (q_off[mid] <= gp) a = mid; else z = mid - 1;
                }
                const int64_t e = q_start[a] + (gp - q_off[a]);
                pr_i[p] = (int32_t)(col[e] - i0);
                pr_v[p] = q_v[a] * val[e];
            }
            __syncthreads();
            if (tid < 32) {
                // walk the window row by row; lanes split one row's entries
                int q = 0;
                while (q < nq && q_off[q + 1] <= w0) ++q;
                for (; q < nq && q_off[q] < w0 + wn; ++q) {
                    const int64_t s0 = max(q_off[q], w0) - w0;
                    const int64_t s1 = min(q_off[q + 1], w0 + wn) - w0;
                    for (int64_t p = s0 + tid; p < s1; p += 32) {
                        const int32_t i = pr_i[p];
                        if (TS_IN(i, kGramChunk)) acc[i] += pr_v[p];
                    }
                    __syncwarp();
                }
            }
            __syncthreads();
        }
    }
    for (int64_t i = i0 + tid; i < i1; i += kGramThreads) G[i + j * ldg] = (T)acc[i - i0];
    if (blockIdx.y == 0 && tid == 0) c[j] = csum;
}

template <typename T>
cudaError_t launch_gram(cudaStream_t s, int64_t m, int64_t n, const int64_t *row_ptr,
                        const int32_t *col, const double *val, const int64_t *col_ptr,
                        const int32_t *row_idx, const double *cval, const double *b, T *G,
                        int64_t ldg, double *c) {
    (void)m;
    if (n == 0) return cudaSuccess;
    dim3 grid((unsigned)n, (unsigned)cdiv(n, kGramChunk));
    gram_kernel<T><<<grid, kGramThreads, 0, s>>>(n, row_ptr, col, val, col_ptr, row_idx, cval, b,
                                                   G, ldg, c);
    note_launches(1);
    return cudaGetLastError();
}

template cudaError_t launch_gram<float>(cudaStream_t, int64_t, int64_t, const int64_t *,
                                        const int32_t *, const double *, const int64_t *,
                                        const int32_t *, const double *, const double *, float *,
                                        int64_t, double *);
template cudaError_t launch_gram<double>(cudaStream_t, int64_t, int64_t, const int64_t *,
                                         const int32_t *, const double *, const int64_t *,
                                         const int32_t *, const double *, const double *,
                                         double *, int64_t, double *);

// ---------------------------------------------------------------------------
// FP64 CSR mat-vec: out = alpha * M x + beta * z.  TPR consecutive lanes own a
// row; each lane strides over the row and the group reduces by a fixed
// butterfly, so the summation order depends only on the row's length.

template <int TPR>
__global__ void __launch_bounds__(256)
    spmv_kernel(int64_t rows, const int64_t *__restrict__ ptr, const int32_t *__restrict__ idx,
                const double *__restrict__ val, double alpha, const double *__restrict__ x, int64_t xlen,
                double beta, const double *__restrict__ z, double *__restrict__ out) {
    // Lanes of one warp own 32/TPR consecutive rows; the loop runs on the
    // warp's first row so that every lane takes part in the shuffles.
    const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride_rows = ((int64_t)gridDim.x * blockDim.x) / TPR;
    const int sub = threadIdx.x % TPR;
    const int64_t warp_row0 = ((gtid >> 5) << 5) / TPR;
    const int64_t my_off = (gtid / TPR) - warp_row0;
    for (int64_t r0 = warp_row0; r0 < rows; r0 += stride_rows) {
        const int64_t r = r0 + my_off;
        double sum = 0.0;
        if (r < rows) {
            const int64_t a = ptr[r], e = ptr[r + 1];
            for (int64_t p = a + sub; p < e; p += TPR) {
                const int32_t j = idx[p];
                if (TS_IN(j, xlen)) sum += val[p] * x[j];
            }
        }
#pragma unroll
        for (int o = TPR / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o, TPR);
        if (sub == 0 && r < rows) out[r] = alpha * sum + (beta != 0.0 ? beta * z[r] : 0.0);
    }
}

cudaError_t launch_spmv(cudaStream_t s, int64_t rows, const int64_t *ptr, const int32_t *idx,
                        const double *val, double alpha, const double *x, int64_t xlen, double beta,
                        const double *z, double *out, double avg_nnz) {
    if (rows == 0) return cudaSuccess;
    auto grid_for = [&](int tpr) {
        return (int)std::min<int64_t>(cdiv(rows * tpr, 256), num_sms() * 32);
    };
    if (avg_nnz <= 3) {
        spmv_kernel<2><<<grid_for(2), 256, 0, s>>>(rows, ptr, idx, val, alpha, x, xlen, beta, z, out);
        note_launches(1);
    } else if (avg_nnz <= 6) {
        spmv_kernel<4><<<grid_for(4), 256, 0, s>>>(rows, ptr, idx, val, alpha, x, xlen, beta, z, out);
        note_launches(1);
    } else if (avg_nnz <= 12) {
        spmv_kernel<8><<<grid_for(8), 256, 0, s>>>(rows, ptr, idx, val, alpha, x, xlen, beta, z, out);
        note_launches(1);
    } else if (avg_nnz <= 24) {
        spmv_kernel<16><<<grid_for(16), 256, 0, s>>>(rows, ptr, idx, val, alpha, x, xlen, beta, z, out);
        note_launches(1);
    } else {
        spmv_kernel<32><<<grid_for(32), 256, 0, s>>>(rows, ptr, idx, val, alpha, x, xlen, beta, z, out);
        note_launches(1);
    }
    return cudaGetLastError();
}

}  // namespace tsnnls

namespace tsnnls {

__global__ void validate_kernel(int64_t m, int64_t n, int64_t nnz,
                                const int64_t *__restrict__ row_ptr,
                                const int32_t *__restrict__ col, const double *__restrict__ val,
                                const double *__restrict__ b, int32_t *bad) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = row_ptr[r], e = row_ptr[r + 1];
        int code = 0;
        if ((r == 0 && a != 0) || (r == m - 1 && e != nnz) || e < a || a < 0 || e > nnz) {
            code = 1;
        } else {
            if (!isfinite(b[r])) code = 4;
            for (int64_t p = a; p < e && !code; ++p) {
                const int32_t c = col[p];
                if (c < 0 || c >= n) code = 2;
                else if (p > a && c <= col[p - 1]) code = 3;
                else if (!isfinite(val[p])) code = 4;
            }
        }
        if (code) atomicCAS(bad, 0, code);
    }
}

cudaError_t launch_validate(cudaStream_t s, int64_t m, int64_t n, int64_t nnz,
                            const int64_t *row_ptr, const int32_t *col, const double *val,
                            const double *b, int32_t *bad) {
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(m, 256), num_sms() * 8));
    validate_kernel<<<g, 256, 0, s>>>(m, n, nnz, row_ptr, col, val, b, bad);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace tsnnls

TSNNLS_CHECK_UNIT("sparse")
