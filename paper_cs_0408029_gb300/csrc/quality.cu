// Quality figures of a finished solve, computed once on the device after the
// last pivot (tsnnls_info.kkt_viol and tsnnls_info.rel_resid_change):
//
//   kkt_viol          largest violation of the LCP conditions of Eq. 3 at the
//                     returned x, with y = A^T (A x - b):
//                       max(-min x, -min y, max_i |x_i y_i| / max(1, |x_i|)),
//                     divided by ||A^T b||_2 (the scale of the 1e-10 target)
//   rel_resid_change  ||A dx||_2 / ||b - A x||_2 for the last refinement
//                     correction dx: how much the last step still moved the
//                     FP64 residual (0 when no refinement step was taken)
//
// Inputs are the final x, s = A^T (b - A x) and r = b - A x that the pivot
// loop leaves behind, so the only extra products are one scatter of dx and
// one SpMV.  Two launches reduce: per-CTA partials, then one CTA that adds
// them in index order (deterministic, no floating-point atomics).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>

#include "check.cuh"
#include "common.cuh"

namespace tsnnls {

namespace {

constexpr int kQT = 256;
constexpr int kQParts = 5;  // per CTA: sum r^2, sum q^2, sum c^2, kkt max, (spare)

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

template <typename T>
__global__ void scatter_list_kernel(int64_t len, const T *__restrict__ vals, const int32_t *__restrict__ list,
                                    double *__restrict__ d, int64_t n) {
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < len;
         a += (int64_t)gridDim.x * blockDim.x) {
        const int32_t j = list[a];
        if (j >= 0 && TS_IN(j, n)) d[j] = (double)vals[a];
    }
}

template <typename V>
__global__ void scatter_scaled_kernel(int64_t n, const V *__restrict__ D, const V *__restrict__ z,
                                      const uint8_t *__restrict__ inF, double *__restrict__ d) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * blockDim.x)
        d[j] = inF[j] ? (double)D[j] * (double)z[j] : 0.0;
}

__global__ void __launch_bounds__(kQT)
    quality_part_kernel(int64_t m, int64_t n, const double *__restrict__ x, const double *__restrict__ sv,
                        const double *__restrict__ c, const double *__restrict__ r,
                        const double *__restrict__ q, double *__restrict__ part) {
    __shared__ double sh[kQParts][kQT / 32];
    double rr = 0.0, qq = 0.0, cc = 0.0, viol = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += stride) {
        const double ri = r[i];
        rr += ri * ri;
        if (q) qq += q[i] * q[i];
    }
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += stride) {
        const double xj = x[j], yj = -sv[j], cj = c[j];
        cc += cj * cj;
        viol = fmax(viol, fmax(-xj, -yj));
        viol = fmax(viol, fabs(xj * yj) / fmax(1.0, fabs(xj)));
    }
    rr = warp_sum(rr);
    qq = warp_sum(qq);
    cc = warp_sum(cc);
    viol = warp_max(viol);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        sh[0][warp] = rr;
        sh[1][warp] = qq;
        sh[2][warp] = cc;
        sh[3][warp] = viol;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0, e = 0.0, v = 0.0;
        for (int w = 0; w < kQT / 32; ++w) {
            a += sh[0][w];
            b += sh[1][w];
            e += sh[2][w];
            v = fmax(v, sh[3][w]);
        }
        double *p = part + (int64_t)blockIdx.x * kQParts;
        p[0] = a;
        p[1] = b;
        p[2] = e;
        p[3] = v;
        p[4] = 0.0;
    }
}

__global__ void __launch_bounds__(32)
    quality_finish_kernel(const double *__restrict__ part, int count, int have_q, DevStatus *st) {
    if (threadIdx.x != 0) return;
    double rr = 0.0, qq = 0.0, cc = 0.0, viol = 0.0;
    for (int b = 0; b < count; ++b) {
        const double *p = part + (int64_t)b * kQParts;
        rr += p[0];
        qq += p[1];
        cc += p[2];
        viol = fmax(viol, p[3]);
    }
    const double cn = sqrt(cc);
    st->kkt_viol = cn > 0.0 ? viol / cn : viol;
    const double rn = sqrt(rr), qn = sqrt(qq);
    st->resid_change = !have_q || qn == 0.0 ? 0.0 : (rn > 0.0 ? qn / rn : INFINITY);
}

}  // namespace

int quality_parts() { return std::max(1, std::min(num_sms() * 4, 1024)); }

size_t quality_scratch_bytes(int64_t m, int64_t n) {
    const size_t part = sizeof(double) * kQParts * 1024;
    return round_up((int64_t)(sizeof(double) * n), 256) + round_up((int64_t)(sizeof(double) * m), 256) + part;
}

template <typename T>
cudaError_t launch_quality(cudaStream_t s, int64_t m, int64_t n, const int64_t *row_ptr, const int32_t *col,
                           const double *val, double avg_row, const double *x, const double *sv,
                           const double *c, const double *r, const T *delta, const int32_t *list,
                           int64_t len, void *scratch, DevStatus *st) {
    double *d = static_cast<double *>(scratch);
    double *q = d + round_up(n, 32);
    double *part = q + round_up(m, 32);
    const bool have_q = delta != nullptr && len > 0;
    if (have_q) {
        cudaError_t e = cudaMemsetAsync(d, 0, sizeof(double) * n, s);
        if (e != cudaSuccess) return e;
        const int g = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(len, 256), num_sms() * 8));
        scatter_list_kernel<T><<<g, 256, 0, s>>>(len, delta, list, d, n);
        note_launches(1);
        e = launch_spmv(s, m, row_ptr, col, val, 1.0, d, n, 0.0, nullptr, q, avg_row);
        if (e != cudaSuccess) return e;
    }
    const int parts = quality_parts();
    quality_part_kernel<<<parts, kQT, 0, s>>>(m, n, x, sv, c, r, have_q ? q : nullptr, part);
    quality_finish_kernel<<<1, 32, 0, s>>>(part, parts, have_q ? 1 : 0, st);
    note_launches(2);
    return cudaGetLastError();
}

template <typename V>
cudaError_t launch_quality_scaled(cudaStream_t s, int64_t m, int64_t n, const int64_t *row_ptr,
                                  const int32_t *col, const double *val, double avg_row, const double *x,
                                  const double *sv, const double *c, const double *r, const V *D,
                                  const V *z, const uint8_t *inF, bool have_delta, void *scratch,
                                  DevStatus *st) {
    double *d = static_cast<double *>(scratch);
    double *q = d + round_up(n, 32);
    double *part = q + round_up(m, 32);
    if (have_delta) {
        const int g = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(n, 256), num_sms() * 8));
        scatter_scaled_kernel<V><<<g, 256, 0, s>>>(n, D, z, inF, d);
        note_launches(1);
        cudaError_t e = launch_spmv(s, m, row_ptr, col, val, 1.0, d, n, 0.0, nullptr, q, avg_row);
        if (e != cudaSuccess) return e;
    }
    const int parts = quality_parts();
    quality_part_kernel<<<parts, kQT, 0, s>>>(m, n, x, sv, c, r, have_delta ? q : nullptr, part);
    quality_finish_kernel<<<1, 32, 0, s>>>(part, parts, have_delta ? 1 : 0, st);
    note_launches(2);
    return cudaGetLastError();
}

template cudaError_t launch_quality<float>(cudaStream_t, int64_t, int64_t, const int64_t *, const int32_t *,
                                           const double *, double, const double *, const double *,
                                           const double *, const double *, const float *, const int32_t *,
                                           int64_t, void *, DevStatus *);
template cudaError_t launch_quality<double>(cudaStream_t, int64_t, int64_t, const int64_t *, const int32_t *,
                                            const double *, double, const double *, const double *,
                                            const double *, const double *, const double *, const int32_t *,
                                            int64_t, void *, DevStatus *);
template cudaError_t launch_quality_scaled<float>(cudaStream_t, int64_t, int64_t, const int64_t *,
                                                  const int32_t *, const double *, double, const double *,
                                                  const double *, const double *, const double *, const float *,
                                                  const float *, const uint8_t *, bool, void *, DevStatus *);
template cudaError_t launch_quality_scaled<double>(cudaStream_t, int64_t, int64_t, const int64_t *,
                                                   const int32_t *, const double *, double, const double *,
                                                   const double *, const double *, const double *,
                                                   const double *, const double *, const uint8_t *, bool,
                                                   void *, DevStatus *);

}  // namespace tsnnls

TSNNLS_CHECK_UNIT("quality")
