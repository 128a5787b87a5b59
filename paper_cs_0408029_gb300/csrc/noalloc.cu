// Allocation-free variant of the factor solve (tsnnls_chol_solve_noalloc).
//
// The blocked triangular solves need global scratch: per block row a "done"
// flag and a helper count, a ticket counter and an abort flag, one partial
// vector per CTA (chol_solve_scratch_bytes), plus a status word that records
// a timed-out wait.  tsnnls_chol_solve takes that scratch from its context,
// which allocates device memory.  This variant keeps it in a file-scope
// __device__ array instead (about 5.3 MB, sized for the largest k accepted),
// so a caller that must not allocate device memory can still run the solve
// on its own buffers.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "common.cuh"
#include "engine.h"

namespace tsnnls {
namespace {

// Largest k accepted: 65536 rows, i.e. 1024 blocks of 64 rows (FP64) or
// 512 of 128 (FP32).  The solve's scratch for that k is bounded by the
// flags, one 64-bit published word per row (FP32 only) and at most nine
// CTAs (a finisher and eight helpers) per block row, each with one partial
// vector of a block's rows (the FP64 partials bound the FP32 ones).
// chol_solve_scratch_bytes gives the exact figure, checked against this
// bound on every call.
constexpr int64_t kNoAllocMaxK = TSNNLS_NOALLOC_MAX_K;
constexpr int64_t kNoAllocBlocks = kNoAllocMaxK / 64;
constexpr size_t kFlagBytes = (size_t)((4 * (2 * kNoAllocBlocks + 2) + 255) / 256 * 256) +
                              (size_t)kNoAllocMaxK * 8 +  // FP32: one published word per row
                              (size_t)kNoAllocBlocks * 9 * 64 * sizeof(double);
constexpr size_t kScratchBytes = kFlagBytes + sizeof(DevStatus);

// Shared by every call on a device; it keeps the last call's contents.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  In host code
// the symbol names a host-side stand-in, so the address must come from
// cudaGetSymbolAddress, once per device, with that device current.  The
// address is kept for the life of the process: a cudaDeviceReset after the
// first call would leave it stale, so the entry point is not for use after
// a device reset.
int scratch_for_current_device(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e == cudaErrorNoDevice ? TSNNLS_ENODEV : TSNNLS_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return TSNNLS_ENODEV;
    std::lock_guard<std::mutex> g(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return TSNNLS_ECUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return TSNNLS_OK;
}

}  // namespace
}  // namespace tsnnls

using namespace tsnnls;

extern "C" int tsnnls_chol_solve_noalloc(int32_t precision, const void *L, int64_t k, int64_t lds,
                                         void *rhs, void *stream) {
    if (!L || !rhs || k < 0 || lds < k) return TSNNLS_EINVAL;
    if (k > kNoAllocMaxK) return TSNNLS_EINVAL;
    if (precision != TSNNLS_MIXED && precision != TSNNLS_FP64) return TSNNLS_EINVAL;
    if (k == 0) return TSNNLS_OK;
    void *base = nullptr;
    int st = scratch_for_current_device(&base);
    if (st != TSNNLS_OK) return st;
    const size_t need = chol_solve_scratch_bytes(k, precision == TSNNLS_FP64 ? sizeof(double) : sizeof(float));
    if (need > kFlagBytes) return TSNNLS_EINVAL;
    void *flags = base;
    DevStatus *status = reinterpret_cast<DevStatus *>(static_cast<char *>(base) + kFlagBytes);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // The flags are cleared by the solve launcher itself; the status word
    // still holds the previous call's result and must start at zero.
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(DevStatus), s);
    if (e == cudaSuccess)
        e = precision == TSNNLS_FP64
                ? launch_chol_solve<double>(s, static_cast<const double *>(L), k, lds,
                                            static_cast<double *>(rhs), flags, status)
                : launch_chol_solve<float>(s, static_cast<const float *>(L), k, lds,
                                           static_cast<float *>(rhs), flags, status);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return status_from_cuda(e);
    int32_t timed_out = 0;
    e = cudaMemcpy(&timed_out, &status->timeout, sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return status_from_cuda(e);
    return timed_out ? TSNNLS_ETIMEOUT : TSNNLS_OK;
}

static_assert(kSpinLimit == TSNNLS_WAIT_PROBE_MAX_POLLS, "the probe's limit is the waits' bound");

extern "C" int tsnnls_wait_probe(int64_t polls) {
    // the same bound as every wait inside the solver: a larger count could
    // keep a shared GPU polling for a practically unlimited time
    if (polls < 0 || polls > kSpinLimit) return TSNNLS_EINVAL;
    int32_t *flag = nullptr;
    DevStatus *st = nullptr;
    cudaStream_t s = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&flag), sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&st), sizeof(DevStatus));
    if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(st, 0, sizeof(DevStatus), s);
    if (e == cudaSuccess) e = launch_wait_probe(s, flag, polls, st);
    int32_t timed_out = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&timed_out, &st->timeout, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (flag) cudaFree(flag);
    if (st) cudaFree(st);
    if (s) cudaStreamDestroy(s);
    if (e != cudaSuccess) return status_from_cuda(e);
    return timed_out ? TSNNLS_ETIMEOUT : TSNNLS_OK;
}
