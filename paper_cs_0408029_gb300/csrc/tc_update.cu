// Tensor-core trailing update of the FP32 blocked Cholesky:
//     C(i, j) -= sum_l X(i, l) X(j, l)      (lower 128 x 128 tiles, l < 128)
// on the 5th-generation tensor cores (tcgen05, kind::tf32), FP32 accumulate in
// tensor memory.  TF32 keeps 10 mantissa bits, too few for a preconditioner
// whose refinement must stay cheap, so every operand is split into
// hi = x with the low 13 mantissa bits cleared (exact in TF32) and lo = x - hi,
// and the tile is accumulated as hi*hi^T + hi*lo^T + lo*hi^T (the lo*lo^T term
// is below FP32 rounding); the products then carry about 2^-21 relative error.
//
// The panel kernel writes X twice more in K-major form (row i holds its 128
// values contiguously), as hi and lo copies; TMA brings 128-row boxes of them
// into shared memory with the 128-byte swizzle the MMA descriptors expect.
// One thread issues the TMA copies and the MMAs and alone waits on the stage
// barriers; all four warps then read the accumulator out of tensor memory
// (tcgen05.ld, one row per thread) and subtract it from C.  Every wait on an mbarrier is bounded: on timeout the
// CTA records st->timeout, waits (bounded) for its own copies, frees its
// tensor memory and returns.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace tsnnls {

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    for (int spin = 0; spin < kSpinLimit; ++spin) {
        if (mbar_test(bar, parity)) return true;
        if (spin > 256) __nanosleep(64);
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes grouped by 8 (1024-byte stride between groups).
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);  // start address (16-byte units)
    d |= (uint64_t)1u << 16;                  // leading byte offset (unused with this swizzle)
    d |= (uint64_t)(1024u >> 4) << 32;        // stride byte offset
    d |= (uint64_t)1u << 46;                  // descriptor version
    d |= (uint64_t)2u << 61;                  // 128-byte swizzle
    return d;
}

// Instruction descriptor: D FP32, A and B TF32, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tri_tile_tc(int64_t b, int64_t &I, int64_t &J) {
    int64_t i = (int64_t)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
    while (i * (i + 1) / 2 > b) --i;
    while ((i + 1) * (i + 2) / 2 <= b) ++i;
    I = i;
    J = b - i * (i + 1) / 2;
}

constexpr int kTile = 128;                    // M = N = 128
constexpr int kBoxBytes = 128 * 32 * 4;       // 128 rows x 32 FP32 (one 128-byte swizzle span)
constexpr int kStages = 4;                    // K = 128 in four 32-column stages
constexpr int kSmemBytes = 4 * kBoxBytes + 1024;  // A hi/lo, B hi/lo of one stage, + alignment
// 65 KB of shared memory and 128 tensor-memory columns per CTA: three CTAs
// share an SM, so one CTA's epilogue overlaps another's copies and MMAs.

}  // namespace

__global__ void __launch_bounds__(128, 3)
    tc_update_kernel(const __grid_constant__ CUtensorMap map_hi,
                     const __grid_constant__ CUtensorMap map_lo, float *__restrict__ S, int64_t k,
                     int64_t lds, int64_t T0, DevStatus *st, int64_t tile0) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ uint64_t bar_tma, bar_mma;
    __shared__ uint32_t tmem_sh;
    __shared__ int fail_sh;
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    unsigned char *sAh = base, *sAl = base + kBoxBytes, *sBh = base + 2 * kBoxBytes,
                  *sBl = base + 3 * kBoxBytes;
    int64_t I, J;
    tri_tile_tc(blockIdx.x + tile0, I, J);  // tiles before tile0 are done elsewhere
    const int64_t r0 = T0 + I * kTile, c0 = T0 + J * kTile;
    if (r0 >= k) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_sh)),
                     "r"(128)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(&bar_tma, 1);
        mbar_init(&bar_mma, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fail_sh = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_sh;
    constexpr uint32_t idesc = idesc_tf32(kTile, kTile);
    // Each thread owns one row of the tile in the epilogue; its first 16
    // values of C are loaded now, so their latency hides behind the MMAs
    // (this CTA is the only writer of its tile while the kernel runs).
    const int64_t row = r0 + 32 * warp + lane;
    auto load_c = [&](int cc, float (&cv)[16]) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int64_t col = c0 + cc * 16 + j;
            cv[j] = (row < k && col < k && row >= col) ? S[row + col * lds] : 0.f;
        }
    };
    float cur[16];
    load_c(0, cur);

    // Only the issuing thread waits on the stage barriers: a thread that
    // polled them alongside it could be overtaken by a full phase (thread 0
    // re-arms the barrier for the next stage as soon as the MMAs are done)
    // and then wait for a parity that never comes.  The others meet it at
    // the barrier after the last stage.
    uint32_t parity = 0;
    if (tid == 0) {
        for (int h = 0; h < kStages; ++h) {
            mbar_expect_tx(&bar_tma, 4 * kBoxBytes);
            const int x = 32 * h;
            tma_load_2d(sAh, &map_hi, x, (int)r0, &bar_tma);
            tma_load_2d(sAl, &map_lo, x, (int)r0, &bar_tma);
            tma_load_2d(sBh, &map_hi, x, (int)c0, &bar_tma);
            tma_load_2d(sBl, &map_lo, x, (int)c0, &bar_tma);
            if (!mbar_wait(&bar_tma, parity)) {
                fail_sh = 1;
                break;
            }
            tc_fence_after();
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const uint32_t off = kk * 32;  // 8 TF32 = 32 bytes of K
                const uint64_t ah = sdesc_sw128(smem_u32(sAh) + off);
                const uint64_t al = sdesc_sw128(smem_u32(sAl) + off);
                const uint64_t bh = sdesc_sw128(smem_u32(sBh) + off);
                const uint64_t bl = sdesc_sw128(smem_u32(sBl) + off);
                mma_tf32(tmem, ah, bh, idesc, (h | kk) != 0);
                mma_tf32(tmem, ah, bl, idesc, 1);
                mma_tf32(tmem, al, bh, idesc, 1);
            }
            mma_commit(&bar_mma);
            // the MMAs must be done with this stage's operands before the
            // next TMA overwrites them (and, after the last stage, before the
            // accumulator is read)
            if (!mbar_wait(&bar_mma, parity)) {
                fail_sh = 1;
                break;
            }
            parity ^= 1;
        }
    }
    __syncthreads();
    if (fail_sh) {
        if (tid == 0) {
            st->timeout = 1;
            // bounded wait for copies that may still be in flight before the CTA goes away
            mbar_wait(&bar_tma, parity);
            mbar_wait(&bar_mma, parity);
        }
    } else {
        tc_fence_after();
        // chunk cc + 1 of C is loaded before chunk cc is stored: all loads of
        // a chunk are issued ahead of stores that, as far as the compiler can
        // tell, could alias them
#pragma unroll 1
        for (int cc = 0; cc < 8; ++cc) {
            float nxt[16];
            if (cc + 1 < 8) load_c(cc + 1, nxt);
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(cc * 16), v);
            if (row < k) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int64_t col = c0 + cc * 16 + j;
                    if (col < k && row >= col) S[row + col * lds] = cur[j] - v[j];
                }
            }
#pragma unroll
            for (int j = 0; j < 16; ++j) cur[j] = nxt[j];
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128) : "memory");
    }
}

// ---------------------------------------------------------------------------
// host side: tensor maps over the K-major hi / lo copies of the panel

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// Looked up once (thread-safe static initialisation: serving lanes call this
// from several threads).
static EncodeTiledFn encode_fn() {
    static const EncodeTiledFn fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return reinterpret_cast<EncodeTiledFn>(p);
        return static_cast<EncodeTiledFn>(nullptr);
    }();
    return fn;
}

bool tc_available() { return encode_fn() != nullptr; }

// Encode a map over a rows x 128 FP32 row-major buffer, boxes of 128 rows x 32.
bool tc_encode_panel_map(void *buf, int64_t rows, CUtensorMap *out) {
    EncodeTiledFn fn = encode_fn();
    if (!fn || rows <= 0) return false;
    cuuint64_t gdim[2] = {128, (cuuint64_t)rows};
    cuuint64_t gstride[1] = {128 * sizeof(float)};
    cuuint32_t box[2] = {32, 128};
    cuuint32_t estride[2] = {1, 1};
    return fn(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, buf, gdim, gstride, box, estride,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool tc_panel_init(TcPanel &tc, float *xhi, float *xlo, int64_t rows) {
    tc.xhi = xhi;
    tc.xlo = xlo;
    tc.rows = rows;
    tc.ok = xhi && xlo && tc_encode_panel_map(xhi, rows, &tc.map_hi) &&
            tc_encode_panel_map(xlo, rows, &tc.map_lo);
    return tc.ok;
}

cudaError_t launch_tc_update(cudaStream_t s, const CUtensorMap &hi, const CUtensorMap &lo, float *S,
                             int64_t k, int64_t lds, int64_t T0, DevStatus *st, int64_t tile0) {
    const int64_t rem = k - T0;
    if (rem <= 0) return cudaSuccess;
    // set on every launch: it is per device, and cheap
    cudaError_t e = cudaFuncSetAttribute(tc_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kSmemBytes);
    if (e != cudaSuccess) return e;
    const int64_t t = cdiv(rem, kTile);
    const int64_t tiles = t * (t + 1) / 2 - tile0;
    if (tiles <= 0) return cudaSuccess;
    tc_update_kernel<<<(unsigned)tiles, 128, kSmemBytes, s>>>(hi, lo, S, k, lds, T0, st, tile0);
    note_launches(1);
    return cudaGetLastError();
}

}  // namespace tsnnls
