// The pivot loop of the block principal pivoting method (Section 2,
// algorithm box) on one stream, on top of the cached A^T A of Section 3:
//
//   validate -> CSC transpose -> G = A^T A, c = A^T b -> F = {}, y = -c
//   repeat: exchange (zeroing, infeasible count, N/p rule, new F)
//           gather S = G_FF -> Cholesky S = L L^T
//           x_F = (L L^T)^{-1} c_F, then FP64 iterative refinement
//               r = b - A x, s = A^T r, x_F += (L L^T)^{-1} s_F
//           y_G = -s_G (Eq. 5 from the last residual)
//
// MIXED keeps G, S, L and the triangular solves in FP32 and everything that
// decides the exchange (x, r, s, y and the sign tests) in FP64.  FP64 runs
// the same loop in FP64 with a single solve per pivot.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "check.cuh"
#include "engine.h"
#include "sparse_chol.h"

namespace tsnnls {

int status_from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return TSNNLS_OK;
    if (e == cudaErrorMemoryAllocation) return TSNNLS_ENOMEM;
    if (e == cudaErrorNoDevice || e == cudaErrorInvalidDevice || e == cudaErrorInsufficientDriver)
        return TSNNLS_ENODEV;
    return TSNNLS_ECUDA;
}

namespace {
thread_local int64_t g_launches = 0;
}

void note_launches(int n) { g_launches += n; }

int num_sms() {
    constexpr int kMaxDev = 64;
    static std::atomic<int> cache[kMaxDev];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return 1;
    int v = cache[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) return 1;
    cache[dev].store(v, std::memory_order_relaxed);
    return v;
}
int64_t launches_so_far() { return g_launches; }

static cudaEvent_t pool_event(Lane &l) {
    if (l.ev_used == l.ev_pool.size()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        l.ev_pool.push_back(e);
    }
    return l.ev_pool[l.ev_used++];
}

// ---- bounds-check records (filled only in the checked build) -------------

namespace {
struct CheckUnit {
    const char *name;
    CheckCollectFn fn;
};
std::vector<CheckUnit> &check_units() {
    static std::vector<CheckUnit> units;
    return units;
}
std::mutex g_check_mu;
int64_t g_check_hits = 0;  // since the last tsnnls_check_report
std::string g_check_first;
}  // namespace

CheckRegistrar::CheckRegistrar(const char *unit, CheckCollectFn fn) { check_units().push_back({unit, fn}); }

int check_collect(char *what, size_t len) {
    std::lock_guard<std::mutex> g(g_check_mu);
    int total = 0;
    for (const CheckUnit &u : check_units()) {
        CheckRecord r{};
        if (u.fn(&r) != 0 || r.hits <= 0) continue;
        char line[256];
        snprintf(line, sizeof line, "%s.cu:%d: index %lld outside [0, %lld)", u.name, r.line,
                 (long long)r.index, (long long)r.bound);
        if (total == 0 && what && len) snprintf(what, len, "%s", line);
        if (g_check_hits == 0 && total == 0) g_check_first = line;
        total += r.hits;
    }
    g_check_hits += total;
    return total;
}

int check_report(char *buf, size_t len) {
    std::lock_guard<std::mutex> g(g_check_mu);
    const int64_t hits = g_check_hits;
    if (buf && len) snprintf(buf, len, "%s", g_check_first.c_str());
    g_check_hits = 0;
    g_check_first.clear();
    return (int)std::min<int64_t>(hits, INT32_MAX);
}

static const char *const kPhaseName[TSNNLS_NUM_PHASES] = {
    "setup", "gram", "exchange", "gather", "factor", "trsv", "spmv", "vector", "lsqr",
    "factor_diag", "factor_panel", "factor_update", "reuse"};

NvtxSolve::NvtxSolve(Lane &lane, const char *what) : l(lane) { nvtxRangePushA(what); }

NvtxSolve::~NvtxSolve() {
    if (l.nvtx_open) nvtxRangePop();
    if (l.nvtx_pivot_open) nvtxRangePop();
    l.nvtx_open = l.nvtx_pivot_open = false;
    nvtxRangePop();
}

void nvtx_pivot(Lane &l, int iter) {
    if (l.nvtx_open) nvtxRangePop();
    if (l.nvtx_pivot_open) nvtxRangePop();
    char name[32];
    snprintf(name, sizeof name, "pivot %d", iter);
    nvtxRangePushA(name);
    l.nvtx_open = false;
    l.nvtx_pivot_open = true;
}

void prof_begin(Lane &l, int phase) {
    if (l.nvtx_open) nvtxRangePop();
    nvtxRangePushA(phase >= 0 && phase < TSNNLS_NUM_PHASES ? kPhaseName[phase] : "phase");
    l.nvtx_open = true;
    l.mark_launch0 = launches_so_far();
    if (!l.prof) return;
    PhaseMark mk{phase, pool_event(l), nullptr, 0.0, 0.0, 0};
    if (mk.e0) cudaEventRecord(mk.e0, l.stream);
    l.marks.push_back(mk);
}

void prof_end(Lane &l, double bytes, double flops) {
    if (l.nvtx_open) nvtxRangePop();
    l.nvtx_open = false;
    if (!l.prof || l.marks.empty()) return;
    PhaseMark &mk = l.marks.back();
    mk.e1 = pool_event(l);
    if (mk.e1) cudaEventRecord(mk.e1, l.stream);
    mk.bytes = bytes;
    mk.flops = flops;
    mk.launches = launches_so_far() - l.mark_launch0;
}

void prof_flush(Lane &l) {
    for (const PhaseMark &mk : l.marks) {
        float ms = 0.f;
        if (mk.e0 && mk.e1 && cudaEventElapsedTime(&ms, mk.e0, mk.e1) == cudaSuccess) {
            tsnnls_phase_stat &st = l.stats[mk.phase];
            st.ms += ms;
            st.launches += mk.launches;
            st.bytes += mk.bytes;
            st.flops += mk.flops;
        }
    }
    l.marks.clear();
    l.ev_used = 0;
}

int lane_create(Lane &l) {
    cudaError_t e = cudaStreamCreateWithFlags(&l.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&l.st_dev, sizeof(DevStatus));
    if (e == cudaSuccess) e = cudaMallocHost(&l.st_host, sizeof(DevStatus));
    if (e == cudaSuccess) e = cudaMalloc(&l.bad_dev, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMallocHost(&l.bad_host, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaEventCreate(&l.ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&l.ev1);
    int least = 0, greatest = 0;
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&l.side, cudaStreamNonBlocking, greatest);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&l.fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&l.head, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&l.ev_status, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&l.join, cudaEventDisableTiming);
    return status_from_cuda(e);
}

void lane_destroy(Lane &l) {
    if (l.stream) cudaStreamSynchronize(l.stream);
    if (l.side) cudaStreamSynchronize(l.side);
    batch_cache_release(l);
    factor_graph_release(l);
    if (l.fork) cudaEventDestroy(l.fork);
    if (l.head) cudaEventDestroy(l.head);
    if (l.ev_status) cudaEventDestroy(l.ev_status);
    if (l.join) cudaEventDestroy(l.join);
    if (l.side) cudaStreamDestroy(l.side);
    if (l.ev0) cudaEventDestroy(l.ev0);
    if (l.ev1) cudaEventDestroy(l.ev1);
    for (cudaEvent_t e : l.ev_pool) cudaEventDestroy(e);
    if (l.st_dev) cudaFree(l.st_dev);
    if (l.st_host) cudaFreeHost(l.st_host);
    if (l.bad_dev) cudaFree(l.bad_dev);
    if (l.bad_host) cudaFreeHost(l.bad_host);
    if (l.stream) cudaStreamDestroy(l.stream);
    l = Lane{};
}

// ---- factorisations replayed as CUDA graphs ---------------------------------
// A factorisation on the look-ahead schedule is a fixed sequence of about
// 3 k/128 launches and event edges over the lane's two streams, determined
// by (S, k, lds, the status block, the tensor-core panels).  The second time
// a lane meets the same key it captures that sequence into a graph (node
// priorities kept, so the side stream's chain stays ahead of the update)
// and replays it from then on: the device then starts each kernel of the
// chain sooner than after separate launches (a 20000 x 8000 solve took
// 17.9 instead of 20.0 ms).  A key seen once is launched directly, so a
// stream of different sizes pays for no capture; a lane keeps at most
// kFactorGraphs graphs (the least recently used is replaced) and remembers
// kFactorSeen keys.

namespace {

constexpr size_t kFactorGraphs = 16, kFactorSeen = 64;

struct FactorGraphKey {
    const void *S, *st, *xhi, *xlo;
    int64_t k, lds, tc_rows;
    bool tc_ok;
    size_t elem;
    bool operator==(const FactorGraphKey &o) const {
        return S == o.S && st == o.st && xhi == o.xhi && xlo == o.xlo && k == o.k && lds == o.lds && tc_rows == o.tc_rows &&
               tc_ok == o.tc_ok && elem == o.elem;
    }
};

struct FactorGraph {
    FactorGraphKey key;
    cudaGraphExec_t exec = nullptr;
    uint64_t used = 0;
    int64_t launches = 0;  // the kernels a replay runs (launch accounting)
};

struct FactorGraphCache {
    std::vector<FactorGraphKey> seen;  // oldest first
    std::vector<FactorGraph> graphs;
    uint64_t tick = 0;
};

}  // namespace

void factor_graph_release(Lane &l) {
    auto *c = static_cast<FactorGraphCache *>(l.factor_graphs);
    if (!c) return;
    for (auto &g : c->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    delete c;
    l.factor_graphs = nullptr;
}

// The look-ahead factorisation of S (k x k, leading dimension lds) on the
// lane's streams: replayed from a graph, captured into one, or launched
// directly (see above); directly too inside a caller's own capture.
template <typename T>
static cudaError_t launch_cholesky_lane(Lane &lane, cudaStream_t s, T *S, int64_t k, int64_t lds,
                                        const TcPanel *tc) {
    const FactorStreams fs{lane.side, lane.fork, lane.head, lane.join};
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return e;
    if (cs != cudaStreamCaptureStatusNone) return launch_cholesky<T>(s, S, k, lds, lane.st_dev, tc, nullptr, &fs);
    auto *c = static_cast<FactorGraphCache *>(lane.factor_graphs);
    if (!c) {
        c = new FactorGraphCache;
        lane.factor_graphs = c;
    }
    const FactorGraphKey key{S,
                             lane.st_dev,
                             tc ? static_cast<const void *>(tc->xhi) : nullptr,
                             tc ? static_cast<const void *>(tc->xlo) : nullptr,
                             k,
                             lds,
                             tc ? tc->rows : 0,
                             tc ? tc->ok : false,
                             sizeof(T)};
    ++c->tick;
    for (auto &g : c->graphs)
        if (g.key == key) {
            g.used = c->tick;
            note_launches((int)g.launches);
            return cudaGraphLaunch(g.exec, s);
        }
    auto seen = std::find(c->seen.begin(), c->seen.end(), key);
    if (seen == c->seen.end()) {
        if (c->seen.size() >= kFactorSeen) c->seen.erase(c->seen.begin());
        c->seen.push_back(key);
        return launch_cholesky<T>(s, S, k, lds, lane.st_dev, tc, nullptr, &fs);
    }
    e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    const int64_t l0 = launches_so_far();
    const cudaError_t el = launch_cholesky<T>(s, S, k, lds, lane.st_dev, tc, nullptr, &fs);
    const int64_t nl = launches_so_far() - l0;
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(s, &graph);
    if (el != cudaSuccess || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return el != cudaSuccess ? el : e;
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiateWithFlags(&exec, graph, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return e;
    if (c->graphs.size() >= kFactorGraphs) {
        auto lru = std::min_element(c->graphs.begin(), c->graphs.end(),
                                    [](const FactorGraph &a, const FactorGraph &b) { return a.used < b.used; });
        e = cudaStreamSynchronize(s);  // a replay of the graph being replaced may still run
        if (e == cudaSuccess) e = cudaGraphExecDestroy(lru->exec);
        c->graphs.erase(lru);
        if (e != cudaSuccess) {
            cudaGraphExecDestroy(exec);
            return e;
        }
    }
    c->seen.erase(seen);
    c->graphs.push_back(FactorGraph{key, exec, c->tick, nl});
    return cudaGraphLaunch(exec, s);
}

namespace {

// Sub-allocator over one stream-ordered allocation.
struct Carve {
    char *base = nullptr;
    size_t off = 0;
    template <typename P>
    P *take(size_t count) {
        off = (size_t)round_up((int64_t)off, 256);
        P *p = reinterpret_cast<P *>(base + off);
        off += sizeof(P) * std::max<size_t>(count, 1);
        return p;
    }
};

// sparse_bytes > 0: the sparse path, whose factor state (sparse_bytes) replaces
// the dense G and S, the reuse buffers and the tensor-core panels.
template <typename T>
size_t layout_bytes(int64_t m, int64_t n, int64_t nnz, bool host_in, size_t sparse_bytes = 0) {
    Carve c;
    const bool sparse = sparse_bytes > 0;
    const int64_t ldg = sparse ? 0 : round_up(n, 32);
    if (host_in) {
        c.take<int64_t>(m + 1);
        c.take<int32_t>(nnz);
        c.take<double>(nnz);
        c.take<double>(m);
    }
    c.take<int64_t>(n + 1);
    c.take<int32_t>(nnz);
    c.take<double>(nnz);
    c.take<int32_t>(n + 1);
    c.take<int64_t>(n + 1);
    c.take<T>((size_t)n * ldg);  // G
    c.take<T>((size_t)n * ldg);  // S / L
    for (int i = 0; i < 5; ++i) c.take<double>(n);  // c, x, y, s, settled-test bound
    c.take<double>(m);                              // r
    c.take<T>(n);                                   // rhs
    c.take<uint8_t>(n);
    c.take<int32_t>(n);
    c.take<char>(quality_scratch_bytes(m, n));
    if (sparse) {
        c.take<char>(sparse_bytes);
        return c.off + 256;
    }
    c.take<char>(chol_solve_scratch_bytes(n, sizeof(T)));
    c.take<char>(border_bytes(n, sizeof(T)));  // reuse of a factor across pivots
    if (sizeof(T) == 4) {
        c.take<float>((size_t)n * 128);  // K-major hi / lo panel copies for the tensor-core update
        c.take<float>((size_t)n * 128);
    }
    return c.off + 256;
}

struct LaneTimer : KernelTimer {
    Lane &l;
    explicit LaneTimer(Lane &lane) : l(lane) {}
    void begin(int phase) override { prof_begin(l, phase); }
    void end(double bytes, double flops) override { prof_end(l, bytes, flops); }
};

struct Sync {
    Lane &l;
    cudaError_t read() {
        cudaError_t e = cudaMemcpyAsync(l.st_host, l.st_dev, sizeof(DevStatus),
                                        cudaMemcpyDeviceToHost, l.stream);
        if (e != cudaSuccess) return e;
        return cudaStreamSynchronize(l.stream);
    }
    // copy the status now, wait for that copy later: work queued in between
    // keeps the device busy while the host waits
    cudaError_t post() {
        cudaError_t e = cudaMemcpyAsync(l.st_host, l.st_dev, sizeof(DevStatus),
                                        cudaMemcpyDeviceToHost, l.stream);
        if (e != cudaSuccess) return e;
        return cudaEventRecord(l.ev_status, l.stream);
    }
    cudaError_t wait() { return cudaEventSynchronize(l.ev_status); }
};

#define TRY_CUDA(expr)                          \
    do {                                        \
        cudaError_t e_ = (expr);                \
        if (e_ != cudaSuccess) {                \
            status = status_from_cuda(e_);      \
            goto cleanup;                       \
        }                                       \
    } while (0)

// Reusing a factor costs three triangular-solve passes of setup (the a
// columns of P^T side by side, then the r columns of Z forward and back)
// against about 30 passes' worth for a gather and refactorisation at any
// k >= 1024 (both scale with the number of 128-wide block steps); the bordered
// solves add a few small kernels to every refinement step.
constexpr int64_t kReuseMinK = 1024;

template <typename T>
int solve_factor(Context &ctx, Lane &lane, const tsnnls_csr &A, const double *b, double *x_out,
                 const tsnnls_opts &o, tsnnls_info *info, const SolveExtras *ex, bool force_refine) {
    (void)ctx;
    const int64_t m = A.m, n = A.n, nnz = A.nnz;
    const bool host_in = A.on_device == 0;
    // refinement with FP64 residuals: always on the FP32 factor; on the FP64
    // factor only when redoing a MIXED solve whose FP32 refinement stagnated
    const bool mixed = o.precision == TSNNLS_MIXED || force_refine;
    // the sparse path (supernodal factor of the permuted G_FF, sparse_chol.cu)
    // replaces the dense G, the gather and the dense factor; the rest of the
    // pivot loop is the same
    const bool sparse = o.path == TSNNLS_PATH_SPARSE;
    std::shared_ptr<const SparseSym> sym;
    double analysis_ms = 0.0;
    if (sparse) {
        sym = ex ? ex->sym : nullptr;
        if (!sym) sym = analyze_gram_pattern(A, kSpNB);
        if (!sym) return TSNNLS_EINVAL;
        analysis_ms = sym->analysis_ms;
    }
    const size_t sparse_bytes = sparse ? SparseChol<T>::device_bytes(*sym, std::max(1, num_sms())) : 0;
    SparseChol<T> sc;
    const int64_t ldg = sparse ? 0 : round_up(n, 32);
    const int32_t max_iter = o.max_iter > 0 ? o.max_iter : (int32_t)std::min<int64_t>(10 * n + 100, INT32_MAX);
    cudaStream_t s = lane.stream;
    Sync sync{lane};
    int status = TSNNLS_OK;
    int refine_total = 0;
    double last_rel = 0.0;
    int64_t trace_rows = 0;
    double cond = 0.0;  // opts.cond_est
    const int64_t launch0 = launches_so_far();

    Carve cv;
    const size_t bytes = layout_bytes<T>(m, n, nnz, host_in, sparse_bytes);
    void *block = nullptr;
    {
        cudaError_t e = cudaMallocAsync(&block, bytes, s);
        if (e != cudaSuccess) return status_from_cuda(e);
    }
    cv.base = static_cast<char *>(block);
    const int64_t *row_ptr;
    const int32_t *col;
    const double *val;
    const double *bd;
    if (host_in) {
        int64_t *rp = cv.take<int64_t>(m + 1);
        int32_t *ci = cv.take<int32_t>(nnz);
        double *va = cv.take<double>(nnz);
        double *bb = cv.take<double>(m);
        TRY_CUDA(cudaMemcpyAsync(rp, A.row_ptr, sizeof(int64_t) * (m + 1), cudaMemcpyHostToDevice, s));
        if (nnz > 0) {
            TRY_CUDA(cudaMemcpyAsync(ci, A.col_idx, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, s));
            TRY_CUDA(cudaMemcpyAsync(va, A.val, sizeof(double) * nnz, cudaMemcpyHostToDevice, s));
        }
        TRY_CUDA(cudaMemcpyAsync(bb, b, sizeof(double) * m, cudaMemcpyHostToDevice, s));
        row_ptr = rp;
        col = ci;
        val = va;
        bd = bb;
    } else {
        row_ptr = A.row_ptr;
        col = A.col_idx;
        val = A.val;
        bd = b;
    }
    {
        int64_t *col_ptr = cv.take<int64_t>(n + 1);
        int32_t *row_idx = cv.take<int32_t>(nnz);
        double *cval = cv.take<double>(nnz);
        int32_t *cnt = cv.take<int32_t>(n + 1);
        int64_t *next = cv.take<int64_t>(n + 1);
        T *G = cv.take<T>((size_t)n * ldg);
        T *S = cv.take<T>((size_t)n * ldg);
        double *c = cv.take<double>(n);
        double *x = cv.take<double>(n);
        double *y = cv.take<double>(n);
        double *sv = cv.take<double>(n);
        double *cbound = cv.take<double>(n);
        double *r = cv.take<double>(m);
        T *rhs = cv.take<T>(n);
        uint8_t *inF = cv.take<uint8_t>(n);
        int32_t *F = cv.take<int32_t>(n);
        void *qscratch = cv.take<char>(quality_scratch_bytes(m, n));
        void *sparse_mem = sparse ? cv.take<char>(sparse_bytes) : nullptr;
        void *trsv_scratch = sparse ? nullptr : cv.take<char>(chol_solve_scratch_bytes(n, sizeof(T)));
        const BorderBuffers bb =
            sparse ? BorderBuffers{} : border_carve(cv.take<char>(border_bytes(n, sizeof(T))), n, sizeof(T));
        TcPanel tc;
        if (sizeof(T) == 4 && !sparse) {
            float *xhi = cv.take<float>((size_t)n * 128);
            float *xlo = cv.take<float>((size_t)n * 128);
            tc_panel_init(tc, xhi, xlo, n);
        }
        const double avg_row = (double)nnz / (double)m, avg_col = (double)nnz / (double)n;
        const double csr_bytes = 12.0 * nnz + 8.0 * (m + 1);
        const double csc_bytes = 12.0 * nnz + 8.0 * (n + 1);

        TRY_CUDA(cudaEventRecord(lane.ev0, s));
        TRY_CUDA(cudaMemsetAsync(lane.bad_dev, 0, sizeof(int32_t), s));
        prof_begin(lane, TSNNLS_PHASE_SETUP);
        TRY_CUDA(launch_validate(s, m, n, nnz, row_ptr, col, val, bd, lane.bad_dev));
        prof_end(lane, csr_bytes + 8.0 * m, 0.0);
        TRY_CUDA(cudaMemcpyAsync(lane.bad_host, lane.bad_dev, sizeof(int32_t),
                                 cudaMemcpyDeviceToHost, s));
        TRY_CUDA(cudaStreamSynchronize(s));
        if (*lane.bad_host != 0) {
            status = TSNNLS_EINVAL;
            goto cleanup;
        }
        // Section 3: transpose once, then G = A^T A and c = A^T b
        prof_begin(lane, TSNNLS_PHASE_SETUP);
        TRY_CUDA(launch_csr_to_csc(s, m, n, nnz, row_ptr, col, val, col_ptr, row_idx, cval, cnt,
                                   next));
        prof_end(lane, csr_bytes + csc_bytes, 0.0);
        if (mixed && o.full_refine == 0) {
            // bound for the settled test (r serves as scratch until the first residual)
            prof_begin(lane, TSNNLS_PHASE_SETUP);
            TRY_CUDA(launch_gram_row_bound(s, m, n, row_ptr, val, col_ptr, row_idx, cval, r, cbound));
            prof_end(lane, csr_bytes + csc_bytes + 8.0 * (2.0 * m + n), 2.0 * nnz);
        }
        prof_begin(lane, TSNNLS_PHASE_GRAM);
        if (sparse) {
            // c = A^T b, and A^T A on the analysed pattern (FP64)
            TRY_CUDA(launch_spmv(s, n, col_ptr, row_idx, cval, 1.0, bd, m, 0.0, nullptr, c, avg_col));
            TRY_CUDA(sc.setup(*sym, sparse_mem, s, col_ptr, row_idx, cval));
            prof_end(lane, csc_bytes + 8.0 * (m + n) + 16.0 * (double)sym->grow.size(), 0.0);
        } else {
            TRY_CUDA(launch_gram<T>(s, m, n, row_ptr, col, val, col_ptr, row_idx, cval, bd, G, ldg, c));
            prof_end(lane, csr_bytes + csc_bytes + 0.5 * (double)n * (n + 1) * sizeof(T) + 8.0 * (m + n), 0.0);
        }
        // F = {}, G = all, x = 0, y = -A^T b, p = p_max, N = infinity
        prof_begin(lane, TSNNLS_PHASE_VECTOR);
        TRY_CUDA(launch_init_state(s, n, c, x, y, inF, o.p_max, lane.st_dev));
        prof_end(lane, 25.0 * n, 0.0);

        // FP64 residual r = b - A_F x_F and s = A^T r (x_G = 0) for the current x
        auto residual = [&]() -> cudaError_t {
            prof_begin(lane, TSNNLS_PHASE_SPMV);
            cudaError_t e = launch_spmv(s, m, row_ptr, col, val, -1.0, x, n, 1.0, bd, r, avg_row);
            if (e == cudaSuccess) e = launch_spmv(s, n, col_ptr, row_idx, cval, 1.0, r, m, 0.0, nullptr, sv, avg_col);
            prof_end(lane, 2.0 * 12.0 * nnz + 8.0 * (m + 1) + 8.0 * (n + 1) + 8.0 * (3.0 * m + 2.0 * n),
                     4.0 * nnz);
            return e;
        };
        int64_t k = 0, lds = 32;
        // The pivot's solver: a fresh factor of G_FF in S (list F, k), or the
        // factor of an earlier base set B (kb, ldsb) reused with ba added and
        // br removed variables (list U, kb + ba entries; border.cu).
        bool base_valid = false, reuse = false;
        int64_t kb = 0, ldsb = 32;
        int ba = 0, br = 0;
        int reuses = 0;
        // sparse: the solves run on all n entries in the factor's order, the
        // list giving each position's variable (-1 outside F: held at zero)
        auto sol_list = [&]() -> const int32_t * { return sparse ? sc.permF : (reuse ? bb.Ul : F); };
        auto sol_len = [&]() -> int64_t { return sparse ? n : (reuse ? kb + ba : k); };
        auto pivot_solve = [&](T *v) -> cudaError_t {
            if (sparse) return sc.solve(s, v, lane.st_dev);
            return reuse ? launch_border_solve<T>(s, S, kb, ldsb, ba, br, bb, v, trsv_scratch, lane.st_dev)
                         : launch_chol_solve<T>(s, S, k, lds, v, trsv_scratch, lane.st_dev);
        };
        // Refinement of the current pivot's x_F on its solver (Section 3: FP32
        // solves, FP64 residuals), from `steps` solves done and the last
        // correction `prev`.  allow_settle: stop before rel_tol once the
        // settled test passes (*settled is then set).
        auto refine = [&](int steps, double prev, bool allow_settle, bool *settled) -> int {
            *settled = false;
            for (;;) {
                const int64_t kl = reuse ? kb : k;
                const double tri = sparse ? (double)sym->nnz_L * sizeof(T)
                                          : 0.5 * (double)kl * (double)(kl + 1) * sizeof(T);
                prof_begin(lane, TSNNLS_PHASE_VECTOR);
                cudaError_t e = launch_gather_rhs<T>(s, sv, n, sol_list(), sol_len(), rhs);
                prof_end(lane, (12.0 + sizeof(T)) * sol_len(), 0.0);
                prof_begin(lane, TSNNLS_PHASE_TRSV);
                if (e == cudaSuccess) e = pivot_solve(rhs);
                prof_end(lane, 2.0 * tri + 4.0 * sizeof(T) * kl, 2.0 * (double)kl * (double)kl);
                prof_begin(lane, TSNNLS_PHASE_VECTOR);
                if (e == cudaSuccess) e = launch_update_x<T>(s, rhs, sol_list(), sol_len(), x, n, lane.st_dev);
                prof_end(lane, (20.0 + sizeof(T)) * sol_len(), 0.0);
                if (e == cudaSuccess) e = sync.post();
                if (e == cudaSuccess) e = residual();
                if (e == cudaSuccess) e = sync.wait();
                if (e != cudaSuccess) return status_from_cuda(e);
                if (lane.st_host->timeout) return TSNNLS_ETIMEOUT;
                ++steps;
                ++refine_total;
                const double d = lane.st_host->dnorm, xn = lane.st_host->xnorm;
                last_rel = xn > 0 ? d / xn : 0.0;
                if (d <= o.rel_tol * xn) return TSNNLS_OK;  // the residual queued above is for this x
                if (d > 0.5 * prev && d <= 1e-9 * xn) return TSNNLS_OK;  // rounding floor, below target
                if (steps >= o.max_refine || (steps > 4 && d > prev))
                    return d <= 1e-9 * xn ? TSNNLS_OK : TSNNLS_ENOCONV;
                if (allow_settle && d <= 0.1 * prev) {
                    // contraction rho = d / prev <= 0.1 observed: while it holds
                    // the error left in x is about rho d / (1 - rho) in the max
                    // norm; E allows 20 times that, at most 0.5 d, plus the
                    // rounding floor
                    const double rho = d / prev;
                    const double E = std::min(0.5, 20.0 * rho) * d + 1e-15 * xn;
                    prof_begin(lane, TSNNLS_PHASE_VECTOR);
                    e = launch_settled(s, n, inF, x, sv, cbound, E, o.zero_tol, lane.st_dev);
                    prof_end(lane, 25.0 * n, 0.0);
                    if (e == cudaSuccess) e = sync.read();
                    if (e != cudaSuccess) return status_from_cuda(e);
                    if (lane.st_host->unsettled == 0) {
                        *settled = true;
                        return TSNNLS_OK;
                    }
                }
                prev = d;
            }
        };
        bool open_pivot = false;  // the last pivot stopped at the settled test
        int open_steps = 0;
        double open_prev = 0.0;

        for (int pivot_range = 1;; ++pivot_range) {
            nvtx_pivot(lane, pivot_range);
            prof_begin(lane, TSNNLS_PHASE_EXCHANGE);
            TRY_CUDA(launch_exchange(s, n, x, y, inF, F, o.zero_tol, o.p_max, max_iter,
                                     lane.st_host->iters > 0 ? 1 : 0, lane.st_dev));
            if (base_valid) TRY_CUDA(launch_border_count(s, n, inF, bb, lane.st_dev));
            prof_end(lane, 17.0 * n + 17.0 * n + 4.0 * n, 0.0);
            TRY_CUDA(sync.read());
            const DevStatus st = *lane.st_host;
            if (st.done && open_pivot && !st.maxiter_hit) {
                // x_F, y_G are feasible: this was the last pivot, so its
                // refinement goes on to rel_tol (the decisions were settled,
                // so the exchange will find the same sets again)
                open_pivot = false;
                TRY_CUDA(residual());
                bool settled_unused = false;
                status = refine(open_steps, open_prev, false, &settled_unused);
                if (status != TSNNLS_OK) goto cleanup;
                prof_begin(lane, TSNNLS_PHASE_VECTOR);
                TRY_CUDA(launch_y_from_s(s, n, sv, inF, y));
                prof_end(lane, 17.0 * n, 0.0);
                continue;
            }
            if (st.done) {
                if (st.maxiter_hit) status = TSNNLS_EMAXITER;
                break;
            }
            if (ex && ex->trace && trace_rows < ex->trace_cap) {
                int64_t *t = ex->trace + kTraceCols * trace_rows;
                t[0] = st.n_inf;
                t[1] = -1;  // filled below from the previous row
                t[2] = st.p;
                t[3] = st.branch;
                t[4] = st.k;
                t[5] = st.moved;
            }
            k = st.k;
            lds = round_up(std::max<int64_t>(k, 1), 32);
            // Reuse the base factor when at most kBorderMax variables were
            // added and removed since it was taken (the FP32 refinement path
            // only; the plain FP64 path refactors every pivot as the paper
            // does, so does the FP64 redo of a failed MIXED solve, and the
            // condition estimate wants the factor of the last F itself).
            reuse = false;
            if (!sparse && sizeof(T) == 4 && mixed && base_valid && k > 0 && o.cond_est == 0 && o.no_reuse == 0 &&
                st.border_a <= kBorderMax && st.border_r <= kBorderMax && kb >= kReuseMinK) {
                ba = st.border_a;
                br = st.border_r;
                prof_begin(lane, TSNNLS_PHASE_REUSE);
                TRY_CUDA(launch_border_diff(s, n, inF, bb, kb, lane.st_dev));
                TRY_CUDA(launch_border_setup<T>(s, G, ldg, S, kb, ldsb, ba, br, bb, lane.st_dev));
                prof_end(lane, (double)(ba + 2 * br) * 0.5 * (double)kb * (double)kb * sizeof(T), 0.0);
                int32_t bad = 0;
                TRY_CUDA(cudaMemcpyAsync(&bad, bb.bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
                TRY_CUDA(cudaStreamSynchronize(s));
                reuse = bad == 0;
                if (reuse) ++reuses;
            }
            if (k > 0 && sparse) {
                prof_begin(lane, TSNNLS_PHASE_FACTOR);
                TRY_CUDA(sc.factor(s, inF, lane.st_dev));
                TRY_CUDA(sc.perm_list(s, inF));
                prof_end(lane, 2.0 * (double)sym->nnz_L * sizeof(T), sym->flops);
            }
            if (k > 0) {
                const double tri = sparse ? (double)sym->nnz_L * sizeof(T)
                                          : 0.5 * (double)k * (double)(k + 1) * sizeof(T);
                if (!reuse && !sparse) {
                    prof_begin(lane, TSNNLS_PHASE_GATHER);
                    TRY_CUDA(launch_gather<T>(s, G, ldg, F, nullptr, k, S, lds));
                    prof_end(lane, 2.0 * tri + 4.0 * k, 0.0);
                    if (lane.prof && lane.prof_kernels) {
                        LaneTimer lt{lane};
                        TRY_CUDA(launch_cholesky<T>(s, S, k, lds, lane.st_dev, &tc, &lt));
                    } else {
                        prof_begin(lane, TSNNLS_PHASE_FACTOR);
                        TRY_CUDA(launch_cholesky_lane<T>(lane, s, S, k, lds, &tc));
                        prof_end(lane, 2.0 * tri, (double)k * (double)k * (double)k / 3.0);
                    }
                    if (sizeof(T) == 4 && mixed) {  // this factor becomes the base for later pivots
                        TRY_CUDA(cudaMemcpyAsync(bb.Bl, F, sizeof(int32_t) * k, cudaMemcpyDeviceToDevice, s));
                        TRY_CUDA(cudaMemcpyAsync(bb.inB, inF, (size_t)n, cudaMemcpyDeviceToDevice, s));
                        base_valid = true;
                        kb = k;
                        ldsb = lds;
                    }
                }
                // first solve: x_F = (L L^T)^{-1} c_F  (x restarts from 0)
                const int64_t kl = reuse ? kb : k;
                const double tril = sparse ? tri : 0.5 * (double)kl * (double)(kl + 1) * sizeof(T);
                prof_begin(lane, TSNNLS_PHASE_VECTOR);
                TRY_CUDA(launch_gather_rhs<T>(s, c, n, sol_list(), sol_len(), rhs));
                prof_end(lane, (12.0 + sizeof(T)) * sol_len(), 0.0);
                prof_begin(lane, TSNNLS_PHASE_TRSV);
                TRY_CUDA(pivot_solve(rhs));
                prof_end(lane, 2.0 * tril + 4.0 * sizeof(T) * kl, 2.0 * (double)kl * (double)kl);
                prof_begin(lane, TSNNLS_PHASE_VECTOR);
                TRY_CUDA(launch_update_x<T>(s, rhs, sol_list(), sol_len(), x, n, lane.st_dev));
                prof_end(lane, (20.0 + sizeof(T)) * sol_len(), 0.0);
                TRY_CUDA(sync.post());
            }
            // the residual of the new x is needed whether the refinement goes
            // on or not (at the end it gives y_G), so it is queued before the
            // host reads the status of the update
            TRY_CUDA(residual());
            if (k > 0) {
                TRY_CUDA(sync.wait());
                if (lane.st_host->chol_info) { status = TSNNLS_ENOTPD; break; }
                if (lane.st_host->timeout) { status = TSNNLS_ETIMEOUT; break; }
                ++refine_total;
            }
            if (mixed && k > 0) {
                bool settled = false;
                const double prev0 = lane.st_host->dnorm;
                status = refine(1, prev0, o.full_refine == 0, &settled);
                if (status != TSNNLS_OK) goto cleanup;
                open_pivot = settled;
                if (settled) {
                    open_steps = 0;  // refine() does not report its count: restart the limits
                    open_prev = lane.st_host->dnorm;
                }
            }
            // Eq. 5: y_G = A_G^T (A_F x_F - b) = -s_G
            prof_begin(lane, TSNNLS_PHASE_VECTOR);
            TRY_CUDA(launch_y_from_s(s, n, sv, inF, y));
            prof_end(lane, 17.0 * n, 0.0);
            ++trace_rows;
        }
        if (status == TSNNLS_OK) {
            // KKT violation and last residual change at the returned x (before
            // the condition estimate reuses rhs); the mixed path's last
            // correction is still in rhs, over the last pivot's list
            if (trace_rows == 0) TRY_CUDA(residual());  // no pivot ran: r, s of x = 0
            prof_begin(lane, TSNNLS_PHASE_VECTOR);
            const bool have_delta = mixed && k > 0;
            TRY_CUDA(launch_quality<T>(s, m, n, row_ptr, col, val, avg_row, x, sv, c, r,
                                       have_delta ? rhs : nullptr, sol_list(), have_delta ? sol_len() : 0,
                                       qscratch, lane.st_dev));
            prof_end(lane, 8.0 * (2.0 * m + 4.0 * n) + (have_delta ? csr_bytes + 16.0 * m : 0.0), 0.0);
        }
        if (status == TSNNLS_OK && o.cond_est && k > 0 && !sparse) {
            // kappa_1 of the last pivot's (A^T A)_FF: its 1-norm times an
            // estimate of ||(A^T A)_FF^-1||_1 from solves with the factor still
            // in S (Hager's method with Higham's refinements, as in dpocon;
            // Section 3 consults dpocon for the final recompute)
            double *dv = nullptr, *part = nullptr;
            T *xi = nullptr;
            double h[8] = {};
            auto solve = [&]() { return launch_chol_solve<T>(s, S, k, lds, rhs, trsv_scratch, lane.st_dev); };
            auto fetch = [&]() -> cudaError_t {
                cudaError_t e = cudaMemcpyAsync(h, dv, sizeof(h), cudaMemcpyDeviceToHost, s);
                return e == cudaSuccess ? cudaStreamSynchronize(s) : e;
            };
            cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&dv), sizeof(h), s);
            if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void **>(&xi), sizeof(T) * k, s);
            if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void **>(&part), gram_norm_scratch_bytes(k), s);
            if (e == cudaSuccess) e = launch_gram_norm1<T>(s, G, ldg, F, k, part, dv + 4);
            // x = (1/k) 1
            if (e == cudaSuccess) e = launch_est_fill<T>(s, rhs, k, 0, 0);
            if (e == cudaSuccess) e = solve();
            if (e == cudaSuccess) e = launch_est_norm_sign<T>(s, rhs, k, xi, dv);
            if (e == cudaSuccess) e = fetch();
            double est = h[0];
            int32_t mode = 0;
            int64_t jprev = 0;
            for (int it = 0; e == cudaSuccess && it < 5 && k > 1; ++it) {
                // z = G^-1 sign(y); stop once ||z||_inf <= z^T x, else x = e_j, j = argmax |z_j|
                e = cudaMemcpyAsync(rhs, xi, sizeof(T) * k, cudaMemcpyDeviceToDevice, s);
                if (e == cudaSuccess) e = solve();
                if (e == cudaSuccess) e = launch_est_argmax<T>(s, rhs, k, mode, jprev, dv);
                if (e == cudaSuccess) e = fetch();
                if (e != cudaSuccess || (it > 0 && h[1] <= h[3])) break;
                const int64_t j = (int64_t)h[2];
                e = launch_est_fill<T>(s, rhs, k, 1, j);
                if (e == cudaSuccess) e = solve();
                if (e == cudaSuccess) e = launch_est_norm_sign<T>(s, rhs, k, xi, dv);
                if (e == cudaSuccess) e = fetch();
                if (e != cudaSuccess || h[0] <= est) break;
                est = h[0];
                mode = 1;
                jprev = j;
            }
            // the alternating probe guards against a poor first direction
            if (e == cudaSuccess) e = launch_est_fill<T>(s, rhs, k, 2, 0);
            if (e == cudaSuccess) e = solve();
            if (e == cudaSuccess) e = launch_est_norm_sign<T>(s, rhs, k, xi, dv);
            if (e == cudaSuccess) e = fetch();
            if (e == cudaSuccess) cond = h[4] * std::max(est, 2.0 * h[0] / (3.0 * (double)k));
            if (dv) cudaFreeAsync(dv, s);
            if (xi) cudaFreeAsync(xi, s);
            if (part) cudaFreeAsync(part, s);
            TRY_CUDA(e);
        }
        if (status == TSNNLS_OK) {
            TRY_CUDA(cudaEventRecord(lane.ev1, s));
            const cudaMemcpyKind kind = host_in ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
            TRY_CUDA(cudaMemcpyAsync(lane.st_host, lane.st_dev, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
            TRY_CUDA(cudaMemcpyAsync(x_out, x, sizeof(double) * n, kind, s));
            if (ex && ex->y_out) TRY_CUDA(cudaMemcpyAsync(ex->y_out, y, sizeof(double) * n, kind, s));
            if (ex && ex->inF_out)
                TRY_CUDA(cudaMemcpyAsync(ex->inF_out, inF, (size_t)n, kind, s));
            TRY_CUDA(cudaStreamSynchronize(s));
            float ms = 0.f;
            // the sparse path's host analysis counts toward the solve's time
            if (cudaEventElapsedTime(&ms, lane.ev0, lane.ev1) == cudaSuccess && info)
                info->time_ms = ms + analysis_ms;
        }
        if (info) {
            info->iters = lane.st_host->iters;
            info->nF = lane.st_host->k;
            info->cond_est = cond;
            info->factor_reuses = reuses;
            if (status == TSNNLS_OK) {
                info->kkt_viol = lane.st_host->kkt_viol;
                info->rel_resid_change = lane.st_host->resid_change;
            }
        }
    }
cleanup:
    cudaFreeAsync(block, s);
    cudaStreamSynchronize(s);
    prof_flush(lane);
    if (ex && ex->trace) {
        // column 1: N before the branch = smallest count over the earlier pivots
        int64_t best = INT64_MAX;
        for (int64_t i = 0; i < std::min(trace_rows, ex->trace_cap); ++i) {
            ex->trace[kTraceCols * i + 1] = best;
            best = std::min(best, ex->trace[kTraceCols * i]);
        }
    }
    if (info) {
        info->status = status;
        info->refine_steps = refine_total;
        info->last_rel_step = last_rel;
        info->path_used = sparse ? TSNNLS_PATH_SPARSE : TSNNLS_PATH_FACTOR;
        info->precision_used = o.precision;
        info->kernel_launches = launches_so_far() - launch0;
    }
    return status;
}

}  // namespace

static size_t factor_footprint(const tsnnls_csr &A, const tsnnls_opts &o) {
    const bool host_in = A.on_device == 0;
    return o.precision == TSNNLS_FP64 ? layout_bytes<double>(A.m, A.n, A.nnz, host_in)
                                      : layout_bytes<float>(A.m, A.n, A.nnz, host_in);
}

std::shared_ptr<const SparseSym> analyze_gram_pattern(const tsnnls_csr &A, int max_width) {
    const auto t0 = std::chrono::steady_clock::now();
    std::vector<int64_t> rp;
    std::vector<int32_t> ci;
    const int64_t *row_ptr = A.row_ptr;
    const int32_t *col = A.col_idx;
    if (A.on_device) {
        rp.resize(A.m + 1);
        ci.resize(std::max<int64_t>(A.nnz, 1));
        if (cudaMemcpy(rp.data(), A.row_ptr, sizeof(int64_t) * (A.m + 1), cudaMemcpyDeviceToHost) != cudaSuccess)
            return nullptr;
        if (A.nnz > 0 &&
            cudaMemcpy(ci.data(), A.col_idx, sizeof(int32_t) * A.nnz, cudaMemcpyDeviceToHost) != cudaSuccess)
            return nullptr;
        row_ptr = rp.data();
        col = ci.data();
    }
    // the pattern must be valid before the analysis walks it
    if (row_ptr[0] != 0 || row_ptr[A.m] != A.nnz) return nullptr;
    for (int64_t r = 0; r < A.m; ++r) {
        if (row_ptr[r + 1] < row_ptr[r]) return nullptr;
        for (int64_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e)
            if (col[e] < 0 || col[e] >= A.n) return nullptr;
    }
    auto sym = std::make_shared<SparseSym>();
    if (sparse_analyze(A.m, A.n, row_ptr, col, max_width, *sym) != 0) return nullptr;
    sym->analysis_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return sym;
}

static size_t sparse_footprint(const tsnnls_csr &A, const tsnnls_opts &o, const SparseSym &S) {
    const bool host_in = A.on_device == 0;
    const int ctas = std::max(1, num_sms());
    return o.precision == TSNNLS_FP64
               ? layout_bytes<double>(A.m, A.n, A.nnz, host_in, SparseChol<double>::device_bytes(S, ctas))
               : layout_bytes<float>(A.m, A.n, A.nnz, host_in, SparseChol<float>::device_bytes(S, ctas));
}

int choose_path(const tsnnls_csr &A, const tsnnls_opts &o, size_t budget) {
    if (o.path == TSNNLS_PATH_FACTOR || o.path == TSNNLS_PATH_LSQR || o.path == TSNNLS_PATH_SPARSE)
        return o.path;
    return factor_footprint(A, o) <= budget ? TSNNLS_PATH_FACTOR : TSNNLS_PATH_LSQR;
}

size_t solve_footprint(const tsnnls_csr &A, const tsnnls_opts &o, size_t budget,
                       std::shared_ptr<const SparseSym> *sym) {
    const int path = choose_path(A, o, budget);
    if (path == TSNNLS_PATH_SPARSE) {
        auto S = analyze_gram_pattern(A, kSpNB);
        if (!S) return 0;  // malformed pattern: the solve reports TSNNLS_EINVAL
        if (sym) *sym = S;
        return sparse_footprint(A, o, *S);
    }
    return path == TSNNLS_PATH_LSQR ? lsqr_footprint(A, o) : factor_footprint(A, o);
}

static int solve_on_lane_unchecked(Context &ctx, Lane &lane, const tsnnls_csr &A, const double *b,
                                   double *x_out, const tsnnls_opts &o, tsnnls_info *info,
                                   const SolveExtras *extras);

int solve_on_lane(Context &ctx, Lane &lane, const tsnnls_csr &A, const double *b, double *x_out,
                  const tsnnls_opts &o, tsnnls_info *info, const SolveExtras *extras) {
    int st = solve_on_lane_unchecked(ctx, lane, A, b, x_out, o, info, extras);
    if (check_collect(nullptr, 0) > 0) {  // checked build: an index left its buffer
        st = TSNNLS_EBOUNDS;
        if (info) info->status = st;
    }
    return st;
}

static int solve_on_lane_unchecked(Context &ctx, Lane &lane, const tsnnls_csr &A, const double *b,
                                   double *x_out, const tsnnls_opts &o, tsnnls_info *info,
                                   const SolveExtras *extras) {
    NvtxSolve range(lane, "tsnnls_solve");
    if (info) std::memset(info, 0, sizeof(*info));
    std::memset(lane.st_host, 0, sizeof(DevStatus));
    if (choose_path(A, o, ctx.budget) == TSNNLS_PATH_LSQR)
        return solve_lsqr(ctx, lane, A, b, x_out, o, info, extras);
    if (o.precision == TSNNLS_FP64)
        return solve_factor<double>(ctx, lane, A, b, x_out, o, info, extras, false);
    int st = solve_factor<float>(ctx, lane, A, b, x_out, o, info, extras, false);
    if ((st == TSNNLS_ENOCONV || st == TSNNLS_ENOTPD) && o.no_fallback == 0) {
        // kappa(A_F)^2 too large for the FP32 factor (it loses positive
        // definiteness, or no longer preconditions the refinement): the FP64
        // factor with the same FP64 refinement
        tsnnls_opts o64 = o;
        o64.precision = TSNNLS_FP64;
        std::memset(lane.st_host, 0, sizeof(DevStatus));
        const tsnnls_info first = info ? *info : tsnnls_info{};
        st = solve_factor<double>(ctx, lane, A, b, x_out, o64, info, extras, true);
        if (st == TSNNLS_ENOMEM) st = first.status;  // no room for the FP64 copy: report the cause
        if (info) {
            info->status = st;
            info->fallback_used = 1;
            info->refine_steps += first.refine_steps;
            info->kernel_launches += first.kernel_launches;
            info->time_ms += first.time_ms;
        }
    }
    return st;
}

}  // namespace tsnnls
