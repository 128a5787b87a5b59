// Host-side solver engine: owns device memory for one solve and runs the
// block principal pivoting loop of Section 2 on one CUDA stream.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "common.cuh"
#include "sparse_sym.h"
#include "tsnnls.h"

namespace tsnnls {

// One stream with its own status block; the blocking API uses lane 0, the
// asynchronous queue one lane per admitted request.
struct PhaseMark {
    int phase;
    cudaEvent_t e0, e1;
    double bytes, flops;
    int64_t launches;
};

struct Lane {
    cudaStream_t stream = nullptr;
    // look-ahead of the factorisation: high-priority side stream and its
    // fork / head / join events
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, head = nullptr, join = nullptr;
    DevStatus *st_dev = nullptr;
    DevStatus *st_host = nullptr;  // pinned mirror
    int32_t *bad_dev = nullptr;
    int32_t *bad_host = nullptr;   // pinned
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaEvent_t ev_status = nullptr;  // a status copy the host waits for later
    // per-phase accounting (tsnnls_profile_*)
    bool prof = false;
    bool prof_kernels = false;  // time the factorisation's kernels one by one
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<PhaseMark> marks;
    int64_t mark_launch0 = 0;
    tsnnls_phase_stat stats[TSNNLS_NUM_PHASES] = {};
    bool nvtx_open = false;        // a phase range is open on the NVTX stack
    bool nvtx_pivot_open = false;  // and under it a pivot's range
    // the batched path's last graph and device arena, replayed by the next
    // call of the same shape (batch.cu owns it; batch_cache_release frees it)
    void *batch_cache = nullptr;
    // the dense factorisations captured as graphs and the keys seen once
    // (engine.cu owns them; factor_graph_release frees them)
    void *factor_graphs = nullptr;
};

// Free a lane's cached batched graph and arena (the lane's stream idle).
void batch_cache_release(Lane &l);

// Free a lane's cached factorisation graphs (the lane's streams idle).
void factor_graph_release(Lane &l);

// NVTX ranges for timeline tools (Nsight Systems): one per solve and one per
// phase that prof_begin opens; inert unless a tool is attached.
struct NvtxSolve {
    Lane &l;
    NvtxSolve(Lane &lane, const char *what);
    ~NvtxSolve();
};

// Start pivot `iter`'s range (ends the previous pivot's and any open phase).
void nvtx_pivot(Lane &l, int iter);

// Bracket a phase with events on the lane's stream (no-ops unless prof).
void prof_begin(Lane &l, int phase);
void prof_end(Lane &l, double bytes, double flops);
// After the lane's stream is idle: fold the marks into l.stats.
void prof_flush(Lane &l);

struct Request {
    tsnnls_csr A;
    const double *b = nullptr;
    double *x_out = nullptr;
    tsnnls_opts opts;
    size_t footprint = 0;
    int status = TSNNLS_PENDING;
    tsnnls_info info{};
    bool done = false;
    std::shared_ptr<const SparseSym> sym;  // sparse path: the analysis made at submission
};

// Columns of a pivot-trace row (tsnnls_solve_ex).
constexpr int kTraceCols = 6;

// Extra outputs of a solve (for tests and tools); any pointer may be NULL.
struct SolveExtras {
    double *y_out = nullptr;       // n entries, same memory space as x_out
    uint8_t *inF_out = nullptr;    // n entries, same memory space as x_out
    int64_t *trace = nullptr;      // host, kTraceCols per pivot
    int64_t trace_cap = 0;
    std::shared_ptr<const SparseSym> sym;  // sparse path: an analysis already made, else NULL
};

struct Context {
    int device = 0;
    size_t budget = 0;
    size_t in_use = 0;  // bytes held by admitted requests
    Lane lane0;
    std::mutex solve_mu;  // serialises blocking calls on lane0

    // asynchronous queue (continuous batching across lanes)
    std::mutex q_mu;
    std::condition_variable q_cv, done_cv;
    std::deque<tsnnls_ticket> waiting;
    std::map<tsnnls_ticket, std::shared_ptr<Request>> requests;
    // tsnnls_submit_batch: batch ticket -> the member tickets (each an
    // ordinary queued request that only the batch ticket refers to)
    std::map<tsnnls_ticket, std::vector<tsnnls_ticket>> batches;
    tsnnls_ticket next_ticket = 1;
    std::vector<std::thread> workers;
    std::vector<Lane> lanes;
    bool stopping = false;
    int active = 0;
    int max_active = 0;
    int64_t submitted = 0, completed = 0;
    size_t max_in_use = 0;
};

int lane_create(Lane &l);
void lane_destroy(Lane &l);

// Device footprint (bytes) of one solve at this size on the path AUTO would
// take under `budget` (the factor path when its cached A^T A fits, else LSQR).
// sym (may be NULL) receives the sparse path's symbolic analysis when that
// path is taken (it is needed to size the path's device state).
size_t solve_footprint(const tsnnls_csr &A, const tsnnls_opts &o, size_t budget,
                       std::shared_ptr<const SparseSym> *sym = nullptr);
// Symbolic analysis of A^T A for the sparse path (the pattern is copied to
// the host first when A is on the device); NULL on failure.
std::shared_ptr<const SparseSym> analyze_gram_pattern(const tsnnls_csr &A, int max_width);
int choose_path(const tsnnls_csr &A, const tsnnls_opts &o, size_t budget);
size_t lsqr_footprint(const tsnnls_csr &A, const tsnnls_opts &o);
int solve_lsqr(Context &ctx, Lane &lane, const tsnnls_csr &A, const double *b, double *x_out,
               const tsnnls_opts &o, tsnnls_info *info, const SolveExtras *ex);

// Run one solve on a lane.  Thread-compatible: one caller per lane at a time.
int solve_on_lane(Context &ctx, Lane &lane, const tsnnls_csr &A, const double *b,
                  double *x_out, const tsnnls_opts &opts, tsnnls_info *info,
                  const SolveExtras *extras);

int status_from_cuda(cudaError_t e);

// Batched dense solves (batch.cu).  nb_override (count entries) forces the
// Cholesky panel width per problem; NULL uses the tuned table.
// trace (count host pointers, may be NULL; entries may be NULL): each
// problem's pivot trace, trace_cap rows of 6 (as tsnnls_solve_ex).
int run_batch_dense(Context &ctx, Lane &lane, int count, const int32_t *m, const int32_t *n,
                    const float *const *a, const double *const *b, double *const *x,
                    const tsnnls_opts &o, int32_t *status_out, tsnnls_info *info,
                    const int *nb_override, int64_t *const *trace = nullptr, int64_t trace_cap = 0);
int batch_autotune(Context &ctx, Lane &lane, bool mixed, int per_bucket);
extern int g_batch_nb_table[2][5];

}  // namespace tsnnls
