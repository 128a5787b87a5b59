// The C ABI declared in include/tsnnls.h: contexts, the blocking and
// asynchronous solves, and the step-level entry points.
#include <cuda_runtime.h>
#include <stdint.h>

#include <chrono>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "check.cuh"
#include "engine.h"

using namespace tsnnls;

struct tsnnls_ctx {
    Context c;
};

namespace {

int check_csr_args(const tsnnls_csr *A, const double *b, const double *x_out) {
    if (!A || !b || !x_out) return TSNNLS_EINVAL;
    if (A->n <= 0 || A->m <= A->n || A->nnz < 0) return TSNNLS_EINVAL;
    if (A->n > INT32_MAX || A->m > INT32_MAX) return TSNNLS_EINVAL;
    if (!A->row_ptr || (A->nnz > 0 && (!A->col_idx || !A->val))) return TSNNLS_EINVAL;
    return TSNNLS_OK;
}

tsnnls_opts resolve_opts(const tsnnls_opts *o) {
    tsnnls_opts r;
    tsnnls_opts_default(&r);
    if (o) r = *o;
    if (r.p_max < 0) r.p_max = 0;
    if (r.max_refine <= 0) r.max_refine = 30;
    if (!(r.rel_tol > 0)) r.rel_tol = 1e-14;
    if (!(r.zero_tol >= 0)) r.zero_tol = 1e-12;
    return r;
}

void worker_loop(tsnnls_ctx *ctx, int lane_id) {
    Context &c = ctx->c;
    cudaSetDevice(c.device);
    Lane &lane = c.lanes[lane_id];
    std::unique_lock<std::mutex> lk(c.q_mu);
    for (;;) {
        std::shared_ptr<Request> req;
        c.q_cv.wait(lk, [&] {
            if (c.stopping) return true;
            for (tsnnls_ticket t : c.waiting) {
                auto &r = c.requests[t];
                if (r->footprint <= c.budget - c.in_use) return true;
            }
            return false;
        });
        if (c.stopping && c.waiting.empty()) return;
        // first request in arrival order that fits the free budget
        for (auto it = c.waiting.begin(); it != c.waiting.end(); ++it) {
            auto &r = c.requests[*it];
            if (r->footprint <= c.budget - c.in_use) {
                req = r;
                c.waiting.erase(it);
                break;
            }
        }
        if (!req) {
            if (c.stopping) return;
            continue;
        }
        c.in_use += req->footprint;
        c.active += 1;
        c.max_active = std::max(c.max_active, c.active);
        c.max_in_use = std::max(c.max_in_use, c.in_use);
        lk.unlock();
        tsnnls_info info;
        SolveExtras ex;
        ex.sym = req->sym;
        int st = solve_on_lane(c, lane, req->A, req->b, req->x_out, req->opts, &info, &ex);
        lk.lock();
        c.in_use -= req->footprint;
        c.active -= 1;
        req->status = st;
        req->info = info;
        req->done = true;
        c.completed += 1;
        c.done_cv.notify_all();
        c.q_cv.notify_all();
    }
}

}  // namespace

extern "C" {

void tsnnls_opts_default(tsnnls_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->rel_tol = 1e-14;
    o->zero_tol = 1e-12;
    o->p_max = 3;
    o->max_iter = 0;
    o->precision = TSNNLS_MIXED;
    o->path = TSNNLS_PATH_AUTO;
    o->max_refine = 30;
}

const char *tsnnls_strerror(int s) {
    switch (s) {
        case TSNNLS_OK: return "ok";
        case TSNNLS_EINVAL: return "invalid argument";
        case TSNNLS_ENOMEM: return "device allocation failed";
        case TSNNLS_EADMIT: return "problem does not fit the HBM budget";
        case TSNNLS_ENOTPD: return "Cholesky breakdown: A_F rank deficient";
        case TSNNLS_EMAXITER: return "pivot limit reached";
        case TSNNLS_ENOCONV: return "iterative refinement did not converge";
        case TSNNLS_ETIMEOUT: return "a device-side wait timed out";
        case TSNNLS_PENDING: return "pending";
        case TSNNLS_ECUDA: return "CUDA runtime error";
        case TSNNLS_ENODEV: return "no usable CUDA device";
        case TSNNLS_ENOTFOUND: return "no cache entry for the key";
        case TSNNLS_EBOUNDS: return "a kernel index left its buffer (bounds-checked build)";
        default: return "unknown status";
    }
}

int tsnnls_ctx_create(tsnnls_ctx **out, int device, size_t hbm_budget_bytes) {
    if (!out) return TSNNLS_EINVAL;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || count <= 0) return TSNNLS_ENODEV;
    if (device < 0 || device >= count) return TSNNLS_ENODEV;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return status_from_cuda(e);
    tsnnls_ctx *ctx = new (std::nothrow) tsnnls_ctx();
    if (!ctx) return TSNNLS_ENOMEM;
    ctx->c.device = device;
    size_t free_b = 0, total_b = 0;
    e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess) {
        delete ctx;
        return status_from_cuda(e);
    }
    ctx->c.budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t)(0.9 * (double)free_b);
    // keep freed stream-ordered allocations in the pool for the next solve
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    int st = lane_create(ctx->c.lane0);
    if (st != TSNNLS_OK) {
        lane_destroy(ctx->c.lane0);
        delete ctx;
        return st;
    }
    *out = ctx;
    return TSNNLS_OK;
}

static int ensure_workers(tsnnls_ctx *ctx) {
    Context &c = ctx->c;
    if (!c.workers.empty()) return TSNNLS_OK;
    int nl = 4;
    if (const char *env = std::getenv("TSNNLS_LANES")) nl = std::max(1, std::atoi(env));
    c.lanes.resize(nl);
    for (int i = 0; i < nl; ++i) {
        int st = lane_create(c.lanes[i]);
        if (st != TSNNLS_OK) return st;
    }
    for (int i = 0; i < nl; ++i) c.workers.emplace_back(worker_loop, ctx, i);
    return TSNNLS_OK;
}

void tsnnls_ctx_destroy(tsnnls_ctx *ctx) {
    if (!ctx) return;
    Context &c = ctx->c;
    {
        std::unique_lock<std::mutex> lk(c.q_mu);
        c.done_cv.wait(lk, [&] { return c.waiting.empty() && c.active == 0; });
        c.stopping = true;
        c.q_cv.notify_all();
    }
    for (auto &t : c.workers) t.join();
    for (auto &l : c.lanes) lane_destroy(l);
    lane_destroy(c.lane0);
    delete ctx;
}

int tsnnls_solve_ex(tsnnls_ctx *ctx, const tsnnls_csr *A, const double *b, double *x_out,
                    double *y_out, uint8_t *inF_out, int64_t *trace, int64_t trace_cap,
                    const tsnnls_opts *opts, tsnnls_info *info);

int tsnnls_solve(tsnnls_ctx *ctx, const tsnnls_csr *A, const double *b, double *x_out,
                 const tsnnls_opts *opts, tsnnls_info *info) {
    return tsnnls_solve_ex(ctx, A, b, x_out, nullptr, nullptr, nullptr, 0, opts, info);
}

int tsnnls_solve_ex(tsnnls_ctx *ctx, const tsnnls_csr *A, const double *b, double *x_out,
                    double *y_out, uint8_t *inF_out, int64_t *trace, int64_t trace_cap,
                    const tsnnls_opts *opts, tsnnls_info *info) {
    if (info) std::memset(info, 0, sizeof(*info));
    int st = ctx ? check_csr_args(A, b, x_out) : TSNNLS_EINVAL;
    if (st != TSNNLS_OK) {
        if (info) info->status = st;
        return st;
    }
    tsnnls_opts o = resolve_opts(opts);
    Context &c = ctx->c;
    std::lock_guard<std::mutex> g(c.solve_mu);
    cudaSetDevice(c.device);
    std::shared_ptr<const SparseSym> sym;
    if (solve_footprint(*A, o, c.budget, &sym) > c.budget) {
        if (info) info->status = TSNNLS_EADMIT;
        return TSNNLS_EADMIT;
    }
    SolveExtras ex;
    ex.sym = sym;
    ex.y_out = y_out;
    ex.inF_out = inF_out;
    ex.trace = trace;
    ex.trace_cap = trace ? trace_cap : 0;
    return solve_on_lane(c, c.lane0, *A, b, x_out, o, info, &ex);
}

int tsnnls_submit(tsnnls_ctx *ctx, const tsnnls_csr *A, const double *b, double *x_out,
                  const tsnnls_opts *opts, tsnnls_ticket *ticket) {
    if (!ctx || !ticket) return TSNNLS_EINVAL;
    int st = check_csr_args(A, b, x_out);
    if (st != TSNNLS_OK) return st;
    Context &c = ctx->c;
    auto req = std::make_shared<Request>();
    req->A = *A;
    req->b = b;
    req->x_out = x_out;
    req->opts = resolve_opts(opts);
    req->footprint = solve_footprint(*A, req->opts, c.budget, &req->sym);
    if (req->footprint > c.budget) return TSNNLS_EADMIT;
    std::lock_guard<std::mutex> g(c.q_mu);
    st = ensure_workers(ctx);
    if (st != TSNNLS_OK) return st;
    const tsnnls_ticket t = c.next_ticket++;
    c.requests[t] = req;
    c.waiting.push_back(t);
    c.submitted += 1;
    *ticket = t;
    c.q_cv.notify_all();
    return TSNNLS_OK;
}

int tsnnls_submit_batch(tsnnls_ctx *ctx, int32_t count, const tsnnls_csr *A, const double *const *b,
                        double *const *x_out, const tsnnls_opts *opts, tsnnls_ticket *ticket) {
    if (!ctx || !ticket || count <= 0 || !A || !b || !x_out) return TSNNLS_EINVAL;
    Context &c = ctx->c;
    const tsnnls_opts o = resolve_opts(opts);
    // all members are checked before any is queued: a batch is accepted whole or not at all
    std::vector<std::shared_ptr<Request>> reqs((size_t)count);
    for (int32_t i = 0; i < count; ++i) {
        int st = check_csr_args(&A[i], b[i], x_out[i]);
        if (st != TSNNLS_OK) return st;
        auto req = std::make_shared<Request>();
        req->A = A[i];
        req->b = b[i];
        req->x_out = x_out[i];
        req->opts = o;
        req->footprint = solve_footprint(A[i], o, c.budget, &req->sym);
        if (req->footprint > c.budget) return TSNNLS_EADMIT;
        reqs[(size_t)i] = std::move(req);
    }
    std::lock_guard<std::mutex> g(c.q_mu);
    int st = ensure_workers(ctx);
    if (st != TSNNLS_OK) return st;
    std::vector<tsnnls_ticket> members;
    members.reserve((size_t)count);
    for (auto &req : reqs) {
        const tsnnls_ticket t = c.next_ticket++;
        c.requests[t] = req;
        c.waiting.push_back(t);
        members.push_back(t);
    }
    const tsnnls_ticket bt = c.next_ticket++;
    c.batches[bt] = std::move(members);
    c.submitted += count;
    *ticket = bt;
    c.q_cv.notify_all();
    return TSNNLS_OK;
}

int tsnnls_batch_member_info(tsnnls_ctx *ctx, tsnnls_ticket t, int32_t i, tsnnls_info *info) {
    if (!ctx) return TSNNLS_EINVAL;
    Context &c = ctx->c;
    std::lock_guard<std::mutex> g(c.q_mu);
    auto it = c.batches.find(t);
    if (it == c.batches.end() || i < 0 || (size_t)i >= it->second.size()) return TSNNLS_EINVAL;
    const auto &req = c.requests[it->second[(size_t)i]];
    if (!req->done) return TSNNLS_PENDING;
    if (info) *info = req->info;
    return req->status;
}

int tsnnls_sparse_analyze(int64_t m, int64_t n, const int64_t *row_ptr, const int32_t *col_idx, int32_t max_width,
                          int32_t *perm_out, int32_t *parent_out, tsnnls_sparse_stats *stats) {
    if (m <= 0 || n <= 0 || n > INT32_MAX || !row_ptr || max_width < 1) return TSNNLS_EINVAL;
    tsnnls_csr A{m, n, row_ptr[m], row_ptr, col_idx, nullptr, 0};
    if (A.nnz > 0 && !col_idx) return TSNNLS_EINVAL;
    auto S = analyze_gram_pattern(A, max_width);
    if (!S) return TSNNLS_EINVAL;
    if (perm_out) std::memcpy(perm_out, S->perm.data(), sizeof(int32_t) * (size_t)n);
    if (parent_out) std::memcpy(parent_out, S->parent.data(), sizeof(int32_t) * (size_t)n);
    if (stats) {
        stats->n = n;
        stats->nnz_gram = (int64_t)S->grow.size();
        stats->nnz_l = S->exact_nnz_L;
        stats->nnz_l_stored = S->nnz_L;
        stats->update_entries = S->U_off[S->ns];
        stats->supernodes = S->ns;
        stats->max_height = S->max_height;
        stats->factor_flops = S->flops;
        stats->analysis_ms = S->analysis_ms;
    }
    return TSNNLS_OK;
}

int tsnnls_sparse_supernodes(int64_t m, int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                             int32_t max_width, int64_t *ns_out, int32_t *sn_first, int32_t *sparent,
                             int32_t *order_up, int32_t *order_down) {
    if (m <= 0 || n <= 0 || n > INT32_MAX || !row_ptr || max_width < 1 || !ns_out) return TSNNLS_EINVAL;
    tsnnls_csr A{m, n, row_ptr[m], row_ptr, col_idx, nullptr, 0};
    if (A.nnz > 0 && !col_idx) return TSNNLS_EINVAL;
    auto S = analyze_gram_pattern(A, max_width);
    if (!S) return TSNNLS_EINVAL;
    const size_t ns = (size_t)S->ns;
    *ns_out = S->ns;
    if (sn_first) std::memcpy(sn_first, S->sn_first.data(), sizeof(int32_t) * (ns + 1));
    if (sparent) std::memcpy(sparent, S->sparent.data(), sizeof(int32_t) * ns);
    if (order_up) std::memcpy(order_up, S->order_up.data(), sizeof(int32_t) * ns);
    if (order_down) std::memcpy(order_down, S->order_down.data(), sizeof(int32_t) * ns);
    return TSNNLS_OK;
}

int tsnnls_queue_stats_read(tsnnls_ctx *ctx, tsnnls_queue_stats *out) {
    if (!ctx || !out) return TSNNLS_EINVAL;
    Context &c = ctx->c;
    std::lock_guard<std::mutex> g(c.q_mu);
    out->submitted = c.submitted;
    out->completed = c.completed;
    out->max_in_use_bytes = (int64_t)c.max_in_use;
    out->budget_bytes = (int64_t)c.budget;
    out->lanes = (int32_t)c.lanes.size();
    out->max_active = c.max_active;
    return TSNNLS_OK;
}

}  // extern "C"

namespace {

// Caller holds q_mu.  True once every member of batch `members` has finished.
bool batch_done(Context &c, const std::vector<tsnnls_ticket> &members) {
    for (tsnnls_ticket m : members)
        if (!c.requests[m]->done) return false;
    return true;
}

// Caller holds q_mu; every member has finished.  The batch's status is the
// first failing member's (in submission order), else OK; info sums the
// members' counts and device times and takes the worst quality figures.
int batch_release(Context &c, tsnnls_ticket t, tsnnls_info *info) {
    auto it = c.batches.find(t);
    int st = TSNNLS_OK;
    tsnnls_info agg;
    std::memset(&agg, 0, sizeof(agg));
    for (tsnnls_ticket m : it->second) {
        const auto &r = c.requests[m];
        if (st == TSNNLS_OK && r->status != TSNNLS_OK) st = r->status;
        const tsnnls_info &v = r->info;
        agg.iters += v.iters;
        agg.refine_steps += v.refine_steps;
        agg.nF += v.nF;
        agg.path_used = agg.path_used ? agg.path_used : v.path_used;
        agg.precision_used = std::max(agg.precision_used, v.precision_used);
        agg.last_rel_step = std::max(agg.last_rel_step, v.last_rel_step);
        agg.time_ms += v.time_ms;
        agg.kernel_launches += v.kernel_launches;
        agg.cond_est = std::max(agg.cond_est, v.cond_est);
        agg.fallback_used += v.fallback_used;
        agg.factor_reuses += v.factor_reuses;
        agg.kkt_viol = std::max(agg.kkt_viol, v.kkt_viol);
        agg.rel_resid_change = std::max(agg.rel_resid_change, v.rel_resid_change);
        c.requests.erase(m);
    }
    c.batches.erase(it);
    agg.status = st;
    if (info) *info = agg;
    return st;
}

}  // namespace

extern "C" {

int tsnnls_poll(tsnnls_ctx *ctx, tsnnls_ticket t, tsnnls_info *info) {
    if (!ctx) return TSNNLS_EINVAL;
    Context &c = ctx->c;
    std::lock_guard<std::mutex> g(c.q_mu);
    auto bit = c.batches.find(t);
    if (bit != c.batches.end()) {
        if (!batch_done(c, bit->second)) return TSNNLS_PENDING;
        return batch_release(c, t, info);
    }
    auto it = c.requests.find(t);
    if (it == c.requests.end()) return TSNNLS_EINVAL;
    if (!it->second->done) return TSNNLS_PENDING;
    const int st = it->second->status;
    if (info) *info = it->second->info;
    c.requests.erase(it);
    return st;
}

int tsnnls_wait(tsnnls_ctx *ctx, tsnnls_ticket t, int64_t timeout_us, tsnnls_info *info) {
    if (!ctx) return TSNNLS_EINVAL;
    Context &c = ctx->c;
    std::unique_lock<std::mutex> lk(c.q_mu);
    auto bit = c.batches.find(t);
    if (bit != c.batches.end()) {
        const std::vector<tsnnls_ticket> members = bit->second;
        auto all_done = [&] { return batch_done(c, members); };
        if (timeout_us < 0) {
            c.done_cv.wait(lk, all_done);
        } else if (!c.done_cv.wait_for(lk, std::chrono::microseconds(timeout_us), all_done)) {
            return TSNNLS_PENDING;
        }
        return batch_release(c, t, info);
    }
    auto it = c.requests.find(t);
    if (it == c.requests.end()) return TSNNLS_EINVAL;
    auto req = it->second;
    if (timeout_us < 0) {
        c.done_cv.wait(lk, [&] { return req->done; });
    } else if (!c.done_cv.wait_for(lk, std::chrono::microseconds(timeout_us),
                                   [&] { return req->done; })) {
        return TSNNLS_PENDING;
    }
    const int st = req->status;
    if (info) *info = req->info;
    c.requests.erase(t);
    return st;
}

int tsnnls_profile_enable(tsnnls_ctx *ctx, int32_t enable) {
    if (!ctx) return TSNNLS_EINVAL;
    Context &c = ctx->c;
    std::lock_guard<std::mutex> g(c.solve_mu);
    c.lane0.prof = enable != 0;
    c.lane0.prof_kernels = enable == 2;
    std::memset(c.lane0.stats, 0, sizeof(c.lane0.stats));
    return TSNNLS_OK;
}

int tsnnls_profile_read(tsnnls_ctx *ctx, tsnnls_phase_stat *out, int32_t count) {
    if (!ctx || !out || count < 0) return TSNNLS_EINVAL;
    Context &c = ctx->c;
    std::lock_guard<std::mutex> g(c.solve_mu);
    const int nc = count < TSNNLS_NUM_PHASES ? count : TSNNLS_NUM_PHASES;
    std::memcpy(out, c.lane0.stats, sizeof(tsnnls_phase_stat) * (size_t)nc);
    return TSNNLS_OK;
}

// ---- step-level entry points ---------------------------------------------

static int finish(Lane &l, cudaError_t e) {
    if (e != cudaSuccess) {
        cudaStreamSynchronize(l.stream);
        return status_from_cuda(e);
    }
    const int st = status_from_cuda(cudaStreamSynchronize(l.stream));
    if (check_collect(nullptr, 0) > 0 && st == TSNNLS_OK) return TSNNLS_EBOUNDS;
    return st;
}

int tsnnls_gram(tsnnls_ctx *ctx, const tsnnls_csr *A, const double *b, int32_t precision,
                void *G, int64_t ldg, double *c_out) {
    if (!ctx || !A || !b || !G || !c_out || !A->on_device || A->n <= 0 || A->m <= 0 || ldg < A->n)
        return TSNNLS_EINVAL;
    Context &c = ctx->c;
    std::lock_guard<std::mutex> g(c.solve_mu);
    cudaSetDevice(c.device);
    Lane &l = c.lane0;
    const int64_t m = A->m, n = A->n, nnz = A->nnz;
    void *blk = nullptr;
    const size_t bytes = 256 * 6 + sizeof(int64_t) * (n + 1) * 2 + (sizeof(int32_t) + sizeof(double)) * (nnz + 1) + sizeof(int32_t) * (n + 1);
    cudaError_t e = cudaMallocAsync(&blk, bytes, l.stream);
    if (e != cudaSuccess) return status_from_cuda(e);
    char *p = static_cast<char *>(blk);
    auto take = [&](size_t sz) {
        char *q = p;
        p += round_up((int64_t)sz, 256);
        return q;
    };
    int64_t *col_ptr = (int64_t *)take(sizeof(int64_t) * (n + 1));
    int64_t *next = (int64_t *)take(sizeof(int64_t) * (n + 1));
    int32_t *row_idx = (int32_t *)take(sizeof(int32_t) * (nnz + 1));
    double *cval = (double *)take(sizeof(double) * (nnz + 1));
    int32_t *cnt = (int32_t *)take(sizeof(int32_t) * (n + 1));
    e = launch_csr_to_csc(l.stream, m, n, nnz, A->row_ptr, A->col_idx, A->val, col_ptr, row_idx,
                          cval, cnt, next);
    if (e == cudaSuccess) {
        if (precision == TSNNLS_FP64)
            e = launch_gram<double>(l.stream, m, n, A->row_ptr, A->col_idx, A->val, col_ptr,
                                    row_idx, cval, b, (double *)G, ldg, c_out);
        else
            e = launch_gram<float>(l.stream, m, n, A->row_ptr, A->col_idx, A->val, col_ptr, row_idx,
                                   cval, b, (float *)G, ldg, c_out);
    }
    cudaFreeAsync(blk, l.stream);
    return finish(l, e);
}

int tsnnls_gather(tsnnls_ctx *ctx, int32_t precision, const void *G, int64_t ldg,
                  const int32_t *F, int64_t k, void *S, int64_t lds) {
    if (!ctx || !G || !S || k < 0 || (k > 0 && !F) || lds < k) return TSNNLS_EINVAL;
    Context &c = ctx->c;
    std::lock_guard<std::mutex> g(c.solve_mu);
    cudaSetDevice(c.device);
    cudaError_t e =
        precision == TSNNLS_FP64
            ? launch_gather<double>(c.lane0.stream, (const double *)G, ldg, F, nullptr, k, (double *)S, lds)
            : launch_gather<float>(c.lane0.stream, (const float *)G, ldg, F, nullptr, k, (float *)S, lds);
    return finish(c.lane0, e);
}

int tsnnls_cholesky(tsnnls_ctx *ctx, int32_t precision, void *S, int64_t k, int64_t lds,
                    int32_t *info_out) {
    if (!ctx || !S || k < 0 || lds < k) return TSNNLS_EINVAL;
    Context &c = ctx->c;
    std::lock_guard<std::mutex> g(c.solve_mu);
    cudaSetDevice(c.device);
    Lane &l = c.lane0;
    cudaError_t e = cudaMemsetAsync(l.st_dev, 0, sizeof(DevStatus), l.stream);
    // the factor kernels want 16-byte aligned columns of a multiple of 32
    // rows: any other layout is factored in an aligned copy and copied back
    const size_t es = precision == TSNNLS_FP64 ? sizeof(double) : sizeof(float);
    void *work = S;
    int64_t ldw = lds;
    void *copy = nullptr;
    if (k > 0 && (lds % 32 != 0 || (reinterpret_cast<uintptr_t>(S) & 15) != 0)) {
        ldw = round_up(k, 32);
        if (e == cudaSuccess) e = cudaMallocAsync(&copy, es * (size_t)ldw * (size_t)k, l.stream);
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(copy, es * ldw, S, es * lds, es * k, k, cudaMemcpyDeviceToDevice, l.stream);
        work = copy;
    }
    float *panel = nullptr;
    TcPanel tc;
    if (e == cudaSuccess && precision != TSNNLS_FP64 && k > 0) {
        e = cudaMallocAsync(reinterpret_cast<void **>(&panel), sizeof(float) * (size_t)k * 256, l.stream);
        if (e == cudaSuccess) tc_panel_init(tc, panel, panel + (size_t)k * 128, k);
    }
    const FactorStreams fs{l.side, l.fork, l.head, l.join};
    if (e == cudaSuccess)
        e = precision == TSNNLS_FP64
                ? launch_cholesky<double>(l.stream, (double *)work, k, ldw, l.st_dev, nullptr, nullptr, &fs)
                : launch_cholesky<float>(l.stream, (float *)work, k, ldw, l.st_dev, &tc, nullptr, &fs);
    if (panel) cudaFreeAsync(panel, l.stream);
    if (copy) {
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(S, es * lds, copy, es * ldw, es * k, k, cudaMemcpyDeviceToDevice, l.stream);
        cudaFreeAsync(copy, l.stream);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(l.st_host, l.st_dev, sizeof(DevStatus), cudaMemcpyDeviceToHost, l.stream);
    int st = finish(l, e);
    if (st != TSNNLS_OK) return st;
    if (info_out) *info_out = l.st_host->chol_info;
    return l.st_host->chol_info ? TSNNLS_ENOTPD : TSNNLS_OK;
}

int tsnnls_chol_solve(tsnnls_ctx *ctx, int32_t precision, const void *L, int64_t k, int64_t lds,
                      void *rhs) {
    if (!ctx || !L || !rhs || k < 0 || lds < k) return TSNNLS_EINVAL;
    Context &c = ctx->c;
    std::lock_guard<std::mutex> g(c.solve_mu);
    cudaSetDevice(c.device);
    Lane &l = c.lane0;
    void *scratch = nullptr;
    const size_t es = precision == TSNNLS_FP64 ? sizeof(double) : sizeof(float);
    cudaError_t e = cudaMallocAsync(&scratch, chol_solve_scratch_bytes(k, es), l.stream);
    if (e != cudaSuccess) return status_from_cuda(e);
    e = cudaMemsetAsync(l.st_dev, 0, sizeof(DevStatus), l.stream);
    if (e == cudaSuccess)
        e = precision == TSNNLS_FP64
                ? launch_chol_solve<double>(l.stream, (const double *)L, k, lds, (double *)rhs, scratch, l.st_dev)
                : launch_chol_solve<float>(l.stream, (const float *)L, k, lds, (float *)rhs, scratch, l.st_dev);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(l.st_host, l.st_dev, sizeof(DevStatus), cudaMemcpyDeviceToHost, l.stream);
    cudaFreeAsync(scratch, l.stream);
    int st = finish(l, e);
    if (st != TSNNLS_OK) return st;
    return l.st_host->timeout ? TSNNLS_ETIMEOUT : TSNNLS_OK;
}

int tsnnls_spmv(tsnnls_ctx *ctx, const tsnnls_csr *A, int32_t trans, double alpha,
                const double *x, double beta, const double *z, double *out) {
    if (!ctx || !A || !A->on_device || !x || !out || (beta != 0.0 && !z) || A->m <= 0 || A->n <= 0)
        return TSNNLS_EINVAL;
    Context &c = ctx->c;
    std::lock_guard<std::mutex> g(c.solve_mu);
    cudaSetDevice(c.device);
    Lane &l = c.lane0;
    const int64_t m = A->m, n = A->n, nnz = A->nnz;
    if (!trans) {
        cudaError_t e = launch_spmv(l.stream, m, A->row_ptr, A->col_idx, A->val, alpha, x, n, beta, z,
                                    out, (double)nnz / (double)m);
        return finish(l, e);
    }
    void *blk = nullptr;
    const size_t bytes = 256 * 6 + sizeof(int64_t) * (n + 1) * 2 + (sizeof(int32_t) + sizeof(double)) * (nnz + 1) + sizeof(int32_t) * (n + 1);
    cudaError_t e = cudaMallocAsync(&blk, bytes, l.stream);
    if (e != cudaSuccess) return status_from_cuda(e);
    char *p = static_cast<char *>(blk);
    auto take = [&](size_t sz) {
        char *q = p;
        p += round_up((int64_t)sz, 256);
        return q;
    };
    int64_t *col_ptr = (int64_t *)take(sizeof(int64_t) * (n + 1));
    int64_t *next = (int64_t *)take(sizeof(int64_t) * (n + 1));
    int32_t *row_idx = (int32_t *)take(sizeof(int32_t) * (nnz + 1));
    double *cval = (double *)take(sizeof(double) * (nnz + 1));
    int32_t *cnt = (int32_t *)take(sizeof(int32_t) * (n + 1));
    e = launch_csr_to_csc(l.stream, m, n, nnz, A->row_ptr, A->col_idx, A->val, col_ptr, row_idx,
                          cval, cnt, next);
    if (e == cudaSuccess)
        e = launch_spmv(l.stream, n, col_ptr, row_idx, cval, alpha, x, m, beta, z, out,
                        (double)nnz / (double)n);
    cudaFreeAsync(blk, l.stream);
    return finish(l, e);
}

int tsnnls_solve_batch_dense(tsnnls_ctx *ctx, int32_t count, const int32_t *m, const int32_t *n,
                             const float *const *a, const double *const *b, double *const *x_out,
                             const tsnnls_opts *opts, int32_t *status_out, tsnnls_info *info);

}  // extern "C"

extern "C" {

int tsnnls_solve_batch_dense_ex(tsnnls_ctx *ctx, int32_t count, const int32_t *m, const int32_t *n,
                                const float *const *a, const double *const *b, double *const *x_out,
                                const tsnnls_opts *opts, int32_t *status_out, tsnnls_info *info,
                                int64_t *const *trace, int64_t trace_cap);

int tsnnls_solve_batch_dense(tsnnls_ctx *ctx, int32_t count, const int32_t *m, const int32_t *n,
                             const float *const *a, const double *const *b, double *const *x_out,
                             const tsnnls_opts *opts, int32_t *status_out, tsnnls_info *info) {
    return tsnnls_solve_batch_dense_ex(ctx, count, m, n, a, b, x_out, opts, status_out, info, nullptr, 0);
}

int tsnnls_solve_batch_dense_ex(tsnnls_ctx *ctx, int32_t count, const int32_t *m, const int32_t *n,
                                const float *const *a, const double *const *b, double *const *x_out,
                                const tsnnls_opts *opts, int32_t *status_out, tsnnls_info *info,
                                int64_t *const *trace, int64_t trace_cap) {
    if (info) std::memset(info, 0, sizeof(*info));
    if (!ctx || count <= 0 || !m || !n || !a || !b || !x_out) return TSNNLS_EINVAL;
    if (trace && (trace_cap <= 0 || trace_cap > (1 << 20))) return TSNNLS_EINVAL;
    for (int i = 0; i < count; ++i) {
        if (n[i] <= 0 || m[i] <= n[i] || n[i] > 1024 || !a[i] || !b[i] || !x_out[i]) {
            if (info) info->status = TSNNLS_EINVAL;
            return TSNNLS_EINVAL;
        }
    }
    tsnnls_opts o = resolve_opts(opts);
    Context &c = ctx->c;
    std::lock_guard<std::mutex> g(c.solve_mu);
    cudaSetDevice(c.device);
    return run_batch_dense(c, c.lane0, count, m, n, a, b, x_out, o, status_out, info, nullptr,
                           trace, trace ? trace_cap : 0);
}

int tsnnls_batch_autotune(tsnnls_ctx *ctx, int32_t precision, int32_t per_bucket, int32_t *nb_out) {
    if (!ctx || (precision != TSNNLS_MIXED && precision != TSNNLS_FP64)) return TSNNLS_EINVAL;
    Context &c = ctx->c;
    std::lock_guard<std::mutex> g(c.solve_mu);
    cudaSetDevice(c.device);
    const bool mixed = precision == TSNNLS_MIXED;
    int st = batch_autotune(c, c.lane0, mixed, per_bucket > 0 ? per_bucket : 64);
    if (nb_out)
        for (int i = 0; i < 5; ++i) nb_out[i] = g_batch_nb_table[mixed ? 0 : 1][i];
    return st;
}

#ifndef TSNNLS_BUILD_ID
#define TSNNLS_BUILD_ID "unversioned"
#endif

static std::string tune_key(const Context &c, int32_t precision, int32_t per_bucket) {
    cudaDeviceProp p{};
    if (cudaGetDeviceProperties(&p, c.device) != cudaSuccess) return std::string();
    char buf[512];
    snprintf(buf, sizeof buf, "%s|sm_%d%d|%d SMs|%s|per_bucket %d|build %s", p.name, p.major, p.minor,
             p.multiProcessorCount, precision == TSNNLS_MIXED ? "mixed" : "fp64",
             per_bucket > 0 ? per_bucket : 64, TSNNLS_BUILD_ID);
    return std::string(buf);
}

int tsnnls_batch_tune_key(tsnnls_ctx *ctx, int32_t precision, int32_t per_bucket, char *buf, size_t len) {
    if (!ctx || !buf || (precision != TSNNLS_MIXED && precision != TSNNLS_FP64)) return TSNNLS_EINVAL;
    const std::string k = tune_key(ctx->c, precision, per_bucket);
    if (k.empty()) return TSNNLS_ECUDA;
    if (k.size() + 1 > len) return TSNNLS_EINVAL;
    memcpy(buf, k.c_str(), k.size() + 1);
    return TSNNLS_OK;
}

int tsnnls_batch_autotune_cached(tsnnls_ctx *ctx, int32_t precision, int32_t per_bucket,
                                 const char *cache_path, int32_t *nb_out, int32_t *hit_out) {
    if (!ctx || !cache_path || (precision != TSNNLS_MIXED && precision != TSNNLS_FP64)) return TSNNLS_EINVAL;
    const std::string key = tune_key(ctx->c, precision, per_bucket);
    if (key.empty()) return TSNNLS_ECUDA;
    int32_t nb[5];
    int st = tsnnls_tune_cache_get(cache_path, key.c_str(), nb);
    if (st == TSNNLS_OK) {
        st = tsnnls_batch_set_panel(precision, nb);
        if (st != TSNNLS_OK) return st;  // an entry outside [4, 64]: not ours
        if (hit_out) *hit_out = 1;
        if (nb_out) memcpy(nb_out, nb, sizeof nb);
        return TSNNLS_OK;
    }
    if (st != TSNNLS_ENOTFOUND) return st;
    st = tsnnls_batch_autotune(ctx, precision, per_bucket, nb);
    if (st != TSNNLS_OK) return st;
    st = tsnnls_tune_cache_put(cache_path, key.c_str(), nb);
    if (st != TSNNLS_OK) return st;
    if (hit_out) *hit_out = 0;
    if (nb_out) memcpy(nb_out, nb, sizeof nb);
    return TSNNLS_OK;
}

int tsnnls_check_build(void) {
#ifdef TSNNLS_CHECK
    return 1;
#else
    return 0;
#endif
}

int tsnnls_check_report(char *buf, size_t len) { return check_report(buf, len); }

int tsnnls_batch_set_panel(int32_t precision, const int32_t *nb) {
    if (!nb || (precision != TSNNLS_MIXED && precision != TSNNLS_FP64)) return TSNNLS_EINVAL;
    for (int i = 0; i < 5; ++i)
        if (nb[i] < 4 || nb[i] > 64) return TSNNLS_EINVAL;
    for (int i = 0; i < 5; ++i) g_batch_nb_table[precision == TSNNLS_MIXED ? 0 : 1][i] = nb[i];
    return TSNNLS_OK;
}

}  // extern "C"
