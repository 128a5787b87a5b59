// Batched dense solves (many small or uneven problems in one launch).
#include <cuda_runtime.h>
#include <stdint.h>

#include "engine.h"

extern "C" int tsnnls_solve_batch_dense(tsnnls_ctx *ctx, int32_t count, const int32_t *m,
                                        const int32_t *n, const float *const *a,
                                        const double *const *b, double *const *x_out,
                                        const tsnnls_opts *opts, int32_t *status_out,
                                        tsnnls_info *info) {
    (void)ctx; (void)count; (void)m; (void)n; (void)a; (void)b; (void)x_out; (void)opts;
    (void)status_out; (void)info;
    return TSNNLS_EINVAL;
}
