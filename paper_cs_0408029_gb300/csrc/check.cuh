// Device-side bounds checks of the debug build (nvcc -DTSNNLS_CHECK).
//
// TS_IN(i, bound) is true when 0 <= i < bound.  In the checked build a false
// result also records the first failing site of this translation unit (source
// line, index, bound) and counts every failure; the caller then skips or
// redirects the access, so a bad index never reaches memory and never traps.
// In the normal build TS_IN is the constant true and costs nothing.
//
// Every .cu file that uses TS_IN ends with TSNNLS_CHECK_UNIT(name): in the
// checked build that registers the file's record with the host, which folds
// all records into the solve's status after the stream is idle
// (check_collect(), TSNNLS_EBOUNDS) and resets them.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tsnnls {

struct CheckRecord {
    int32_t hits;   // failing accesses since the last collection
    int32_t line;   // source line of the first one
    int64_t index;  // its index
    int64_t bound;  // and the bound it broke
};

using CheckCollectFn = int (*)(CheckRecord *out);  // copies and clears one unit's record

// Host registry of the units' collectors (empty in the normal build).
struct CheckRegistrar {
    CheckRegistrar(const char *unit, CheckCollectFn fn);
};

// Fold every unit's record: the number of failing accesses since the last
// call (0 in the normal build) and a one-line description of the first.
int check_collect(char *what, size_t len);

// Failing accesses collected since the previous call, and the first one's
// description in buf; clears both (tsnnls_check_report).
int check_report(char *buf, size_t len);

}  // namespace tsnnls

#ifdef TSNNLS_CHECK

namespace tsnnls {
namespace {
__device__ CheckRecord g_check_record;  // this translation unit's

__device__ __noinline__ bool check_fail(int line, int64_t index, int64_t bound) {
    if (atomicAdd(&g_check_record.hits, 1) == 0) {
        g_check_record.line = line;
        g_check_record.index = index;
        g_check_record.bound = bound;
    }
    return false;
}
}  // namespace
}  // namespace tsnnls

#define TS_IN(i, bound)                                                                     \
    ((unsigned long long)(long long)(i) < (unsigned long long)(long long)(bound) ||        \
     ::tsnnls::check_fail(__LINE__, (int64_t)(i), (int64_t)(bound)))

#define TSNNLS_CHECK_UNIT(name)                                                             \
    namespace tsnnls {                                                                      \
    namespace {                                                                             \
    int check_collect_unit(CheckRecord *out) {                                              \
        CheckRecord zero{};                                                                 \
        if (cudaMemcpyFromSymbol(out, g_check_record, sizeof(CheckRecord)) != cudaSuccess)  \
            return -1;                                                                      \
        if (out->hits != 0) cudaMemcpyToSymbol(g_check_record, &zero, sizeof(CheckRecord)); \
        return 0;                                                                           \
    }                                                                                       \
    const CheckRegistrar check_registrar(name, &check_collect_unit);                        \
    }                                                                                       \
    }

#else

#define TS_IN(i, bound) true
#define TSNNLS_CHECK_UNIT(name)

#endif
