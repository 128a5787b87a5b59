// Supernodal sparse Cholesky on the GPU (sparse_chol.cu): device copy of the
// symbolic structure and the per-pivot factor and solves.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "sparse_sym.h"

namespace tsnnls {

// Device view of a SparseSym (pointers into one allocation).
struct SpDev {
    int64_t n, ns;
    const int32_t *sn_first;
    const int64_t *rows_off;
    const int32_t *rows;
    const int64_t *L_off, *W_off, *U_off, *u_off, *c_off, *a_off;
    const int32_t *clist, *alist, *rel;
    const int32_t *perm;
    const int64_t *gptr;
    const int32_t *grow_orig, *gcol_orig;
    const int64_t *gpos;
    double *gval;        // A^T A on its lower pattern (FP64)
    const int32_t *order_up, *order_down;  // ticket -> supernode (factor and forward; backward)
    int32_t *flags;      // per supernode: done
    int32_t *ticket;     // ticket counter, then the abort flag
    int32_t *abort;
    // shared jobs of the FP32 factor (extend-add, rows below, update
    // matrix), two slots per CTA: the word holds kind << 62 | (supernode + 1)
    // << 40 | blocks << 20 | next block to claim (0 = no job); done counts
    // the finished blocks
    unsigned long long *job_word;
    int32_t *job_done;
    int32_t njobs;
};

// Job slots (the factor launches at most this many CTAs).
constexpr int kSpJobSlots = 1024;

// Widest supernode, for both precisions (the FP64 redo of a mixed solve
// reuses the same analysis): the dense block size of the factor kernel.
constexpr int kSpNB = 64;

template <typename T>
struct SparseChol {
    SpDev D{};
    T *Lmem = nullptr;      // panels
    T *Wmem = nullptr;      // inverses of the diagonal blocks
    T *Umem = nullptr;      // update matrices
    T *umem = nullptr;      // update vectors of the forward solve
    int32_t *permF = nullptr;  // per position of the order: its variable if in F, else -1
    int64_t max_height = 0;
    int ctas = 1;

    static int nb();  // widest supernode: the dense block size of the factor
    // device bytes for S (one allocation, 256-byte aligned pieces)
    static size_t device_bytes(const SparseSym &S, int ctas);
    // copy the structure into mem and compute A^T A on its pattern from the
    // CSC copy of A (rows ascending); waits for the copies
    cudaError_t setup(const SparseSym &S, void *mem, cudaStream_t s, const int64_t *col_ptr,
                      const int32_t *row_idx, const double *cval);
    cudaError_t reset(cudaStream_t s);
    // factor P (A^T A)_FF P^T (+ identity outside F); st->chol_info, st->timeout
    cudaError_t factor(cudaStream_t s, const uint8_t *inF, DevStatus *st);
    // permF for the current F
    cudaError_t perm_list(cudaStream_t s, const uint8_t *inF);
    // v (n entries in the factor's order) <- (L L^T)^{-1} v
    cudaError_t solve(cudaStream_t s, T *v, DevStatus *st);
};

}  // namespace tsnnls
