// Symbolic structure of the supernodal sparse Cholesky (sparse_sym.cpp).
#pragma once

#include <stdint.h>

#include <vector>

namespace tsnnls {

struct SparseSym {
    int64_t n = 0, ns = 0;           // columns, supernodes
    std::vector<int32_t> perm;       // new -> original column
    std::vector<int32_t> iperm;      // original -> new
    std::vector<int32_t> parent;     // elimination tree (new indices), -1 at roots
    // lower triangle of P (A^T A) P^T by column, diagonal first in each column
    std::vector<int64_t> gptr;       // n + 1
    std::vector<int32_t> grow;       // new row index of each entry
    std::vector<int32_t> gpair_orig_row;  // original index of that row
    std::vector<int64_t> gpos;       // position of each entry in the panel arena
    // supernodes, in postorder: columns sn_first[s] .. sn_first[s + 1] - 1
    std::vector<int32_t> sn_first;   // ns + 1
    std::vector<int32_t> col_sn;     // supernode of each column
    std::vector<int64_t> rows_off;   // ns + 1: rows[rows_off[s] ..] = the panel's rows,
    std::vector<int32_t> rows;       //   its own columns first, then the rows below
    std::vector<int64_t> L_off;      // ns + 1: panel s is ld x w, ld = rows rounded up to 4
    std::vector<int64_t> W_off;      // ns + 1: inverse of the diagonal block, w x w
    std::vector<int64_t> U_off;      // ns + 1: update matrix (rows below)^2, ld = rows below rounded up to 4
    std::vector<int64_t> u_off;      // ns + 1: u_off[s] .. = one entry per row below (update
                                     //   vectors of the forward solve, and rel)
    std::vector<int32_t> rel;        // position of each row below among the parent's rows
    std::vector<int32_t> sparent;    // supernodal tree, -1 at a root
    std::vector<int32_t> order_up;   // ns: the order in which CTAs take supernodes for the factor and
                                     //   the forward solve: by height (leaves first), ties in postorder
    std::vector<int32_t> order_down; // ns: the same for the backward solve: by depth (roots first),
                                     //   ties in reverse postorder
    std::vector<int64_t> c_off;      // ns + 1: clist[c_off[s] ..] = children of s, ascending
    std::vector<int32_t> clist;
    std::vector<int64_t> a_off;      // ns + 1: alist[a_off[s] ..] = supernodes holding s's rows below
    std::vector<int32_t> alist;
    int64_t nnz_L = 0;               // entries stored in the panels (lower trapezoids, with the
                                     //   zeros that amalgamation adds)
    int64_t exact_nnz_L = 0;         // entries of L's structure
    int64_t max_height = 0;          // rows of the tallest panel
    double flops = 0.0;              // sum over columns of (entries in the column)^2
    double analysis_ms = 0.0;        // host wall time of the analysis
};

// The analysis of A^T A's pattern for an m x n CSR pattern (host arrays);
// max_width caps the supernode width.  Returns 0, or -1 on bad arguments.
int sparse_analyze(int64_t m, int64_t n, const int64_t *row_ptr, const int32_t *col, int max_width,
                   SparseSym &out);

}  // namespace tsnnls
