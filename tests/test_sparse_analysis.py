"""Symbolic analysis of the sparse path (host only, no GPU).

tsnnls_sparse_analyze orders A^T A by nested dissection, builds the
elimination tree in postorder and the structure of L.  The checks below
recompute that structure from the definition: boolean elimination on the
reordered pattern (eliminating column k joins every pair of rows below it
that column k holds), independent of the library's merging algorithm.
"""
import numpy as np
import pytest

import workloads

ts = pytest.importorskip("paper_cs_0408029_gb300")


def _gram_pattern(p):
    a = np.zeros((p.m, p.n), dtype=bool)
    rows = np.repeat(np.arange(p.m), np.diff(p.row_ptr))
    a[rows, p.col_idx] = True
    g = (a.T.astype(np.int64) @ a.astype(np.int64)) > 0
    np.fill_diagonal(g, True)
    return g


def _elimination_fill(pat):
    """Boolean Cholesky structure (lower, diagonal included) of a symmetric pattern."""
    b = pat.copy()
    n = b.shape[0]
    for k in range(n):
        below = np.nonzero(b[k + 1:, k])[0] + k + 1
        if below.size:
            b[np.ix_(below, below)] = True
    return np.tril(b)


def _cases():
    return [workloads.grid_sparse(9, seed=3), workloads.grid_sparse(12, seed=4, per_row=3),
            workloads.random_sparse(60, 40, 0.08, seed=5),
            workloads.dense_to_csr(np.random.default_rng(6).standard_normal((30, 20)),
                                   np.zeros(30))]


@pytest.mark.parametrize("case", range(4))
def test_structure_matches_boolean_elimination(case):
    p = _cases()[case]
    perm, parent, st = ts.sparse_analyze(p.m, p.n, p.row_ptr, p.col_idx)
    n = p.n
    assert np.array_equal(np.sort(perm), np.arange(n))
    assert st["nnz_l_stored"] >= st["nnz_l"]
    g = _gram_pattern(p)
    pg = g[np.ix_(perm, perm)]
    assert st["nnz_gram"] == np.tril(pg).sum()
    L = _elimination_fill(pg)
    assert st["nnz_l"] == L.sum()
    counts = L.sum(axis=0)
    # without merging (one column per supernode) the stored structure is L's own
    _, _, narrow = ts.sparse_analyze(p.m, p.n, p.row_ptr, p.col_idx, max_width=1)
    assert narrow["nnz_l_stored"] == narrow["nnz_l"] == L.sum()
    assert narrow["factor_flops"] == pytest.approx(float((counts.astype(np.float64) ** 2).sum()))
    # elimination tree: the first row below the diagonal in each column of L
    for j in range(n):
        below = np.nonzero(L[j + 1:, j])[0]
        assert parent[j] == (j + 1 + below[0] if below.size else -1), j
    # postorder: every subtree occupies the positions just before its root
    size = np.ones(n, dtype=np.int64)
    for j in range(n):
        if parent[j] >= 0:
            assert parent[j] > j
            size[parent[j]] += size[j]
    for j in range(n):
        if parent[j] >= 0:
            assert j >= parent[j] - size[parent[j]] + 1


def test_width_cap_changes_supernodes_not_structure():
    p = workloads.grid_sparse(14, seed=7)
    _, _, wide = ts.sparse_analyze(p.m, p.n, p.row_ptr, p.col_idx, max_width=64)
    _, _, narrow = ts.sparse_analyze(p.m, p.n, p.row_ptr, p.col_idx, max_width=1)
    assert narrow["supernodes"] == p.n
    assert wide["supernodes"] < narrow["supernodes"]
    assert wide["nnz_l"] == narrow["nnz_l"]


def test_dissection_beats_a_random_order():
    """Nested dissection on the grid pattern fills far less than a random order."""
    p = workloads.grid_sparse(14, seed=8)
    perm, _, st = ts.sparse_analyze(p.m, p.n, p.row_ptr, p.col_idx)
    g = _gram_pattern(p)
    rnd = np.random.default_rng(0).permutation(p.n)
    assert st["nnz_l"] < 0.6 * _elimination_fill(g[np.ix_(rnd, rnd)]).sum()


def test_gram_density_of_the_grid_workload():
    """The sparse-path workload keeps A^T A far below 5 % dense."""
    p = workloads.grid_sparse(64, seed=9)
    _, _, st = ts.sparse_analyze(p.m, p.n, p.row_ptr, p.col_idx)
    density = (2 * st["nnz_gram"] - p.n) / float(p.n) ** 2
    assert density < 0.01
    assert st["nnz_l"] < 0.05 * p.n * (p.n + 1) / 2


def test_malformed_pattern_rejected():
    p = workloads.grid_sparse(5, seed=1)
    bad = p.col_idx.copy()
    bad[3] = p.n  # out of range
    with pytest.raises(ts.TsnnlsError) as e:
        ts.sparse_analyze(p.m, p.n, p.row_ptr, bad)
    assert e.value.status == ts.EINVAL


def test_threaded_analysis_is_repeatable():
    """A 160 x 160 grid (25600 columns) runs every threaded stage and the
    dissection's one-search rule for large subgraphs: repeated analyses
    give the same order, tree and structure, the tree is a postorder
    (children before parents, every subtree just before its root) and the
    order is a permutation."""
    p = workloads.grid_sparse(160, seed=10)
    runs = [ts.sparse_analyze(p.m, p.n, p.row_ptr, p.col_idx) for _ in range(3)]
    perm, parent, st = runs[0]
    for pm, pa, s in runs[1:]:
        assert np.array_equal(pm, perm) and np.array_equal(pa, parent)
        assert {k: v for k, v in s.items() if k != "analysis_ms"} == \
            {k: v for k, v in st.items() if k != "analysis_ms"}
    n = p.n
    assert np.array_equal(np.sort(perm), np.arange(n))
    size = np.ones(n, dtype=np.int64)
    for j in range(n):
        if parent[j] >= 0:
            assert parent[j] > j
            size[parent[j]] += size[j]
    for j in range(n):
        if parent[j] >= 0:
            assert j >= parent[j] - size[parent[j]] + 1
    assert st["nnz_l_stored"] >= st["nnz_l"] > 0


@pytest.mark.parametrize("case", range(3))
def test_ticket_orders_are_topological(case):
    """The persistent sparse kernels take supernodes by ticket and wait only
    on smaller tickets: the factor and the forward solve on children
    (order_up must put every child before its parent), the backward solve on
    the supernodes holding a supernode's rows below, its ancestors (order_down
    must put every parent before its children).  Both orders are
    permutations; order_up goes by height and order_down by depth; the
    supernodes tile the columns in postorder with parents after children."""
    p = [workloads.grid_sparse(96, seed=11), workloads.random_sparse(900, 700, 0.01, seed=31),
         workloads.grid_sparse(7, seed=2)][case]
    first, sparent, up, down = ts.sparse_supernodes(p.m, p.n, p.row_ptr, p.col_idx)
    ns = sparent.size
    assert first[0] == 0 and first[-1] == p.n and np.all(np.diff(first) >= 1)
    assert np.all(np.diff(first) <= 64)
    assert np.all((sparent == -1) | (sparent > np.arange(ns)))
    for order in (up, down):
        assert np.array_equal(np.sort(order), np.arange(ns))
    pos_up = np.empty(ns, dtype=np.int64)
    pos_up[up] = np.arange(ns)
    pos_down = np.empty(ns, dtype=np.int64)
    pos_down[down] = np.arange(ns)
    has = sparent >= 0
    child = np.nonzero(has)[0]
    assert np.all(pos_up[child] < pos_up[sparent[child]])
    assert np.all(pos_down[child] > pos_down[sparent[child]])
    height = np.zeros(ns, dtype=np.int64)
    for s in range(ns):  # children before parents
        if sparent[s] >= 0:
            height[sparent[s]] = max(height[sparent[s]], height[s] + 1)
    depth = np.zeros(ns, dtype=np.int64)
    for s in range(ns - 1, -1, -1):  # parents before children
        if sparent[s] >= 0:
            depth[s] = depth[sparent[s]] + 1
    assert np.all(np.diff(height[up]) >= 0)
    assert np.all(np.diff(depth[down]) >= 0)
