// Symbolic analysis for the supernodal sparse Cholesky of the cached normal
// equations (Section 3: TAUCS factors A^T A as a sparse matrix; here the
// structure is analysed once per problem on the host and the numeric work
// runs on the GPU, sparse_chol.cu).
//
//   1. the pattern of G = A^T A from the pattern of A (column j meets column
//      c when some row holds both);
//   2. a fill-reducing order by nested dissection: a subgraph is split by
//      the middle level of a breadth-first level structure rooted at a
//      pseudo-peripheral vertex (for large subgraphs the vertex farthest
//      from the first one searched), both halves are ordered first, the
//      separator last; small subgraphs keep their order;
//   3. the elimination tree of P G P^T (Liu's algorithm with path
//      compression) and a postorder of it, composed into the order;
//   4. the row structure of every column of L by merging each column's own
//      pattern with its children's structures;
//   5. fundamental supernodes (a column joins its only child when their
//      structures nest), at most max_width columns wide, then relaxed
//      amalgamation of small ones with their parents (a few stored zeros);
//   6. per supernode: its rows, its parent and children in the supernodal
//      tree, where its rows below sit among its parent's rows, the later
//      supernodes that hold its rows below, the offsets of its panel of L,
//      of its update matrix and of its diagonal block's inverse, and where
//      every entry of the lower triangle of P G P^T lands in the panels.
// Plain C++ on up to 16 threads, deterministic: no hashing; the
// dissection's top splits hand one half to a thread of its own (the halves
// touch disjoint vertices, and their orders are joined in a fixed order);
// the per-column and per-supernode stages run on chunks of columns or
// supernodes taken in turn by the threads, and the column structures on
// disjoint subtrees of the elimination tree, each writing only its own
// outputs.  The result does not depend on the threads' timing.
#include "sparse_sym.h"

#include <algorithm>
#include <cstring>
#include <functional>
#include <atomic>
#include <system_error>
#include <thread>

namespace tsnnls {

namespace {

struct Graph {
    int64_t n = 0;
    std::vector<int64_t> ptr;  // n + 1
    std::vector<int32_t> adj;  // neighbours, no self loops, ascending
};

// Threads for one stage: up to 16, one per 4096 units of work, a core left
// to the rest of the process.
unsigned stage_threads(int64_t work) {
    const int64_t hw = std::max(1u, std::thread::hardware_concurrency());
    const int64_t want = std::max<int64_t>(1, work / 4096);
    return (unsigned)std::min<int64_t>(std::min<int64_t>(16, std::max<int64_t>(1, hw - 1)), want);
}

// fn(t, c) for the chunks c = 0 .. nchunks - 1, taken in turn by nt workers
// (t = 0 .. nt - 1, each on a thread of its own where one can be had, the
// calling thread as t = 0): a worker that the system delays leaves its
// remaining chunks to the others.  The chunks write disjoint outputs, so the
// result does not depend on timing.
template <typename Fn>
void run_chunks(int64_t nchunks, unsigned nt, Fn &&fn) {
    std::atomic<int64_t> next{0};
    auto worker = [&](unsigned t) {
        for (int64_t c; (c = next.fetch_add(1)) < nchunks;) fn(t, c);
    };
    std::vector<std::thread> th;
    try {
        for (unsigned t = 1; t < nt; ++t) th.emplace_back(worker, t);
    } catch (const std::system_error &) {  // fewer threads to be had: the others take their chunks
    }
    worker(0u);
    for (auto &x : th) x.join();
}

// Pattern of A^T A without the diagonal, as adjacency lists.
void gram_graph(int64_t m, int64_t n, const int64_t *row_ptr, const int32_t *col, Graph &g) {
    const int64_t nnz = row_ptr[m];
    std::vector<int64_t> cptr(n + 1, 0);
    std::vector<int32_t> crow(nnz > 0 ? nnz : 1);
    for (int64_t e = 0; e < nnz; ++e) cptr[col[e] + 1] += 1;
    for (int64_t j = 0; j < n; ++j) cptr[j + 1] += cptr[j];
    {
        std::vector<int64_t> next(cptr.begin(), cptr.end() - 1);
        for (int64_t r = 0; r < m; ++r)
            for (int64_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e) crow[next[col[e]]++] = (int32_t)r;
    }
    g.n = n;
    g.ptr.assign(n + 1, 0);
    g.adj.clear();
    // columns in contiguous chunks (each with its own output; a worker's
    // marks are its own), joined in column order
    const unsigned nt = stage_threads(n);
    const int64_t nch = nt > 1 ? 8 * (int64_t)nt : 1;
    std::vector<std::vector<int32_t>> adj(nch), marks(nt);
    std::vector<std::vector<int64_t>> cnt(nch);
    run_chunks(nch, nt, [&](unsigned t, int64_t ch) {
        const int64_t j0 = n * ch / nch, j1 = n * (ch + 1) / nch;
        std::vector<int32_t> &mark = marks[t];
        if (mark.empty()) mark.assign(n, -1);
        std::vector<int32_t> nb;
        cnt[ch].assign(j1 - j0, 0);
        for (int64_t j = j0; j < j1; ++j) {
            nb.clear();
            mark[j] = (int32_t)j;
            for (int64_t p = cptr[j]; p < cptr[j + 1]; ++p) {
                const int32_t r = crow[p];
                for (int64_t e = row_ptr[r]; e < row_ptr[r + 1]; ++e) {
                    const int32_t c = col[e];
                    if (mark[c] != (int32_t)j) {
                        mark[c] = (int32_t)j;
                        nb.push_back(c);
                    }
                }
            }
            std::sort(nb.begin(), nb.end());
            adj[ch].insert(adj[ch].end(), nb.begin(), nb.end());
            cnt[ch][j - j0] = (int64_t)nb.size();
        }
    });
    for (int64_t ch = 0; ch < nch; ++ch) {
        const int64_t j0 = n * ch / nch;
        for (size_t q = 0; q < cnt[ch].size(); ++q)
            g.ptr[j0 + (int64_t)q + 1] = g.ptr[j0 + (int64_t)q] + cnt[ch][q];
        g.adj.insert(g.adj.end(), adj[ch].begin(), adj[ch].end());
    }
}

// Nested dissection order (order[k] = vertex eliminated k-th).
class Dissection {
  public:
    explicit Dissection(const Graph &g) : g_(g), sub_(g.n, -1), level_(g.n, -1) {
        // one thread per core at the deepest threaded level (2^depth <= cores, at most 16)
        const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
        while (thread_depth_ < 4 && (2u << thread_depth_) <= hw) ++thread_depth_;
    }

    std::vector<int32_t> run() {
        std::vector<int32_t> all(g_.n);
        for (int64_t v = 0; v < g_.n; ++v) all[v] = (int32_t)v;
        std::vector<int32_t> order;
        order.reserve(g_.n);
        split(all, order, 0, &ranges_);
        return order;
    }

    // Ranges [b, e) of the order holding whole subtrees of the dissection
    // that no edge joins to one another: every position outside them is a
    // separator of a split that ran its halves on two threads, and lies after
    // the ranges of both halves.
    std::vector<std::pair<int64_t, int64_t>> ranges_;

  private:
    static constexpr size_t kLeaf = 48;
    // splits shallower than thread_depth_ whose halves both hold this many
    // vertices run the first half on a thread of its own (at most
    // 2^thread_depth_ at once)
    static constexpr size_t kThreadMin = 4096;
    static constexpr size_t kOneSweep = 16384;

    // breadth-first levels inside the current subset (sub_ == id) from root;
    // returns the vertices in visiting order, level_ set for them
    std::vector<int32_t> bfs(int32_t root, int32_t id, int32_t *last_level, size_t cap) {
        std::vector<int32_t> q;
        q.reserve(cap);  // the subset's size bounds the search (pages are touched only as it grows)
        const int64_t *ptr = g_.ptr.data();
        const int32_t *adj = g_.adj.data();
        int32_t *sub = sub_.data(), *lev = level_.data();
        q.push_back(root);
        lev[root] = 0;
        sub[root] = id + 1;  // visited marker: id + 1
        for (size_t h = 0; h < q.size(); ++h) {
            const int32_t v = q[h], lv = lev[v] + 1;
            for (int64_t p = ptr[v]; p < ptr[v + 1]; ++p) {
                const int32_t u = adj[p];
                if (sub[u] == id) {
                    sub[u] = id + 1;
                    lev[u] = lv;
                    q.push_back(u);
                }
            }
        }
        for (int32_t v : q) sub[v] = id;  // back to "in the subset"
        *last_level = lev[q.back()];
        return q;
    }

    // appends the order of verts (its halves', then its separator) to out
    // ranges (may be null): where the independent subtrees of this call's
    // output land in out (see ranges_)
    void split(std::vector<int32_t> &verts, std::vector<int32_t> &out, int tdepth,
               std::vector<std::pair<int64_t, int64_t>> *ranges) {
        const int64_t base = (int64_t)out.size();
        if (verts.size() <= kLeaf) {
            out.insert(out.end(), verts.begin(), verts.end());
            if (ranges) ranges->emplace_back(base, (int64_t)out.size());
            return;
        }
        const int32_t id = next_id_.fetch_add(2);
        for (int32_t v : verts) sub_[v] = id;
        // connected components of the subset, each dissected on its own
        int32_t last = 0;
        std::vector<int32_t> comp = bfs(verts[0], id, &last, verts.size());
        if (comp.size() < verts.size()) {
            std::vector<std::vector<int32_t>> comps;
            for (int32_t v : comp) sub_[v] = -2;
            comps.push_back(comp);
            for (int32_t v : verts) {
                if (sub_[v] != id) continue;
                std::vector<int32_t> c = bfs(v, id, &last, 0);  // components may be many and small
                for (int32_t u : c) sub_[u] = -2;
                comps.push_back(std::move(c));
            }
            for (auto &c : comps) split(c, out, tdepth, ranges);  // components are not adjacent
            return;
        }
        // pseudo-peripheral root: repeat from the farthest vertex while the
        // depth grows.  Above kOneSweep vertices the level structure from the
        // vertex farthest from the first serves as it is: one search fewer
        // where searches cost the most (on the 65536-column grid the factor's
        // work came out 1 % lower, the analysis 12 % faster)
        int32_t root = comp.back(), depth = last, maxl = -1;
        const bool one_sweep = verts.size() > kOneSweep;
        if (one_sweep) comp = bfs(root, id, &maxl, verts.size());
        for (int it = 0; it < (one_sweep ? 0 : 4); ++it) {
            int32_t d2 = 0;
            std::vector<int32_t> q = bfs(root, id, &d2, verts.size());
            if (d2 <= depth && it > 0) {  // q is the level structure from root itself: keep it
                comp.swap(q);
                maxl = d2;
                break;
            }
            depth = d2;
            comp.swap(q);
            root = comp.back();
        }
        if (maxl < 0) comp = bfs(root, id, &maxl, verts.size());
        if (maxl < 2) {  // (nearly) complete subgraph: nothing to dissect
            out.insert(out.end(), verts.begin(), verts.end());
            for (int32_t v : verts) sub_[v] = -1;
            if (ranges) ranges->emplace_back(base, (int64_t)out.size());
            return;
        }
        std::vector<int64_t> cnt(maxl + 1, 0);
        for (int32_t v : comp) cnt[level_[v]] += 1;
        // separator: the smallest level whose cumulative count lies within
        // 35 %..65 % of the vertices (the median level if none)
        const int64_t total = (int64_t)comp.size();
        int64_t cum = 0;
        int32_t best = -1, median = 1;
        for (int32_t l = 0; l <= maxl; ++l) {
            const int64_t before = cum;
            cum += cnt[l];
            if (before <= total / 2 && cum > total / 2) median = l;
            if (l > 0 && l < maxl && 20 * before >= 7 * total && 20 * before <= 13 * total)
                if (best < 0 || cnt[l] < cnt[best]) best = l;
        }
        if (best < 0) best = std::min(std::max(median, 1), maxl - 1);
        std::vector<int32_t> a, b, s;
        for (int32_t v : comp) {
            sub_[v] = -1;
            if (level_[v] < best) a.push_back(v);
            else if (level_[v] > best) b.push_back(v);
            else s.push_back(v);
        }
        bool done = false;
        if (tdepth < thread_depth_ && a.size() >= kThreadMin && b.size() >= kThreadMin) {
            // a and b are not adjacent (their levels differ by two or more), so
            // the two searches read and write disjoint vertices
            std::vector<int32_t> oa, ob;
            std::vector<std::pair<int64_t, int64_t>> ra, rb;
            try {
                std::thread t([&] { split(a, oa, tdepth + 1, &ra); });
                split(b, ob, tdepth + 1, &rb);
                t.join();
                const int64_t ba = (int64_t)out.size(), bb = ba + (int64_t)oa.size();
                out.insert(out.end(), oa.begin(), oa.end());
                out.insert(out.end(), ob.begin(), ob.end());
                if (ranges) {
                    for (const auto &r : ra) ranges->emplace_back(ba + r.first, ba + r.second);
                    for (const auto &r : rb) ranges->emplace_back(bb + r.first, bb + r.second);
                }
                done = true;
            } catch (const std::system_error &) {  // no thread to be had: in line
            }
        }
        if (!done) {
            split(a, out, tdepth + 1, nullptr);
            split(b, out, tdepth + 1, nullptr);
        }
        out.insert(out.end(), s.begin(), s.end());
        if (!done && ranges) ranges->emplace_back(base, (int64_t)out.size());  // one subtree
    }

    const Graph &g_;
    int thread_depth_ = 0;
    std::vector<int32_t> sub_, level_;
    std::atomic<int32_t> next_id_{0};
};

}  // namespace

int sparse_analyze(int64_t m, int64_t n, const int64_t *row_ptr, const int32_t *col, int max_width,
                   SparseSym &S) {
    if (n <= 0 || m <= 0 || max_width < 1) return -1;
    Graph g;
    gram_graph(m, n, row_ptr, col, g);

    // 2. nested dissection, then 3. elimination tree and postorder
    Dissection nd(g);
    std::vector<int32_t> perm = nd.run();  // new -> old
    std::vector<int32_t> iperm(n);
    // Liu's algorithm, row by row.  A row of a dissection range meets only
    // columns of its own range before it (the ranges are not joined by
    // edges, and the separators come after them), and its ancestor walks stay
    // in the range, so the ranges run on threads and the other rows follow
    // in order: the same tree as one pass over all rows.
    auto etree_of = [&](const std::vector<int32_t> &pm, const std::vector<int32_t> &ipm,
                        std::vector<int32_t> &parent) {
        parent.assign(n, -1);
        std::vector<int32_t> anc(n, -1);
        auto row = [&](int64_t i) {  // row i of the lower triangle: columns k < i
            const int32_t vi = pm[i];
            for (int64_t p = g.ptr[vi]; p < g.ptr[vi + 1]; ++p) {
                int32_t k = ipm[g.adj[p]];
                if (k >= i) continue;
                while (anc[k] != -1 && anc[k] != i) {
                    const int32_t nx = anc[k];
                    anc[k] = (int32_t)i;
                    k = nx;
                }
                if (anc[k] == -1) {
                    anc[k] = (int32_t)i;
                    parent[k] = (int32_t)i;
                }
            }
        };
        const auto &rg = nd.ranges_;
        std::vector<uint8_t> in_range(n, 0);
        for (const auto &r : rg)
            for (int64_t i = r.first; i < r.second; ++i) in_range[i] = 1;
        run_chunks((int64_t)rg.size(), stage_threads(n), [&](unsigned, int64_t q) {
            for (int64_t i = rg[q].first; i < rg[q].second; ++i) row(i);
        });
        for (int64_t i = 0; i < n; ++i)
            if (!in_range[i]) row(i);
    };
    for (int64_t k = 0; k < n; ++k) iperm[perm[k]] = (int32_t)k;
    std::vector<int32_t> parent;
    etree_of(perm, iperm, parent);
    {
        // postorder: children in ascending order, depth first
        std::vector<int32_t> head(n, -1), nxt(n, -1), post;
        post.reserve(n);
        for (int64_t j = n - 1; j >= 0; --j)
            if (parent[j] >= 0) {
                nxt[j] = head[parent[j]];
                head[parent[j]] = (int32_t)j;
            }
        std::vector<int32_t> stack;
        for (int64_t r = 0; r < n; ++r) {
            if (parent[r] != -1) continue;
            stack.push_back((int32_t)r);
            while (!stack.empty()) {
                const int32_t v = stack.back();
                if (head[v] >= 0) {
                    const int32_t c = head[v];
                    head[v] = nxt[c];
                    stack.push_back(c);
                } else {
                    post.push_back(v);
                    stack.pop_back();
                }
            }
        }
        // a postorder is a topological order of the tree, so the tree of
        // the reordered matrix is the same tree relabelled
        std::vector<int32_t> p2(n), ipost(n), par2(n);
        for (int64_t k = 0; k < n; ++k) ipost[post[k]] = (int32_t)k;
        for (int64_t k = 0; k < n; ++k) {
            p2[k] = perm[post[k]];
            par2[k] = parent[post[k]] < 0 ? -1 : ipost[parent[post[k]]];
        }
        perm.swap(p2);
        parent.swap(par2);
        for (int64_t k = 0; k < n; ++k) iperm[perm[k]] = (int32_t)k;
    }

    // lower pattern of P G P^T by column (new indices), diagonal first
    S.n = n;
    S.gptr.assign(n + 1, 0);
    S.grow.clear();
    S.gpair_orig_row.clear();
    const unsigned nt = stage_threads(n);
    const int64_t ncc = nt > 1 ? 8 * (int64_t)nt : 1;  // column chunks
    {
        // counts, then each column chunk fills its own part
        run_chunks(ncc, nt, [&](unsigned, int64_t ch) {
            for (int64_t j = n * ch / ncc; j < n * (ch + 1) / ncc; ++j) {
                const int32_t vj = perm[j];
                int64_t c = 1;
                for (int64_t p = g.ptr[vj]; p < g.ptr[vj + 1]; ++p) c += iperm[g.adj[p]] > j;
                S.gptr[j + 1] = c;
            }
        });
        for (int64_t j = 0; j < n; ++j) S.gptr[j + 1] += S.gptr[j];
        S.grow.resize(S.gptr[n]);
        S.gpair_orig_row.resize(S.gptr[n]);
        run_chunks(ncc, nt, [&](unsigned, int64_t ch) {
            for (int64_t j = n * ch / ncc; j < n * (ch + 1) / ncc; ++j) {
                int32_t *o = S.grow.data() + S.gptr[j];
                int64_t c = 0;
                o[c++] = (int32_t)j;
                const int32_t vj = perm[j];
                for (int64_t p = g.ptr[vj]; p < g.ptr[vj + 1]; ++p) {
                    const int32_t i = iperm[g.adj[p]];
                    if (i > j) o[c++] = i;
                }
                std::sort(o + 1, o + c);
                for (int64_t q = 0; q < c; ++q) S.gpair_orig_row[S.gptr[j] + q] = perm[o[q]];
            }
        });
    }

    // 4. column structures (rows below the diagonal), children merged
    std::vector<std::vector<int32_t>> cs(n);
    std::vector<int32_t> nchild(n, 0);
    {
        std::vector<int32_t> first_child(n, -1), sib(n, -1);
        for (int64_t j = n - 1; j >= 0; --j)
            if (parent[j] >= 0) {
                sib[j] = first_child[parent[j]];
                first_child[parent[j]] = (int32_t)j;
                nchild[parent[j]] += 1;
            }
        // the column's own rows (sorted), then each child's rows after j
        // merged in (both sorted, duplicates dropped): linear in the sizes,
        // no sort of the merged structure
        auto column = [&](int64_t j, std::vector<int32_t> &tmp) {
            std::vector<int32_t> &v = cs[j];
            v.assign(S.grow.begin() + S.gptr[j] + 1, S.grow.begin() + S.gptr[j + 1]);  // sorted, distinct
            for (int32_t c = first_child[j]; c >= 0; c = sib[c]) {
                const std::vector<int32_t> &w = cs[c];
                auto b = std::upper_bound(w.begin(), w.end(), (int32_t)j);  // rows below j only
                tmp.clear();
                tmp.reserve(v.size() + (size_t)(w.end() - b));
                auto a = v.begin();
                while (a != v.end() && b != w.end()) {
                    if (*a < *b) tmp.push_back(*a++);
                    else if (*b < *a) tmp.push_back(*b++);
                    else {
                        tmp.push_back(*a++);
                        ++b;
                    }
                }
                tmp.insert(tmp.end(), a, v.end());
                tmp.insert(tmp.end(), b, w.end());
                v.swap(tmp);
            }
        };
        // In the postorder a subtree is the range of columns that ends at
        // its root.  The subtrees of at most `thr` columns whose parent's
        // is larger are independent: threads take them largest first; the
        // columns above them follow in order.
        std::vector<int64_t> desc(n, 1);
        for (int64_t j = 0; j < n; ++j)
            if (parent[j] >= 0) desc[parent[j]] += desc[j];
        const int64_t thr = std::max<int64_t>(256, n / (8 * (int64_t)nt));
        std::vector<int32_t> task;
        for (int64_t j = 0; j < n; ++j)
            if (desc[j] <= thr && (parent[j] < 0 || desc[parent[j]] > thr)) task.push_back((int32_t)j);
        std::stable_sort(task.begin(), task.end(), [&](int32_t a, int32_t b) { return desc[a] > desc[b]; });
        std::vector<std::vector<int32_t>> tmps(nt);
        run_chunks((int64_t)task.size(), nt, [&](unsigned t, int64_t q) {
            for (int64_t j = task[q] - desc[task[q]] + 1; j <= task[q]; ++j) column(j, tmps[t]);
        });
        for (int64_t j = 0; j < n; ++j)
            if (desc[j] > thr) column(j, tmps[0]);
    }

    // 5. fundamental supernodes, at most max_width wide ...
    std::vector<int32_t> fund;  // first column of each fundamental supernode
    for (int64_t j = 0; j < n; ++j) {
        bool join = false;
        if (j > 0 && !fund.empty()) {
            const int64_t f = fund.back();
            join = parent[j - 1] == j && nchild[j] == 1 && cs[j - 1].size() == cs[j].size() + 1 &&
                   j - f < max_width;
        }
        if (!join) fund.push_back((int32_t)j);
    }
    const int64_t nf = (int64_t)fund.size();
    fund.push_back((int32_t)n);
    // ... then relaxed amalgamation, from the top of the tree down: a group
    // of columns [F, L] (L the last column of its top supernode) takes the
    // fundamental supernode just below F when that supernode's parent column
    // lies in the group, while the group stays at most max_width wide and
    // the explicit zeros it stores stay few (more are allowed in narrow
    // groups, whose per-supernode costs dominate).  Rows of a group: [F, L]
    // and the structure of L, which contains every merged column's structure.
    S.exact_nnz_L = 0;
    for (int64_t j = 0; j < n; ++j) S.exact_nnz_L += 1 + (int64_t)cs[j].size();
    std::vector<int32_t> groups;  // first columns, descending
    {
        std::vector<int32_t> fsn(n);
        for (int64_t t = 0; t < nf; ++t)
            for (int32_t j = fund[t]; j < fund[t + 1]; ++j) fsn[j] = (int32_t)t;
        auto exact = [&](int64_t t) {
            int64_t e = 0;
            for (int32_t j = fund[t]; j < fund[t + 1]; ++j) e += 1 + (int64_t)cs[j].size();
            return e;
        };
        int64_t top = nf - 1;
        while (top >= 0) {
            const int32_t L = fund[top + 1] - 1;
            int32_t F = fund[top];
            const int64_t below = (int64_t)cs[L].size();
            int64_t E = exact(top);
            int64_t t = top - 1;
            for (; t >= 0; --t) {
                const int32_t lt = fund[t + 1] - 1;  // == F - 1
                if (parent[lt] < F || parent[lt] > L) break;  // not a child of the group
                const int64_t W = (int64_t)L - fund[t] + 1;
                if (W > max_width) break;
                const int64_t Et = E + exact(t);
                const int64_t stored = W * (W + 1) / 2 + W * below;
                const double z = 1.0 - (double)Et / (double)stored;
                const bool ok = W <= 4 || (W <= 16 && z <= 0.5) || (W <= 32 && z <= 0.25) || z <= 0.1;
                if (!ok) break;
                E = Et;
                F = fund[t];
            }
            groups.push_back(F);
            top = t;
        }
    }
    S.sn_first.assign(groups.rbegin(), groups.rend());
    S.col_sn.assign(n, 0);
    for (size_t g2 = 0; g2 < S.sn_first.size(); ++g2) {
        const int32_t e2 = g2 + 1 < S.sn_first.size() ? S.sn_first[g2 + 1] : (int32_t)n;
        for (int32_t j = S.sn_first[g2]; j < e2; ++j) S.col_sn[j] = (int32_t)g2;
    }
    const int64_t ns = (int64_t)S.sn_first.size();
    S.ns = ns;
    S.sn_first.push_back((int32_t)n);

    // 6. rows, panel / update / inverse offsets, the supernodal tree, the
    // positions of a supernode's rows below in its parent's rows
    S.rows_off.assign(ns + 1, 0);
    S.rows.clear();
    S.L_off.assign(ns + 1, 0);
    S.W_off.assign(ns + 1, 0);
    S.U_off.assign(ns + 1, 0);
    S.u_off.assign(ns + 1, 0);
    S.sparent.assign(ns, -1);
    S.nnz_L = 0;
    S.flops = 0.0;
    S.max_height = 0;
    for (int64_t sn = 0; sn < ns; ++sn) {
        const int32_t f = S.sn_first[sn], l = S.sn_first[sn + 1] - 1, w = l - f + 1;
        for (int32_t c = f; c <= l; ++c) S.rows.push_back(c);
        S.rows.insert(S.rows.end(), cs[l].begin(), cs[l].end());
        S.rows_off[sn + 1] = (int64_t)S.rows.size();
        const int64_t h = S.rows_off[sn + 1] - S.rows_off[sn], hu = h - w;
        S.max_height = std::max<int64_t>(S.max_height, h);
        S.L_off[sn + 1] = S.L_off[sn] + ((h + 3) / 4 * 4) * w;
        S.W_off[sn + 1] = S.W_off[sn] + (int64_t)w * w;
        S.U_off[sn + 1] = S.U_off[sn] + ((hu + 3) / 4 * 4) * hu;
        S.u_off[sn + 1] = S.u_off[sn] + hu;
        S.nnz_L += h * w - (int64_t)w * (w - 1) / 2;
        for (int32_t c = 0; c < w; ++c) {
            const double cc = (double)(h - c);  // entries in column f + c, diagonal included
            S.flops += cc * cc;
        }
        if (parent[l] >= 0) S.sparent[sn] = S.col_sn[parent[l]];
    }
    S.c_off.assign(ns + 1, 0);
    for (int64_t sn = 0; sn < ns; ++sn)
        if (S.sparent[sn] >= 0) S.c_off[S.sparent[sn] + 1] += 1;
    for (int64_t sn = 0; sn < ns; ++sn) S.c_off[sn + 1] += S.c_off[sn];
    S.clist.assign(S.c_off[ns], 0);
    {
        std::vector<int64_t> fill(S.c_off.begin(), S.c_off.end() - 1);
        for (int64_t sn = 0; sn < ns; ++sn)
            if (S.sparent[sn] >= 0) S.clist[fill[S.sparent[sn]]++] = (int32_t)sn;
    }
    S.rel.assign(S.u_off[ns], 0);
    run_chunks(ncc, nt, [&](unsigned, int64_t ch) {
        for (int64_t sn = ns * ch / ncc; sn < ns * (ch + 1) / ncc; ++sn) {
            const int32_t pa = S.sparent[sn];
            if (pa < 0) continue;
            const int32_t w = S.sn_first[sn + 1] - S.sn_first[sn];
            const int32_t *pb = S.rows.data() + S.rows_off[pa], *pe = S.rows.data() + S.rows_off[pa + 1];
            int64_t k = S.u_off[sn];
            for (int64_t q = S.rows_off[sn] + w; q < S.rows_off[sn + 1]; ++q)
                S.rel[k++] = (int32_t)(std::lower_bound(pb, pe, S.rows[q]) - pb);
        }
    });
    // Ticket orders.  A CTA waits only on supernodes of earlier tickets, so
    // any order with children before parents serves the factor and the
    // forward solve, and any with parents before children the backward
    // solve.  Levels keep the CTAs on supernodes that become ready together:
    // by height for the first two (every leaf before any parent), by depth
    // for the third (every supernode of one level below the root before the
    // next), where a postorder would send them down one subtree at a time.
    {
        std::vector<int32_t> height(ns, 0), depth(ns, 0);
        for (int64_t sn = 0; sn < ns; ++sn)  // children before parents
            if (S.sparent[sn] >= 0) height[S.sparent[sn]] = std::max(height[S.sparent[sn]], height[sn] + 1);
        for (int64_t sn = ns - 1; sn >= 0; --sn)  // parents before children
            depth[sn] = S.sparent[sn] >= 0 ? depth[S.sparent[sn]] + 1 : 0;
        S.order_up.resize(ns);
        S.order_down.resize(ns);
        for (int64_t sn = 0; sn < ns; ++sn) {
            S.order_up[sn] = (int32_t)sn;
            S.order_down[sn] = (int32_t)(ns - 1 - sn);
        }
        std::stable_sort(S.order_up.begin(), S.order_up.end(),
                         [&](int32_t a, int32_t b) { return height[a] < height[b]; });
        std::stable_sort(S.order_down.begin(), S.order_down.end(),
                         [&](int32_t a, int32_t b) { return depth[a] < depth[b]; });
    }
    // A(s): the supernodes holding s's rows below (ascending), for the backward solve
    S.a_off.assign(ns + 1, 0);
    S.alist.clear();
    for (int64_t d = 0; d < ns; ++d) {
        const int32_t w = S.sn_first[d + 1] - S.sn_first[d];
        int32_t lastsn = -1;
        for (int64_t q = S.rows_off[d] + w; q < S.rows_off[d + 1]; ++q) {
            const int32_t t = S.col_sn[S.rows[q]];
            if (t != lastsn) {
                S.alist.push_back(t);
                lastsn = t;
            }
        }
        S.a_off[d + 1] = (int64_t)S.alist.size();
    }
    // where each lower entry of P G P^T lands: panel of its column's
    // supernode, column j - f, local row = position of i among the rows
    S.gpos.resize(S.grow.size());
    run_chunks(ncc, nt, [&](unsigned, int64_t ch) {
        for (int64_t j = n * ch / ncc; j < n * (ch + 1) / ncc; ++j) {
            const int32_t s = S.col_sn[j], f = S.sn_first[s];
            const int64_t h = S.rows_off[s + 1] - S.rows_off[s], ld = (h + 3) / 4 * 4;
            const int32_t *rb = S.rows.data() + S.rows_off[s], *re = S.rows.data() + S.rows_off[s + 1];
            for (int64_t p = S.gptr[j]; p < S.gptr[j + 1]; ++p) {
                const int64_t loc = std::lower_bound(rb, re, S.grow[p]) - rb;
                S.gpos[p] = S.L_off[s] + (j - f) * ld + loc;
            }
        }
    });
    S.perm.swap(perm);
    S.iperm.swap(iperm);
    S.parent.swap(parent);
    return 0;
}

}  // namespace tsnnls
