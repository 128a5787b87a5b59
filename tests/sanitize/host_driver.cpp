// Host sanitizer run of the library's host-only C++ (test infrastructure).
//
// Compiled together with csrc/sparse_sym.cpp and csrc/tune_cache.cpp under
// -fsanitize=address,undefined.  It runs the sparse symbolic analysis over
// seeded patterns (a 2-D grid, random rows, an empty column, a single
// column, a dense block, a path) at both supernode widths and checks the
// structure it returns: perm and iperm are inverse permutations, the
// elimination tree points upward, the supernodes tile the columns, every
// entry of the lower pattern of P (A^T A) P^T lands inside its supernode's
// panel, and every row below a supernode is found among its parent's rows.
// It then writes and reads a tuning cache file.  Exit status 0 iff every
// check holds; a sanitizer report aborts the run.
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <unistd.h>

#include <algorithm>
#include <set>
#include <string>
#include <vector>

#include "sparse_sym.h"
#include "tsnnls.h"

using namespace tsnnls;

static uint64_t g_state = 0x243f6a8885a308d3ull;
static uint64_t next_u64() {  // splitmix64
    uint64_t z = (g_state += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

struct Pattern {
    int64_t m, n;
    std::vector<int64_t> rp;
    std::vector<int32_t> ci;
};

static Pattern from_rows(int64_t n, const std::vector<std::vector<int32_t>> &rows) {
    Pattern p{(int64_t)rows.size(), n, {0}, {}};
    for (auto r : rows) {
        std::sort(r.begin(), r.end());
        r.erase(std::unique(r.begin(), r.end()), r.end());
        for (int32_t c : r) p.ci.push_back(c);
        p.rp.push_back((int64_t)p.ci.size());
    }
    return p;
}

static Pattern grid(int g) {  // rows couple grid neighbours, two rows per point
    const int64_t n = (int64_t)g * g;
    std::vector<std::vector<int32_t>> rows;
    for (int rep = 0; rep < 2; ++rep)
        for (int i = 0; i < g; ++i)
            for (int j = 0; j < g; ++j) {
                const int32_t c = i * g + j;
                std::vector<int32_t> r{c};
                if (rep == 0 && j + 1 < g) r.push_back(c + 1);
                if (rep == 1 && i + 1 < g) r.push_back(c + g);
                rows.push_back(r);
            }
    return from_rows(n, rows);
}

static Pattern random_rows(int64_t m, int64_t n, int per_row, int64_t empty_col) {
    std::vector<std::vector<int32_t>> rows(m);
    for (int64_t i = 0; i < m; ++i) {
        if (i < n && i != empty_col) rows[i].push_back((int32_t)i);
        for (int k = 0; k < per_row; ++k) {
            const int32_t c = (int32_t)(next_u64() % (uint64_t)n);
            if (c != empty_col) rows[i].push_back(c);
        }
    }
    return from_rows(n, rows);
}

static int fail(const char *what, int64_t a = 0, int64_t b = 0) {
    fprintf(stderr, "check failed: %s (%lld, %lld)\n", what, (long long)a, (long long)b);
    return 1;
}

static int check(const Pattern &p, int width) {
    SparseSym S;
    if (sparse_analyze(p.m, p.n, p.rp.data(), p.ci.data(), width, S) != 0) return fail("analyze");
    const int64_t n = p.n;
    if (S.n != n || (int64_t)S.perm.size() != n || (int64_t)S.iperm.size() != n) return fail("sizes");
    for (int64_t j = 0; j < n; ++j) {
        if (S.perm[j] < 0 || S.perm[j] >= n || S.iperm[S.perm[j]] != j) return fail("perm", j);
        if (S.parent[j] != -1 && S.parent[j] <= j) return fail("etree", j, S.parent[j]);
    }
    if (S.sn_first.front() != 0 || S.sn_first.back() != n) return fail("supernode ends");
    for (int64_t s = 0; s < S.ns; ++s) {
        const int w = S.sn_first[s + 1] - S.sn_first[s];
        if (w <= 0 || w > width) return fail("width", s, w);
        const int64_t h = S.rows_off[s + 1] - S.rows_off[s];
        if (h < w) return fail("height", s, h);
        for (int64_t q = 0; q < h; ++q) {  // own columns first, then ascending rows below
            const int32_t r = S.rows[S.rows_off[s] + q];
            if (q < w && r != S.sn_first[s] + q) return fail("own rows", s, q);
            if (q > 0 && r <= S.rows[S.rows_off[s] + q - 1]) return fail("row order", s, q);
            if (r < 0 || r >= n) return fail("row range", s, r);
        }
        const int32_t ps = S.sparent[s];
        const int64_t hu = h - w;
        if (hu > 0 && ps < 0) return fail("rows below a root", s);
        for (int64_t i = 0; i < hu; ++i) {
            const int32_t r = S.rows[S.rows_off[s] + w + i];
            const int32_t rel = S.rel[S.u_off[s] + i];
            const int64_t hp = S.rows_off[ps + 1] - S.rows_off[ps];
            if (rel < 0 || rel >= hp || S.rows[S.rows_off[ps] + rel] != r) return fail("rel", s, i);
        }
    }
    // every lower entry of P (A^T A) P^T has a slot in its supernode's panel
    std::vector<std::set<int32_t>> cols(n);
    for (int64_t i = 0; i < p.m; ++i)
        for (int64_t a = p.rp[i]; a < p.rp[i + 1]; ++a)
            for (int64_t b = p.rp[i]; b < p.rp[i + 1]; ++b) {
                const int32_t u = S.iperm[p.ci[a]], v = S.iperm[p.ci[b]];
                if (u >= v) cols[v].insert(u);
            }
    for (int64_t j = 0; j < n; ++j) {
        cols[j].insert((int32_t)j);
        const int64_t cnt = S.gptr[j + 1] - S.gptr[j];
        if (cnt != (int64_t)cols[j].size()) return fail("pattern count", j, cnt);
        const int32_t s = S.col_sn[j];
        const int64_t h = S.rows_off[s + 1] - S.rows_off[s], ld = (h + 3) / 4 * 4;
        const int w = S.sn_first[s + 1] - S.sn_first[s];
        for (int64_t q = S.gptr[j]; q < S.gptr[j + 1]; ++q) {
            const int64_t off = S.gpos[q] - S.L_off[s];
            if (off < 0 || off >= ld * w) return fail("gpos", j, q);
            if (!cols[j].count(S.grow[q])) return fail("grow", j, S.grow[q]);
        }
    }
    return 0;
}

static int cache_round_trip() {
    char path[] = "/tmp/tsnnls_cache_XXXXXX";
    const int fd = mkstemp(path);
    if (fd < 0) return fail("mkstemp");
    close(fd);
    unlink(path);  // start from no file
    const int32_t a[5] = {8, 16, 32, 32, 48}, b[5] = {16, 16, 16, 16, 16};
    int32_t got[5];
    int bad = 0;
    if (tsnnls_tune_cache_get(path, "k1", got) != TSNNLS_ENOTFOUND) bad |= fail("absent file");
    if (tsnnls_tune_cache_put(path, "k1", a) != TSNNLS_OK) bad |= fail("put k1");
    if (tsnnls_tune_cache_put(path, "k \"2\" \\", b) != TSNNLS_OK) bad |= fail("put k2");
    if (tsnnls_tune_cache_get(path, "k1", got) != TSNNLS_OK || got[4] != 48) bad |= fail("get k1");
    if (tsnnls_tune_cache_get(path, "k \"2\" \\", got) != TSNNLS_OK || got[0] != 16) bad |= fail("get k2");
    unlink(path);
    return bad;
}

int main() {
    int bad = 0;
    const Pattern pats[] = {grid(9), random_rows(300, 150, 3, -1), random_rows(80, 40, 2, 17),
                            random_rows(3, 1, 1, -1), random_rows(90, 60, 50, -1), grid(1)};
    for (const Pattern &p : pats)
        for (int width : {32, 64}) bad |= check(p, width);
    bad |= cache_round_trip();
    if (bad) fprintf(stderr, "host sanitizer run: failures\n");
    return bad;
}
