// JSON cache of the batched path's autotuned panel widths
// (tsnnls_tune_cache_get / tsnnls_tune_cache_put, and the lookup behind
// tsnnls_batch_autotune_cached).
//
// The file holds one object:
//
//   {
//     "format": "tsnnls-batch-panel-widths/1",
//     "entries": {
//       "<key>": [w0, w1, w2, w3, w4],
//       ...
//     }
//   }
//
// where a key names the device, the precision, the timing batch size and the
// build of the library, and the five widths are those of the size buckets
// n <= 64, 128, 256, 512, 1024.  The reader accepts any JSON whitespace and
// string escapes of the form \" \\ \/ in keys; it refuses anything else, so a
// file that is not one of ours is reported rather than overwritten.  A write
// replaces the file through a rename, so a reader never sees half a file.
#include <stdint.h>
#include <stdio.h>
#include <string.h>
#include <unistd.h>

#include <map>
#include <string>
#include <vector>

#include "tsnnls.h"

namespace {

constexpr const char *kFormat = "tsnnls-batch-panel-widths/1";
constexpr int kBuckets = 5;

struct Parser {
    const std::string &s;
    size_t i = 0;
    explicit Parser(const std::string &t) : s(t) {}
    void ws() {
        while (i < s.size() && (s[i] == ' ' || s[i] == '\t' || s[i] == '\n' || s[i] == '\r')) ++i;
    }
    bool eat(char c) {
        ws();
        if (i < s.size() && s[i] == c) {
            ++i;
            return true;
        }
        return false;
    }
    bool str(std::string *out) {
        if (!eat('"')) return false;
        out->clear();
        while (i < s.size() && s[i] != '"') {
            char c = s[i++];
            if (c == '\\') {
                if (i >= s.size()) return false;
                c = s[i++];
                if (c != '"' && c != '\\' && c != '/') return false;
            }
            out->push_back(c);
        }
        return eat('"');
    }
    bool integer(long *v) {
        ws();
        size_t j = i;
        if (j < s.size() && s[j] == '-') ++j;
        const size_t d0 = j;
        while (j < s.size() && s[j] >= '0' && s[j] <= '9') ++j;
        if (j == d0 || j - d0 > 9) return false;
        *v = strtol(s.c_str() + i, nullptr, 10);
        i = j;
        return true;
    }
};

using Table = std::map<std::string, std::vector<int>>;

// TSNNLS_OK with the entries (an absent file is an empty table), or
// TSNNLS_EINVAL for a file that does not parse.
int read_table(const char *path, Table *t) {
    t->clear();
    FILE *f = fopen(path, "rb");
    if (!f) return TSNNLS_OK;
    std::string text;
    char buf[4096];
    size_t r;
    while ((r = fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, r);
    fclose(f);
    Parser p(text);
    if (!p.eat('{')) return TSNNLS_EINVAL;
    bool first = true, have_format = false;
    while (!p.eat('}')) {
        if (!first && !p.eat(',')) return TSNNLS_EINVAL;
        first = false;
        std::string name;
        if (!p.str(&name) || !p.eat(':')) return TSNNLS_EINVAL;
        if (name == "format") {
            std::string v;
            if (!p.str(&v) || v != kFormat) return TSNNLS_EINVAL;
            have_format = true;
        } else if (name == "entries") {
            if (!p.eat('{')) return TSNNLS_EINVAL;
            bool efirst = true;
            while (!p.eat('}')) {
                if (!efirst && !p.eat(',')) return TSNNLS_EINVAL;
                efirst = false;
                std::string key;
                if (!p.str(&key) || !p.eat(':') || !p.eat('[')) return TSNNLS_EINVAL;
                std::vector<int> nb;
                bool vfirst = true;
                while (!p.eat(']')) {
                    if (!vfirst && !p.eat(',')) return TSNNLS_EINVAL;
                    vfirst = false;
                    long v;
                    if (!p.integer(&v)) return TSNNLS_EINVAL;
                    nb.push_back((int)v);
                }
                if ((int)nb.size() != kBuckets) return TSNNLS_EINVAL;
                (*t)[key] = nb;
            }
        } else {
            return TSNNLS_EINVAL;
        }
    }
    p.ws();
    if (p.i != text.size() || !have_format) return TSNNLS_EINVAL;
    return TSNNLS_OK;
}

std::string quote(const std::string &k) {
    std::string o = "\"";
    for (char c : k) {
        if (c == '"' || c == '\\') o.push_back('\\');
        o.push_back(c);
    }
    return o + "\"";
}

int write_table(const char *path, const Table &t) {
    std::string tmp = std::string(path) + ".tmp" + std::to_string((long)getpid());
    FILE *f = fopen(tmp.c_str(), "wb");
    if (!f) return TSNNLS_EINVAL;
    fprintf(f, "{\n  \"format\": \"%s\",\n  \"entries\": {", kFormat);
    bool first = true;
    for (const auto &kv : t) {
        fprintf(f, "%s\n    %s: [", first ? "" : ",", quote(kv.first).c_str());
        for (int b = 0; b < kBuckets; ++b) fprintf(f, "%s%d", b ? ", " : "", kv.second[b]);
        fprintf(f, "]");
        first = false;
    }
    fprintf(f, "%s}\n}\n", first ? "" : "\n  ");
    const bool ok = fflush(f) == 0;
    fclose(f);
    if (!ok || rename(tmp.c_str(), path) != 0) {
        remove(tmp.c_str());
        return TSNNLS_EINVAL;
    }
    return TSNNLS_OK;
}

bool valid_key(const char *key) {
    if (!key || !*key) return false;
    for (const char *c = key; *c; ++c)
        if ((unsigned char)*c < 0x20) return false;
    return true;
}

}  // namespace

extern "C" {

int tsnnls_tune_cache_get(const char *path, const char *key, int32_t *nb_out) {
    if (!path || !valid_key(key) || !nb_out) return TSNNLS_EINVAL;
    Table t;
    const int st = read_table(path, &t);
    if (st != TSNNLS_OK) return st;
    auto it = t.find(key);
    if (it == t.end()) return TSNNLS_ENOTFOUND;
    for (int b = 0; b < kBuckets; ++b) nb_out[b] = it->second[b];
    return TSNNLS_OK;
}

int tsnnls_tune_cache_put(const char *path, const char *key, const int32_t *nb) {
    if (!path || !valid_key(key) || !nb) return TSNNLS_EINVAL;
    Table t;
    const int st = read_table(path, &t);
    if (st != TSNNLS_OK) return st;
    t[key] = std::vector<int>(nb, nb + kBuckets);
    return write_table(path, t);
}

}  // extern "C"
