// tune.cpp -- launch configuration: built-in defaults, a tuned table keyed by
// problem size class, a process-wide override, and JSON persistence.
//
// Size class = (bits of len, bits of the packed key, bits of len / 2^(column
// bits)).  The last term is the density -- triplets per column, which sets
// the bucket width and the run lengths -- as far as it is known before an
// assembly (nnz is not).  The autotuner itself (timing candidates with CUDA
// events) is fsparse_autotune in api.cu.
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "internal.hpp"

namespace fsp {

static std::mutex g_mu;
static bool g_has_override = false;
static fsparse_config g_override{};
static std::map<std::string, fsparse_config> g_table;

static std::string size_class(int64_t len, const KeyLayout &key) {
    char buf[64];
    const uint64_t l = (uint64_t)(len > 0 ? len : 0);
    std::snprintf(buf, sizeof buf, "L%d_K%d_D%d", bits_for(l), key.total(), bits_for(l >> key.cb));
    return buf;
}

bool config_valid(const fsparse_config &c) {
    const bool items = c.sweep_items == 8 || c.sweep_items == 12 || c.sweep_items == 16;
    const bool threads = c.sweep_threads == 256 || c.sweep_threads == 512;
    const bool tile = c.numeric_tile == 1024 || c.numeric_tile == 2048 || c.numeric_tile == 4096;
    // digits of 9 and 10 bits only in 256-thread passes (their per-warp
    // counters would not fit shared memory beside a 512-thread tile)
    const bool radix = c.radix_bits >= 6 && (c.radix_bits <= 8 || (c.radix_bits <= 10 && c.sweep_threads == 256));
    return c.strategy >= 0 && c.strategy <= 3 && radix && items && threads && c.bucket_target >= 1024 &&
           c.bucket_target <= 16384 && tile;
}

fsparse_config default_config(int64_t len, const KeyLayout &key) {
    fsparse_config c{};
    c.strategy = bucket_supported(len, 1 << key.cb, key, fsparse_config{FSPARSE_SORT_BUCKET, 8, 16, 256, 8192, 4096})
                     ? FSPARSE_SORT_BUCKET
                     : FSPARSE_SORT_ONESWEEP;
    c.radix_bits = 8;
    c.sweep_items = 16;
    c.sweep_threads = 256;
    c.bucket_target = 8192;
    // 64-thread blocks of 16-position chunks measured fastest at every size tried
    // (0.361 vs 0.382 ms on 93M mesh triplets, equal on uniform random ones).
    c.numeric_tile = 1024;
    return c;
}

fsparse_config resolve_config(int64_t len, const KeyLayout &key) {
    fsparse_config c = default_config(len, key);
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_table.find(size_class(len, key));
    if (it != g_table.end()) c = it->second;
    if (g_has_override) {
        const fsparse_config &o = g_override;
        if (o.strategy > 0) c.strategy = o.strategy;
        if (o.radix_bits > 0) c.radix_bits = o.radix_bits;
        if (o.sweep_items > 0) c.sweep_items = o.sweep_items;
        if (o.sweep_threads > 0) c.sweep_threads = o.sweep_threads;
        if (o.bucket_target > 0) c.bucket_target = o.bucket_target;
        if (o.numeric_tile > 0) c.numeric_tile = o.numeric_tile;
    }
    if (c.strategy == FSPARSE_SORT_AUTO) c.strategy = default_config(len, key).strategy;
    return c;
}

void tune_store(int64_t len, const KeyLayout &key, const fsparse_config &cfg) {
    std::lock_guard<std::mutex> lock(g_mu);
    g_table[size_class(len, key)] = cfg;
}

// Candidates: every onesweep shape, the bucket path at several bucket sizes,
// each with the numeric tile sizes.
// Sort candidates (the numeric tile is tuned separately, on the winner's plan).
std::vector<fsparse_config> tune_candidates(int64_t len, const KeyLayout &key) {
    std::vector<fsparse_config> out;
    const int tile = default_config(len, key).numeric_tile;
    for (int r = 6; r <= 10; ++r)
        for (int th : {256, 512})
            for (int it : {8, 12, 16}) {
                const fsparse_config c{FSPARSE_SORT_ONESWEEP, r, it, th, 8192, tile};
                if (config_valid(c)) out.push_back(c);
            }
    for (int strat : {FSPARSE_SORT_BUCKET, FSPARSE_SORT_BUCKET_RADIX})
        for (int bt : {2048, 4096, 8192, 12288}) {
            fsparse_config c{strat, 8, 16, 256, bt, tile};
            if (bucket_supported(len, 1 << key.cb, key, c)) out.push_back(c);
        }
    return out;
}

}  // namespace fsp

using namespace fsp;

extern "C" {

fsparse_status fsparse_get_config(int64_t len, int32_t m, int32_t n, fsparse_config *out) {
    if (!out || len < 0 || m < 0 || n < 0) return set_error(FSPARSE_ERR_ARG, "bad arguments");
    KeyLayout key;
    key.rb = m > 0 ? bits_for((uint64_t)m - 1) : 0;
    key.cb = n > 0 ? bits_for((uint64_t)n - 1) : 0;
    *out = resolve_config(len, key);
    return FSPARSE_OK;
}

fsparse_status fsparse_set_config(const fsparse_config *cfg) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!cfg) {
        g_has_override = false;
        return FSPARSE_OK;
    }
    fsparse_config probe{1, 8, 16, 256, 8192, 4096};
    if (cfg->strategy > 0) probe.strategy = cfg->strategy;
    if (cfg->radix_bits > 0) probe.radix_bits = cfg->radix_bits;
    if (cfg->sweep_items > 0) probe.sweep_items = cfg->sweep_items;
    if (cfg->sweep_threads > 0) probe.sweep_threads = cfg->sweep_threads;
    if (cfg->bucket_target > 0) probe.bucket_target = cfg->bucket_target;
    if (cfg->numeric_tile > 0) probe.numeric_tile = cfg->numeric_tile;
    if (!config_valid(probe)) return set_error(FSPARSE_ERR_ARG, "invalid configuration");
    g_override = *cfg;
    g_has_override = true;
    return FSPARSE_OK;
}

fsparse_status fsparse_tune_clear(void) {
    std::lock_guard<std::mutex> lock(g_mu);
    g_table.clear();
    return FSPARSE_OK;
}

fsparse_status fsparse_tune_save(const char *path) {
    if (!path) return set_error(FSPARSE_ERR_ARG, "path is NULL");
    std::lock_guard<std::mutex> lock(g_mu);
    FILE *f = std::fopen(path, "w");
    if (!f) return set_error(FSPARSE_ERR_ARG, std::string("cannot write ") + path);
    std::fprintf(f, "{\"version\": 1, \"entries\": [");
    bool first = true;
    for (const auto &kv : g_table) {
        const fsparse_config &c = kv.second;
        std::fprintf(f,
                     "%s\n  {\"class\": \"%s\", \"strategy\": %d, \"radix_bits\": %d, \"sweep_items\": %d, "
                     "\"sweep_threads\": %d, \"bucket_target\": %d, \"numeric_tile\": %d}",
                     first ? "" : ",", kv.first.c_str(), c.strategy, c.radix_bits, c.sweep_items,
                     c.sweep_threads, c.bucket_target, c.numeric_tile);
        first = false;
    }
    std::fprintf(f, "\n]}\n");
    std::fclose(f);
    return FSPARSE_OK;
}

static bool json_int(const char *obj, const char *end, const char *name, int32_t *out) {
    char pat[64];
    std::snprintf(pat, sizeof pat, "\"%s\"", name);
    const char *p = std::strstr(obj, pat);
    if (!p || p >= end) return false;
    p = std::strchr(p + std::strlen(pat), ':');
    if (!p || p >= end) return false;
    return std::sscanf(p + 1, "%d", out) == 1;
}

fsparse_status fsparse_tune_load(const char *path) {
    if (!path) return set_error(FSPARSE_ERR_ARG, "path is NULL");
    FILE *f = std::fopen(path, "r");
    if (!f) return set_error(FSPARSE_ERR_ARG, std::string("cannot read ") + path);
    std::string text;
    char buf[4096];
    size_t got;
    while ((got = std::fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, got);
    std::fclose(f);
    std::map<std::string, fsparse_config> table;
    const char *p = text.c_str();
    while ((p = std::strstr(p, "\"class\"")) != nullptr) {
        const char *end = std::strchr(p, '}');
        const char *q1 = std::strchr(p + 7, '"');
        const char *q2 = q1 ? std::strchr(q1 + 1, '"') : nullptr;
        if (!end || !q1 || !q2 || q2 > end) return set_error(FSPARSE_ERR_ARG, "malformed tuning file");
        std::string cls(q1 + 1, q2);
        fsparse_config c{};
        if (!json_int(p, end, "strategy", &c.strategy) || !json_int(p, end, "radix_bits", &c.radix_bits) ||
            !json_int(p, end, "sweep_items", &c.sweep_items) ||
            !json_int(p, end, "sweep_threads", &c.sweep_threads) ||
            !json_int(p, end, "bucket_target", &c.bucket_target) ||
            !json_int(p, end, "numeric_tile", &c.numeric_tile) || !config_valid(c))
            return set_error(FSPARSE_ERR_ARG, "malformed tuning entry " + cls);
        table[cls] = c;
        p = end;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    for (auto &kv : table) g_table[kv.first] = kv.second;
    return FSPARSE_OK;
}

}  // extern "C"
