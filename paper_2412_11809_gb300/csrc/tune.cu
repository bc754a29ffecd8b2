// Autotuner of the batched step (tpc_tune_batch) and its cache file.
//
// The paper sizes its GPU work by hand: a chunk of at least 10,000 hits per
// thread, each thread with its own pixel matrix (Section 4.1, Algorithm 3
// step 4).  Here the work per CTA is fixed by the tile (4096 hits in shared
// memory) and what is left to choose is how the launches fill the GPU: CTAs
// per SM for each group of persistent kernels, the positions per pass of the
// feature kernel, which link kernel a sensor takes (the shared-memory table
// or the general one) and the order of the detectors in a batch.  Results
// never depend on these choices, only the time does.
//
// The tuner times the caller's own batch (its pending hits, left pending):
// the default choices first, then coordinate descent over the knobs, two
// passes, keeping a change only if the median of three timed runs improves
// by more than 1 %.  The choice is kept per (GPU, sensor geometries, size
// bucket of each geometry's hits) in a text cache file, one line per entry:
//   key <TAB> ctas_sort ctas_link ctas_acc ctas_out acc_span general_link order <TAB> ms
// where the last line with a key wins.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "ctx_internal.h"

using namespace tpc;

namespace {

Tuning from_public(const tpc_tuning &p) {
    Tuning t;
    t.cap[G_SORT] = p.ctas_sort;
    t.cap[G_LINK] = p.ctas_link;
    t.cap[G_ACC] = p.ctas_acc;
    t.cap[G_OUT] = p.ctas_out;
    t.acc_span = p.acc_span ? p.acc_span : 1024;
    t.general_link = p.general_link;
    t.order = p.order;
    return t;
}

tpc_tuning to_public(const Tuning &t) {
    tpc_tuning p{};
    p.ctas_sort = t.cap[G_SORT];
    p.ctas_link = t.cap[G_LINK];
    p.ctas_acc = t.cap[G_ACC];
    p.ctas_out = t.cap[G_OUT];
    p.acc_span = t.acc_span;
    p.general_link = t.general_link;
    p.order = t.order;
    return p;
}

bool valid(const tpc_tuning &p) {
    return p.ctas_sort <= 64 && p.ctas_link <= 64 && p.ctas_acc <= 64 && p.ctas_out <= 64 &&
           (p.acc_span == 0 || p.acc_span == 512 || p.acc_span == 1024 || p.acc_span == 2048) &&
           p.general_link <= 3 && p.order <= 1;
}

// The cache key of a batch: GPU name and SM count, then per sensor geometry
// the bucket floor(log2(hits)) of its pending hits, geometries sorted.
std::string batch_key(tpc_ctx **ctxs, int n) {
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, ctx_device(ctxs[0]));
    std::map<std::pair<uint32_t, uint32_t>, uint64_t> hits;
    for (int i = 0; i < n; ++i) {
        uint32_t w = 0, h = 0;
        ctx_sensor(ctxs[i], &w, &h);
        hits[{w, h}] += ctx_pending(ctxs[i]);
    }
    std::string key = std::string(prop.name) + "|" + std::to_string(prop.multiProcessorCount);
    for (const auto &kv : hits) {
        const uint64_t m = std::max<uint64_t>(kv.second, 1);
        key += "|" + std::to_string(kv.first.first) + "x" + std::to_string(kv.first.second) + ":b" +
               std::to_string(63 - __builtin_clzll(m));
    }
    return key + "|n" + std::to_string(n);
}

// Median device time (ms) of `reps` batched steps with launch choices t,
// after one untimed step (which captures the step's graph).
int time_batch(tpc_ctx **ctxs, int n, const Tuning &t, int reps, double *ms) {
    Tuning &lead = ctx_tuning(ctxs[0]);
    const Tuning saved = lead;
    lead = t;
    cudaStream_t st = ctx_stream(ctxs[0]);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = TPC_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = TPC_ERR_CUDA;
    std::vector<float> times;
    if (rc == TPC_OK) rc = batch_step(ctxs, n, false);
    for (int r = 0; rc == TPC_OK && r < reps; ++r) {
        float x = 0;
        if (cudaEventRecord(e0, st) != cudaSuccess) { rc = TPC_ERR_CUDA; break; }
        rc = batch_step(ctxs, n, false);
        if (rc) break;
        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&x, e0, e1) != cudaSuccess) {
            rc = TPC_ERR_CUDA;
            break;
        }
        times.push_back(x);
    }
    if (rc == TPC_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = TPC_ERR_CUDA;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    lead = saved;
    if (rc == TPC_OK) {
        std::sort(times.begin(), times.end());
        *ms = times[times.size() / 2];
    }
    return rc;
}

bool parse_line(const char *line, const char *key, tpc_tuning *t, double *ms) {
    const char *tab = std::strchr(line, '\t');
    if (!tab || (size_t)(tab - line) != std::strlen(key) || std::strncmp(line, key, tab - line) != 0) return false;
    unsigned v[7];
    double m = 0;
    if (std::sscanf(tab + 1, "%u %u %u %u %u %u %u\t%lf", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5], &v[6], &m) != 8)
        return false;
    for (unsigned x : v) if (x > 65535) return false;
    tpc_tuning p{};
    p.ctas_sort = (uint8_t)std::min(v[0], 255u);
    p.ctas_link = (uint8_t)std::min(v[1], 255u);
    p.ctas_acc = (uint8_t)std::min(v[2], 255u);
    p.ctas_out = (uint8_t)std::min(v[3], 255u);
    p.acc_span = (uint16_t)v[4];
    p.general_link = (uint8_t)std::min(v[5], 255u);
    p.order = (uint8_t)std::min(v[6], 255u);
    if (!valid(p) || v[0] > 64 || v[1] > 64 || v[2] > 64 || v[3] > 64 || v[5] > 3 || v[6] > 1) return false;
    *t = p;
    if (ms) *ms = m;
    return true;
}

}  // namespace

extern "C" {

int tpc_set_tuning(tpc_ctx *c, const tpc_tuning *t) {
    if (!c) return TPC_ERR_ARG;
    tpc_tuning p{};
    if (t) {
        if (!valid(*t)) return TPC_ERR_ARG;
        p = *t;
    }
    std::lock_guard<std::mutex> lk(ctx_mutex(c));
    ctx_tuning(c) = from_public(p);
    return TPC_OK;
}

int tpc_get_tuning(tpc_ctx *c, tpc_tuning *t) {
    if (!c || !t) return TPC_ERR_ARG;
    std::lock_guard<std::mutex> lk(ctx_mutex(c));
    *t = to_public(ctx_tuning(c));
    return TPC_OK;
}

int tpc_tune_cache_lookup(const char *path, const char *key, tpc_tuning *out, double *ms) {
    if (!path || !key || !out || std::strchr(key, '\t') || std::strchr(key, '\n')) return TPC_ERR_ARG;
    FILE *f = std::fopen(path, "r");
    if (!f) return TPC_ERR_STATE;
    char line[1024];
    bool found = false;
    while (std::fgets(line, sizeof line, f)) {
        tpc_tuning t;
        double m = 0;
        if (parse_line(line, key, &t, &m)) {   // the last matching line wins
            *out = t;
            if (ms) *ms = m;
            found = true;
        }
    }
    std::fclose(f);
    return found ? TPC_OK : TPC_ERR_STATE;
}

int tpc_tune_cache_store(const char *path, const char *key, const tpc_tuning *t, double ms) {
    if (!path || !key || !t || !valid(*t) || !*key || std::strlen(key) > 512 || std::strchr(key, '\t') ||
        std::strchr(key, '\n'))
        return TPC_ERR_ARG;
    FILE *f = std::fopen(path, "a");
    if (!f) return TPC_ERR_ARG;
    const int ok = std::fprintf(f, "%s\t%u %u %u %u %u %u %u\t%.6f\n", key, t->ctas_sort, t->ctas_link, t->ctas_acc,
                                t->ctas_out, t->acc_span ? t->acc_span : 1024, t->general_link, t->order, ms);
    return std::fclose(f) == 0 && ok > 0 ? TPC_OK : TPC_ERR_ARG;
}

int tpc_tune_batch(tpc_ctx **ctxs, int n, const char *cache_path, int flags, tpc_tune_report *rep) {
    int rc = check_batch(ctxs, n);
    if (rc) return rc;
    if (!rep) return TPC_ERR_ARG;
    std::memset(rep, 0, sizeof(*rep));
    for (int i = 0; i < n; ++i)
        if (!ctx_pending(ctxs[i])) return TPC_ERR_STATE;   // the batch to time is the pending one
    std::vector<std::unique_lock<std::mutex>> locks;
    for (int i = 0; i < n; ++i) locks.emplace_back(ctx_mutex(ctxs[i]));
    const std::string key = batch_key(ctxs, n);
    std::snprintf(rep->key, sizeof rep->key, "%s", key.c_str());
    if (cache_path && !(flags & TPC_TUNE_FORCE)) {
        tpc_tuning t;
        double ms = 0;
        locks.clear();   // the lookup touches no context
        if (tpc_tune_cache_lookup(cache_path, key.c_str(), &t, &ms) == TPC_OK) {
            std::lock_guard<std::mutex> lk(ctx_mutex(ctxs[0]));
            ctx_tuning(ctxs[0]) = from_public(t);
            rep->chosen = t;
            rep->from_cache = 1;
            rep->tuned_ms = ms;
            return TPC_OK;
        }
        for (int i = 0; i < n; ++i) locks.emplace_back(ctx_mutex(ctxs[i]));
    }
    const int REPS = 3;
    Tuning best{};   // the defaults
    double best_ms = 0;
    rc = time_batch(ctxs, n, best, REPS, &best_ms);
    if (rc) return rc;
    rep->untuned_ms = best_ms;
    rep->trials = 1;
    // knob k of a Tuning, read and written through one accessor
    auto knob = [](Tuning &t, int k) -> int {
        switch (k) {
        case 0: return t.cap[G_SORT];
        case 1: return t.cap[G_LINK];
        case 2: return t.cap[G_ACC];
        case 3: return t.cap[G_OUT];
        case 4: return t.acc_span;
        case 5: return t.general_link;
        default: return t.order;
        }
    };
    auto set = [](Tuning &t, int k, int v) {
        switch (k) {
        case 0: t.cap[G_SORT] = (uint8_t)v; break;
        case 1: t.cap[G_LINK] = (uint8_t)v; break;
        case 2: t.cap[G_ACC] = (uint8_t)v; break;
        case 3: t.cap[G_OUT] = (uint8_t)v; break;
        case 4: t.acc_span = (uint16_t)v; break;
        case 5: t.general_link = (uint8_t)v; break;
        default: t.order = (uint8_t)v; break;
        }
    };
    const std::vector<std::vector<int>> cands = {
        {0, 1, 2}, {0, 1, 2, 4}, {0, 1, 2, 3}, {0, 2, 4, 8}, {1024, 512, 2048}, {0, 1, 2, 3}, {0, 1}};
    for (int pass = 0; pass < 2; ++pass) {
        bool moved = false;
        for (int k = 0; k < (int)cands.size(); ++k) {
            for (int v : cands[k]) {
                if (v == knob(best, k)) continue;
                Tuning t = best;
                set(t, k, v);
                double ms = 0;
                rc = time_batch(ctxs, n, t, REPS, &ms);
                if (rc) return rc;
                ++rep->trials;
                if (ms < best_ms * 0.99) {
                    best = t;
                    best_ms = ms;
                    moved = true;
                }
            }
        }
        if (!moved) break;
    }
    ctx_tuning(ctxs[0]) = best;
    rep->chosen = to_public(best);
    rep->tuned_ms = best_ms;
    locks.clear();
    if (cache_path) {
        rc = tpc_tune_cache_store(cache_path, key.c_str(), &rep->chosen, best_ms);
        if (rc) return rc;
    }
    return TPC_OK;
}

}  // extern "C"
