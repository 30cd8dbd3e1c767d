// Autotuner: picks database splits, column parts per row and candidate list
// widths by timing them on the caller's data, and remembers the choice in a
// process-wide table that the planners consult when options are automatic.
//
// Every candidate configuration is exact by construction (each column part's
// list can hold the whole top-k; the FP32 re-rank fixes the final order), so
// the tuner only compares speed.  Keys bucket n by floor(log2 n): a choice
// tuned on one size is reused for sizes within a factor of two.
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace rsc {

namespace {

using Key = std::tuple<int, int, int, int, int, int, int>;   // kind, precision, metric, d, k, kx, log2 n

std::mutex g_tune_mu;
std::map<Key, TunedChoice> g_table;

int log2_bucket(int64_t n) {
    int b = 0;
    while ((int64_t(1) << (b + 1)) <= n) ++b;
    return b;
}

Key make_key(int kind, int precision, int metric, int d, int k, int kx, int64_t n) {
    return Key(kind, precision, metric, d, k, kx, log2_bucket(n));
}

// Times `run` (enqueued on st) `trials` times after one warm-up; min in ms.
template <class F>
rsc_status time_config(F run, cudaStream_t st, int trials, float *best) {
    cudaEvent_t a = nullptr, b = nullptr;
    RSC_CUDA_TRY(cudaEventCreate(&a));
    RSC_CUDA_TRY(cudaEventCreate(&b));
    rsc_status s = run();
    float ms_min = INFINITY;
    for (int t = 0; t < trials && s == RSC_OK; ++t) {
        cudaEventRecord(a, st);
        s = run();
        cudaEventRecord(b, st);
        if (cudaEventSynchronize(b) != cudaSuccess) s = fail(RSC_ERR_CUDA, "event synchronize failed");
        float ms = 0.f;
        if (s == RSC_OK) {
            cudaEventElapsedTime(&ms, a, b);
            ms_min = std::min(ms_min, ms);
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *best = ms_min;
    return s;
}

}  // namespace

bool tuned_lookup(int kind, int precision, int metric, int d, int k, int kx, int64_t n, TunedChoice *out) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_table.find(make_key(kind, precision, metric, d, k, kx, n));
    if (it == g_table.end()) return false;
    *out = it->second;
    return true;
}

void tuned_store(int kind, int precision, int metric, int d, int k, int kx, int64_t n, const TunedChoice &c) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_table[make_key(kind, precision, metric, d, k, kx, n)] = c;
}

}  // namespace rsc

using namespace rsc;

namespace {

// First round of rsc_knn configurations: database splits x column parts
// (all explicit, so the planner does not consult the table while tuning).
std::vector<rsc_knn_opts> knn_candidates(const rsc_knn_opts &base, int64_t n, int32_t d, int32_t k, int32_t metric) {
    std::vector<rsc_knn_opts> out;
    std::vector<int> parts_opts = {0};
    if (base.precision != RSC_FP32) parts_opts = {4, 2};
    for (int parts : parts_opts) {
        for (int sp : {1, 2, 4, 8}) {
            rsc_knn_opts o = base;
            o.db_splits = sp;
            o.candidates = 0;
            o.tc_parts = parts;
            o.stages = 0;
            size_t bytes = 0;
            if (rsc_knn_workspace_size(n, d, k, metric, &o, &bytes) == RSC_OK) out.push_back(o);
        }
    }
    return out;
}

// Later rounds around the best so far: the pipeline stages (tensor-core
// paths), then candidate lists twice the default length (never shorter, so
// the recall of the chosen configuration is at least the default's).
std::vector<rsc_knn_opts> knn_refinements(const rsc_knn_opts &best, int round, int64_t n, int32_t d, int32_t k,
                                          int32_t metric) {
    std::vector<rsc_knn_opts> out;
    if (round == 0 && best.precision != RSC_FP32) {
        for (int stg : {3, 4, 5}) {
            rsc_knn_opts o = best;
            o.stages = stg;
            size_t bytes = 0;
            if (rsc_knn_workspace_size(n, d, k, metric, &o, &bytes) == RSC_OK) out.push_back(o);
        }
    } else if (round == 1) {
        rsc_knn_opts def = best;
        def.candidates = 0;
        const int base_c = (best.precision == RSC_FP32) ? k + 8
                           : (best.precision == RSC_FP8) ? 8 * k
                                                         : (metric == RSC_COSINE ? 4 * k : 2 * k);
        rsc_knn_opts o = best;
        o.candidates = 2 * base_c;
        size_t bytes = 0;
        if (o.candidates <= 128 && rsc_knn_workspace_size(n, d, k, metric, &o, &bytes) == RSC_OK) out.push_back(o);
    }
    return out;
}

}  // namespace

extern "C" {

rsc_status rsc_autotune_workspace_size(int64_t n, int32_t d, int32_t k, int32_t metric, int32_t precision,
                                       size_t *bytes) {
    if (!bytes) return fail(RSC_ERR_INVALID_ARG, "bytes is NULL");
    rsc_knn_opts base = {};
    base.precision = precision;
    size_t most = 0;
    for (auto &o : knn_candidates(base, n, d, k, metric)) {
        size_t b = 0;
        if (rsc_knn_workspace_size(n, d, k, metric, &o, &b) == RSC_OK) most = std::max(most, b);
    }
    if (most == 0) return rsc_knn_workspace_size(n, d, k, metric, &base, bytes);
    *bytes = most;
    return RSC_OK;
}

rsc_status rsc_autotune_knn(const float *X, int64_t n, int32_t d, int32_t k, int32_t metric,
                            const rsc_knn_opts *opts, int32_t trials, int32_t *idx, float *dist,
                            rsc_knn_opts *best, float *best_ms, void *workspace, size_t workspace_bytes) {
    RSC_TRACE("rsc_autotune_knn");
    if (!opts || !best || !X || !idx || !dist) return fail(RSC_ERR_INVALID_ARG, "NULL argument");
    if (trials < 1) return fail(RSC_ERR_INVALID_ARG, "trials must be >= 1");
    cudaStream_t st = static_cast<cudaStream_t>(opts->stream);
    auto cands = knn_candidates(*opts, n, d, k, metric);
    if (cands.empty()) return fail(RSC_ERR_UNSUPPORTED, "no configuration supports this problem");
    float best_t = INFINITY;
    rsc_knn_opts chosen = cands[0];
    auto try_all = [&](const std::vector<rsc_knn_opts> &set) -> rsc_status {
        for (auto &o : set) {
            float t = INFINITY;
            rsc_status s = time_config(
                [&]() { return rsc_knn(X, n, d, k, metric, idx, dist, &o, workspace, workspace_bytes); }, st,
                trials, &t);
            if (s != RSC_OK) return s;
            if (t < best_t) {
                best_t = t;
                chosen = o;
            }
        }
        return RSC_OK;
    };
    rsc_status s0 = try_all(cands);
    for (int round = 0; s0 == RSC_OK && round < 2; ++round) s0 = try_all(knn_refinements(chosen, round, n, d, k, metric));
    if (s0 != RSC_OK) return s0;
    // leave the chosen configuration's result in the outputs
    rsc_status s = rsc_knn(X, n, d, k, metric, idx, dist, &chosen, workspace, workspace_bytes);
    if (s != RSC_OK) return s;
    RSC_CUDA_TRY(cudaStreamSynchronize(st));
    tuned_store(0, opts->precision, metric, d, k, 0, n,
                TunedChoice{chosen.db_splits, chosen.candidates, chosen.tc_parts, chosen.stages});
    *best = chosen;
    if (best_ms) *best_ms = best_t;
    return RSC_OK;
}

rsc_status rsc_autotune_knn_batched(const float *X, int64_t n, int32_t d, const int64_t *sample_offsets,
                                    int32_t n_samples, int32_t k_within, int32_t k_cross, int32_t metric,
                                    const rsc_knn_opts *opts, int32_t trials, int32_t *idx_within,
                                    float *dist_within, int32_t *idx_cross, float *dist_cross, rsc_knn_opts *best,
                                    float *best_ms, void *workspace, size_t workspace_bytes) {
    RSC_TRACE("rsc_autotune_knn_batched");
    if (!opts || !best) return fail(RSC_ERR_INVALID_ARG, "NULL argument");
    if (trials < 1) return fail(RSC_ERR_INVALID_ARG, "trials must be >= 1");
    cudaStream_t st = static_cast<cudaStream_t>(opts->stream);
    float best_t = INFINITY;
    rsc_knn_opts chosen = *opts;
    std::vector<rsc_knn_opts> cands;
    for (int parts : {4, 2})
        for (int stg : {0, 3, 4}) {
            rsc_knn_opts o = *opts;
            o.tc_parts = parts;
            o.stages = stg;
            cands.push_back(o);
        }
    for (auto &o : cands) {
        float t = INFINITY;
        rsc_status s = time_config(
            [&]() {
                return rsc_knn_batched(X, n, d, sample_offsets, n_samples, k_within, k_cross, metric, idx_within,
                                       dist_within, idx_cross, dist_cross, &o, workspace, workspace_bytes);
            },
            st, trials, &t);
        if (s != RSC_OK) return s;
        if (t < best_t) {
            best_t = t;
            chosen = o;
        }
    }
    rsc_status s = rsc_knn_batched(X, n, d, sample_offsets, n_samples, k_within, k_cross, metric, idx_within,
                                   dist_within, idx_cross, dist_cross, &chosen, workspace, workspace_bytes);
    if (s != RSC_OK) return s;
    RSC_CUDA_TRY(cudaStreamSynchronize(st));
    tuned_store(1, opts->precision, metric, d, k_within, k_cross, n, TunedChoice{0, 0, chosen.tc_parts, chosen.stages});
    *best = chosen;
    if (best_ms) *best_ms = best_t;
    return RSC_OK;
}

rsc_status rsc_autotune_save(const char *path) {
    if (!path) return fail(RSC_ERR_INVALID_ARG, "path is NULL");
    FILE *f = fopen(path, "w");
    if (!f) return fail(RSC_ERR_INVALID_ARG, "cannot open %s for writing", path);
    std::lock_guard<std::mutex> lock(g_tune_mu);
    fprintf(f, "# rsc autotune v2: kind precision metric d k k_cross log2n db_splits candidates tc_parts stages\n");
    for (auto &kv : g_table) {
        const Key &key = kv.first;
        fprintf(f, "%d %d %d %d %d %d %d %d %d %d %d\n", std::get<0>(key), std::get<1>(key), std::get<2>(key),
                std::get<3>(key), std::get<4>(key), std::get<5>(key), std::get<6>(key), kv.second.db_splits,
                kv.second.candidates, kv.second.tc_parts, kv.second.stages);
    }
    const bool ok = fclose(f) == 0;
    return ok ? RSC_OK : fail(RSC_ERR_INVALID_ARG, "write to %s failed", path);
}

rsc_status rsc_autotune_load(const char *path) {
    if (!path) return fail(RSC_ERR_INVALID_ARG, "path is NULL");
    FILE *f = fopen(path, "r");
    if (!f) return fail(RSC_ERR_INVALID_ARG, "cannot open %s", path);
    char line[256];
    int lineno = 0, bad = 0;
    std::vector<std::pair<Key, TunedChoice>> rows;
    while (fgets(line, sizeof(line), f)) {
        ++lineno;
        if (line[0] == '#' || line[0] == '\n') continue;
        int v[11] = {0};
        const int got = sscanf(line, "%d %d %d %d %d %d %d %d %d %d %d", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5],
                               &v[6], &v[7], &v[8], &v[9], &v[10]);
        if ((got != 10 && got != 11) || v[7] < 0 || v[8] < 0 || (v[9] != 0 && v[9] != 2 && v[9] != 4) ||
            (v[10] != 0 && (v[10] < 2 || v[10] > 6))) {
            bad = lineno;
            break;
        }
        rows.push_back({Key(v[0], v[1], v[2], v[3], v[4], v[5], v[6]), TunedChoice{v[7], v[8], v[9], v[10]}});
    }
    fclose(f);
    if (bad) return fail(RSC_ERR_INVALID_ARG, "%s: malformed line %d", path, bad);
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (auto &r : rows) g_table[r.first] = r.second;
    return RSC_OK;
}

rsc_status rsc_autotune_clear(void) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_table.clear();
    return RSC_OK;
}

}  // extern "C"
