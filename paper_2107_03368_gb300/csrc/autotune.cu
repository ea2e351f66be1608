// autotune.cu — launch-shape autotuner for the search kernels.
//
// Knobs (none changes a result, only speed):
//   TREE   dt_search traversal: threads per block (128 or 256) and resident
//          blocks per SM of the persistent grid (how many queries are in
//          flight at once);
//   POPC   popcount brute force: number of database splits (grid depth);
//   TC     tensor-core brute force: number of database splits (work units
//          per persistent CTA), and whether the database is widened inside
//          the kernel or once beforehand (b = 1 / 2);
//   TREE_TC  the batched tree search's scan: the same two knobs;
//   RETRIEVE the engine retrieve_objects uses when asked for engine 0, and
//          engine 1's resident blocks per SM (keyed by the database size
//          and whether the threshold is 0).
// dt_autotune times each candidate on the caller's data with CUDA events
// and keeps the fastest per key (kind, log2 n, log2 nq, k, SM count) in a
// process-wide table; launchers look the key up and fall back to their
// built-in heuristics.  The table can be saved to and loaded from a text
// file (one "kind n_log nq_log k sms a b" line per entry).
#include <cmath>
#include <cstdio>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "dt_internal.cuh"

namespace dtk {
namespace {

using Key = std::tuple<int, int, int, int, int>;
std::mutex g_tune_mu;
std::map<Key, TuneCfg> g_tune;

int log2i(int64_t v)
{
    int r = 0;
    while (v > 1) {
        v >>= 1;
        ++r;
    }
    return r;
}

Key make_key(TuneKind kind, int64_t n, int64_t nq, int k)
{
    return Key((int)kind, log2i(n), log2i(nq), k, sm_count());
}

}  // namespace

bool tune_lookup(TuneKind kind, int64_t n, int64_t nq, int k, TuneCfg *cfg)
{
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune.find(make_key(kind, n, nq, k));
    if (it == g_tune.end()) return false;
    *cfg = it->second;
    return true;
}

void tune_store(TuneKind kind, int64_t n, int64_t nq, int k, const TuneCfg &cfg)
{
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[make_key(kind, n, nq, k)] = cfg;
}

void tune_clear()
{
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune.clear();
}

namespace {

// Time fn() once after one warm-up; milliseconds, or -1 on failure.
template <typename F>
float time_call(F fn, cudaStream_t s)
{
    if (fn() != DT_OK) return -1.f;
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return -1.f;
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return -1.f;
    }
    cudaEventRecord(a, s);
    int rc = fn();
    cudaEventRecord(b, s);
    float ms = -1.f;
    if (rc == DT_OK && cudaEventSynchronize(b) == cudaSuccess) cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ms;
}

// The batched traversal's scan: database splits x widening; each candidate
// is put in the table for the call that times it, the fastest stays.
int tune_tree_tc(const dt_index *ix, const uint64_t *d_q, int64_t nq, int k, uint32_t *idx,
                 float *score, cudaStream_t s, dt_tune_report *report, int *tried)
{
    TuneCfg best{0, 0}, saved{0, 0};
    const bool had = tune_lookup(TUNE_TREE_TC, ix->n, nq, k, &saved);
    float best_ms = 1e30f;
    for (int pre : {1, 2})
        for (int splits : {4, 8, 16, 19, 32, 64}) {
            const TuneCfg c{splits, pre};
            tune_store(TUNE_TREE_TC, ix->n, nq, k, c);
            float ms = time_call([&] {
                return launch_dt_search_batched(ix, d_q, nq, k, nullptr, 0, idx, score, nullptr,
                                                nullptr, s);
            }, s);
            ++*tried;
            if (ms > 0.f && ms < best_ms) {
                best_ms = ms;
                best = c;
            }
        }
    if (best.a) tune_store(TUNE_TREE_TC, ix->n, nq, k, best);
    else if (had) tune_store(TUNE_TREE_TC, ix->n, nq, k, saved);
    if (report && best.a) {
        report->tree_tc_splits = best.a;
        report->tree_tc_prewiden = best.b;
        report->tree_tc_ms = best_ms;
    }
    return DT_OK;
}

}  // namespace
}  // namespace dtk

using namespace dtk;

extern "C" {

int dt_autotune(const dt_index *ix, const uint64_t *d_db, int64_t n, const uint64_t *d_q,
                int64_t nq, int32_t k, void *stream, dt_tune_report *report)
{
    if (report) *report = dt_tune_report{};
    DT_CHECK_ARG(d_q != nullptr && nq >= 1, "queries required");
    DT_CHECK_ARG(k >= 1 && k <= DT_MAX_K, "k must be in [1, DT_MAX_K]");
    DT_CHECK_ARG(ix != nullptr || (d_db != nullptr && n >= 1), "an index or a database is required");
    cudaStream_t s = (cudaStream_t)stream;
    Scratch scratch(s);
    uint32_t *idx = nullptr;
    float *score = nullptr;
    DT_CUDA_TRY(scratch.alloc(&idx, (size_t)nq * k * 4));
    DT_CUDA_TRY(scratch.alloc(&score, (size_t)nq * k * 4));
    int tried = 0;
    if (ix) {
        TuneCfg best{0, 0};
        float best_ms = 1e30f;
        for (int threads : {128, 256})
            for (int bps : {1, 2, 3, 4, 6, 8}) {
                if (threads * bps > 2048) continue;
                TuneCfg c{threads, bps};
                float ms = time_call([&] {
                    return launch_dt_search_cfg(ix, d_q, nq, k, idx, score, nullptr, nullptr, s, &c, nullptr, 0);
                }, s);
                ++tried;
                if (ms > 0.f && ms < best_ms) {
                    best_ms = ms;
                    best = c;
                }
            }
        if (best.a) {
            tune_store(TUNE_TREE, ix->n, nq, k, best);
            if (report) {
                report->tree_threads = best.a;
                report->tree_blocks_per_sm = best.b;
                report->tree_ms = best_ms;
            }
        }
    }
    if (ix) {
        if (int r = tune_tree_tc(ix, d_q, nq, k, idx, score, s, report, &tried)) return r;
    }
    if (d_db) {
        for (int kind = TUNE_POPC; kind <= TUNE_TC; ++kind) {
            TuneCfg best{0, 0};
            float best_ms = 1e30f;
            for (int pre : {0, 1, 2}) {
                if ((kind == TUNE_POPC) != (pre == 0)) continue;   // widening: tensor path only
                for (int splits : {1, 2, 4, 8, 16, 32, 64, 128}) {
                    TuneCfg c{splits, pre};
                    float ms = time_call([&] {
                        return kind == TUNE_POPC
                                   ? launch_bf_popc_cfg(d_db, n, d_q, nq, k, idx, score, nullptr, s, &c)
                                   : launch_bf_tc_cfg(d_db, n, d_q, nq, k, idx, score, nullptr, s, &c);
                    }, s);
                    ++tried;
                    if (ms > 0.f && ms < best_ms) {
                        best_ms = ms;
                        best = c;
                    }
                }
            }
            if (best.a) {
                tune_store((TuneKind)kind, n, nq, k, best);
                if (report) {
                    if (kind == TUNE_POPC) {
                        report->popc_splits = best.a;
                        report->popc_ms = best_ms;
                    } else {
                        report->tc_splits = best.a;
                        report->tc_prewiden = best.b;
                        report->tc_ms = best_ms;
                    }
                }
            }
        }
    }
    DT_CUDA_TRY(cudaStreamSynchronize(s));
    if (report) report->candidates_timed = tried;
    return DT_OK;
}

int dt_autotune_retrieve(const dt_index *ix, const uint32_t *d_object_of_desc, int32_t n_objects,
                         const uint64_t *d_qdesc, const int64_t *d_qoffsets, int32_t nq,
                         int64_t n_qdesc, int32_t vote_threshold, void *stream,
                         dt_tune_report *report)
{
    if (report) *report = dt_tune_report{};
    DT_CHECK_ARG(ix != nullptr && d_object_of_desc != nullptr && d_qdesc != nullptr &&
                 d_qoffsets != nullptr, "index, object ids, query descriptors and offsets required");
    DT_CHECK_ARG(n_objects >= 1 && nq >= 1 && n_qdesc >= 1 && n_qdesc < (1LL << 31) &&
                 vote_threshold >= 0, "sizes out of range");
    cudaStream_t s = (cudaStream_t)stream;
    Scratch scratch(s);
    uint32_t *votes = nullptr;
    int32_t *winner = nullptr;
    int64_t *consumed = nullptr;
    DT_CUDA_TRY(scratch.alloc(&votes, (size_t)nq * n_objects * 4));
    DT_CUDA_TRY(scratch.alloc(&winner, (size_t)nq * 4));
    DT_CUDA_TRY(scratch.alloc(&consumed, (size_t)nq * 8));
    // the batched search behind engine 3 at this batch size first
    dt_tune_report sub{};
    int tried = 0;
    if (vote_threshold == 0) {
        uint32_t *nn = nullptr;
        float *sc = nullptr;
        DT_CUDA_TRY(scratch.alloc(&nn, (size_t)n_qdesc * 4));
        DT_CUDA_TRY(scratch.alloc(&sc, (size_t)n_qdesc * 4));
        if (int r = tune_tree_tc(ix, d_qdesc, n_qdesc, 1, nn, sc, s, &sub, &tried)) return r;
    }
    const int key_nq = vote_threshold > 0 ? 2 : 1;
    TuneCfg best{0, 0};
    float best_ms = 1e30f;
    const TuneCfg cands[] = {{1, 0}, {1, 2}, {1, 4}, {2, 0}, {3, 0}};
    for (const TuneCfg &c : cands) {
        float ms = time_call([&] {
            return launch_retrieve(ix, d_object_of_desc, n_objects, d_qdesc, d_qoffsets, nq, n_qdesc,
                                   vote_threshold, 0x9e3779b97f4a7c15ull, votes, winner, consumed, 0,
                                   s, &c);
        }, s);
        ++tried;
        if (ms > 0.f && ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    DT_CUDA_TRY(cudaStreamSynchronize(s));
    if (best.a) tune_store(TUNE_RETRIEVE, ix->n, key_nq, 1, best);
    if (report) {
        *report = sub;
        report->retrieve_engine = best.a;
        report->retrieve_blocks_per_sm = best.b;
        report->retrieve_ms = best.a ? best_ms : 0.f;
        report->candidates_timed = tried;
    }
    return best.a ? DT_OK : DT_ECUDA;
}

int dt_tune_save(const char *path)
{
    DT_CHECK_ARG(path != nullptr, "path must not be NULL");
    std::lock_guard<std::mutex> lock(g_tune_mu);
    FILE *f = std::fopen(path, "w");
    DT_CHECK_ARG(f != nullptr, "cannot open the tuning file for writing");
    for (const auto &e : g_tune)
        std::fprintf(f, "%d %d %d %d %d %d %d\n", std::get<0>(e.first), std::get<1>(e.first),
                     std::get<2>(e.first), std::get<3>(e.first), std::get<4>(e.first), e.second.a,
                     e.second.b);
    std::fclose(f);
    return DT_OK;
}

int dt_tune_load(const char *path)
{
    DT_CHECK_ARG(path != nullptr, "path must not be NULL");
    FILE *f = std::fopen(path, "r");
    DT_CHECK_ARG(f != nullptr, "cannot open the tuning file");
    std::lock_guard<std::mutex> lock(g_tune_mu);
    int kind, nl, ql, k, sms, a, b, loaded = 0;
    while (std::fscanf(f, "%d %d %d %d %d %d %d", &kind, &nl, &ql, &k, &sms, &a, &b) == 7) {
        if (kind < TUNE_TREE || kind > TUNE_RETRIEVE || a <= 0 || b < 0) continue;
        g_tune[Key(kind, nl, ql, k, sms)] = TuneCfg{a, b};
        ++loaded;
    }
    std::fclose(f);
    return loaded;
}

void dt_tune_clear(void) { tune_clear(); }

}  // extern "C"
