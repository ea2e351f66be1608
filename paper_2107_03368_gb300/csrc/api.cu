// api.cu — the C ABI of include/dt.h: argument checks, index lifetime and
// dispatch to the kernel launchers.  No computation happens here.
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "dt_internal.cuh"
#include "encoder_layout.cuh"

namespace dtk {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

int sm_count()
{
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    if (!cached[dev]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = v > 0 ? v : 1;
        cudaGetLastError();
    }
    return cached[dev];
}

// The library's own stream-ordered memory pool on the current device,
// created on first use and kept until the process exits.  Its release
// threshold is 16 GiB, so scratch freed by one call is reused by the next
// instead of being unmapped at every synchronisation.  A pool of its own
// leaves the caller's default pool and its settings untouched.
static cudaError_t library_pool(cudaMemPool_t *out)
{
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        e = cudaMemPoolCreate(&pool, &props);
        if (e != cudaSuccess) return e;
        uint64_t keep = 16ull << 30;
        e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(pool);
            return e;
        }
        pools[dev] = pool;
    }
    *out = pools[dev];
    return cudaSuccess;
}

cudaError_t allow_smem(const void *func, int bytes)
{
    static std::mutex mu;
    static std::vector<std::pair<std::pair<const void *, int>, int>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    for (const auto &d : done)
        if (d.first.first == func && d.first.second == dev && d.second >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done.push_back({{func, dev}, bytes});
    return e;
}

// Kernel timing: event pairs per kernel name, read and released by
// dt_kernel_time / dt_kernel_timing.
static std::mutex g_timing_mu;
static std::atomic<bool> g_timing_on{false};
static std::vector<std::pair<std::string, std::pair<cudaEvent_t, cudaEvent_t>>> g_timing;

bool kernel_timing_on() { return g_timing_on.load(); }

void kernel_timing_add(const char *name, cudaEvent_t start, cudaEvent_t stop)
{
    std::lock_guard<std::mutex> lock(g_timing_mu);
    g_timing.push_back({std::string(name), {start, stop}});
}

static void kernel_timing_clear()
{
    std::lock_guard<std::mutex> lock(g_timing_mu);
    for (auto &e : g_timing) {
        cudaEventDestroy(e.second.first);
        cudaEventDestroy(e.second.second);
    }
    g_timing.clear();
}

// Test hook: when positive, the n-th scratch allocation from now fails.
static std::atomic<int> g_fail_alloc{0};

cudaError_t dt_malloc_async(void **p, size_t bytes, cudaStream_t s)
{
    int n = g_fail_alloc.load();
    while (n > 0 && !g_fail_alloc.compare_exchange_weak(n, n - 1)) {
    }
    if (n == 1) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    // Under stream capture the allocation becomes a node of the graph and
    // its memory belongs to the graph, whichever pool is named.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
        cudaGetLastError();
        cap = cudaStreamCaptureStatusNone;
    }
    if (cap != cudaStreamCaptureStatusNone) return cudaMallocAsync(p, bytes, s);
    cudaMemPool_t pool = nullptr;
    const cudaError_t e = library_pool(&pool);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

// A device (or managed) allocation; host pointers would make kernels fault.
static bool is_device_ptr(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace dtk

using namespace dtk;

#define REQUIRE_DEV(p, name)                                                     \
    DT_CHECK_ARG((p) != nullptr && aligned16_ok(p) && is_device_ptr(p),           \
                 std::string(name) + " must be a non-null device pointer")

template <typename T>
static bool aligned16_ok(const T *) { return true; }
static bool aligned16_ok(const uint64_t *p) { return aligned16(p); }

static int check_k(int32_t k)
{
    DT_CHECK_ARG(k >= 1 && k <= DT_MAX_K, "k must be in [1, DT_MAX_K]");
    return DT_OK;
}

extern "C" {

const char *dt_status_string(int status)
{
    switch (status) {
    case DT_OK: return "DT_OK";
    case DT_EINVAL: return "DT_EINVAL";
    case DT_ENOMEM: return "DT_ENOMEM";
    case DT_ECUDA: return "DT_ECUDA";
    case DT_ETIMEOUT: return "DT_ETIMEOUT";
    case DT_EUNSUPPORTED: return "DT_EUNSUPPORTED";
    case DT_EIO: return "DT_EIO";
    default: return "DT_UNKNOWN";
    }
}

const char *dt_last_error(void) { return g_last_error.c_str(); }

int dt_build(const uint64_t *d_db, int64_t n, const dt_build_params *params, void *stream,
             dt_index **out)
{
    g_last_error.clear();
    DT_CHECK_ARG(out != nullptr, "out must not be NULL");
    *out = nullptr;
    DT_CHECK_ARG(n >= 1 && n <= DT_MAX_N - 65536, "n out of range");
    REQUIRE_DEV(d_db, "d_db");
    dt_build_params p{32, 0, 0, 0};
    if (params) p = *params;
    DT_CHECK_ARG(p.reserved == 0, "params->reserved must be 0");
    if (p.leaf_size <= 0) p.leaf_size = 32;
    DT_CHECK_ARG(p.leaf_size <= 4096, "leaf_size must be <= 4096");
    cudaStream_t s = (cudaStream_t)stream;
    dt_index *ix = new dt_index();
    DT_CUDA_TRY(cudaGetDevice(&ix->device));
    int rc = build_tree(d_db, n, p.leaf_size, p.use_and_image ? 1 : 0, p.fused_cap, s, ix);
    if (rc != DT_OK) {
        dt_free(ix);
        return rc;
    }
    *out = ix;
    return DT_OK;
}

int dt_insert(dt_index *ix, const uint64_t *d_new, int64_t m, void *stream)
{
    g_last_error.clear();
    DT_CHECK_ARG(ix != nullptr, "index must not be NULL");
    DT_CHECK_ARG(m >= 0 && m <= DT_MAX_N - 65536 - ix->n, "m out of range");
    if (m == 0) return DT_OK;
    REQUIRE_DEV(d_new, "d_new");
    int dev = -1;
    DT_CUDA_TRY(cudaGetDevice(&dev));
    DT_CHECK_ARG(dev == ix->device, "the current device must be the index's device");
    const bool kept = ix->scan_exp != nullptr;
    const int rc = insert_tree(ix, d_new, m, (cudaStream_t)stream);
    if (rc == DT_OK && kept) {
        // the rows moved: rebuild the kept widened copy, or leave it off
        // when it no longer fits (searches stay exact, only slower)
        if (int r = index_keep_widened(ix, false, (cudaStream_t)stream)) return r;
        const int r = index_keep_widened(ix, true, (cudaStream_t)stream);
        if (r != DT_OK && r != DT_ENOMEM) return r;
    }
    return rc;
}

int dt_keep_widened(dt_index *ix, int32_t on, void *stream)
{
    g_last_error.clear();
    DT_CHECK_ARG(ix != nullptr, "index must not be NULL");
    DT_CHECK_ARG(on == 0 || on == 1, "on must be 0 or 1");
    int dev = -1;
    DT_CUDA_TRY(cudaGetDevice(&dev));
    DT_CHECK_ARG(dev == ix->device, "the current device must be the index's device");
    const int rc = index_keep_widened(ix, on != 0, (cudaStream_t)stream);
    if (rc == DT_ENOMEM) set_error("no room for the widened copy (4 KB per descriptor)");
    return rc;
}

int quicci_generate(const float *d_vertices, int64_t n_vertices, const int32_t *d_triangles,
                    int64_t n_triangles, const float *d_points, const float *d_normals,
                    int64_t n_points, float support_radius, int32_t modified, uint64_t *d_out,
                    void *stream)
{
    g_last_error.clear();
    DT_CHECK_ARG(n_vertices >= 0 && n_vertices <= 2147483647LL, "n_vertices out of range");
    DT_CHECK_ARG(n_triangles >= 0 && n_triangles <= 2147483647LL, "n_triangles out of range");
    DT_CHECK_ARG(n_points >= 0 && n_points < (1LL << 40), "n_points out of range");
    DT_CHECK_ARG(support_radius > 0.f && std::isfinite(support_radius),
                 "support_radius must be positive and finite");
    DT_CHECK_ARG(n_triangles == 0 || n_vertices >= 1, "triangles need vertices");
    if (n_points == 0) return DT_OK;
    if (n_triangles > 0) {
        REQUIRE_DEV(d_vertices, "d_vertices");
        REQUIRE_DEV(d_triangles, "d_triangles");
    }
    REQUIRE_DEV(d_points, "d_points");
    REQUIRE_DEV(d_normals, "d_normals");
    REQUIRE_DEV(d_out, "d_out");
    return launch_quicci(d_vertices, n_vertices, d_triangles, n_triangles, d_points, d_normals,
                         n_points, support_radius, modified, d_out, (cudaStream_t)stream);
}

int dt_get_info(const dt_index *ix, dt_index_info *info)
{
    DT_CHECK_ARG(ix && info, "index and info must not be NULL");
    std::memset(info, 0, sizeof(*info));
    info->n_nodes = ix->n_nodes;
    info->n_leaves = ix->n_leaves;
    info->depth = ix->depth;
    info->leaf_size = ix->leaf_size;
    info->n = ix->n;
    info->use_and_image = ix->use_and;
    return DT_OK;
}

int dt_export(const dt_index *ix, int64_t *h_child, int64_t *h_begin, int64_t *h_count,
              int32_t *h_level, uint64_t *h_or, uint64_t *h_and, int64_t *h_perm)
{
    g_last_error.clear();
    DT_CHECK_ARG(ix != nullptr, "index must not be NULL");
    DT_CHECK_ARG(!h_and || ix->use_and, "index has no AND images");
    const int64_t m = ix->n_nodes;
    std::vector<NodeRec> recs((size_t)m);
    DT_CUDA_TRY(cudaMemcpy(recs.data(), ix->node, (size_t)m * sizeof(NodeRec), cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < m; ++i) {
        const NodeRec &r = recs[(size_t)i];
        if (h_child) {
            h_child[2 * i] = r.first_child < 0 ? -1 : r.first_child;
            h_child[2 * i + 1] = r.first_child < 0 ? -1 : r.first_child + 1;
        }
        if (h_begin) h_begin[i] = r.begin;
        if (h_count) h_count[i] = r.count;
        if (h_level) h_level[i] = r.level;
    }
    if (h_or)
        DT_CUDA_TRY(cudaMemcpy(h_or, ix->or_img, (size_t)m * DT_WORDS * 8, cudaMemcpyDeviceToHost));
    if (h_and)
        DT_CUDA_TRY(cudaMemcpy(h_and, ix->and_img, (size_t)m * DT_WORDS * 8, cudaMemcpyDeviceToHost));
    if (h_perm) {
        std::vector<uint32_t> p((size_t)ix->n);
        DT_CUDA_TRY(cudaMemcpy(p.data(), ix->perm, (size_t)ix->n * 4, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < ix->n; ++i) h_perm[i] = p[(size_t)i];
    }
    return DT_OK;
}

// Both traversals give identical results.  The batched one shares each scan
// of the database among tiles of queries and wins from a few dozen queries;
// on a large index it also wins for a single query, because a per-query
// walk is one warp streaming most of the database (10M descriptors, 1 to 32
// queries: 2.1-2.3 s per query walk, 13 ms batched, 9 ms with the rows kept
// widened).
constexpr int64_t kBatchedMinQueries = 64;
constexpr int64_t kBatchedMinRows = int64_t(1) << 17;
static int search_any(const dt_index *ix, const uint64_t *d_q, int64_t nq, int32_t k,
                      const uint32_t *d_seed, int32_t n_seed, uint32_t *d_idx, float *d_score,
                      uint16_t *d_ab, dt_stats *h_stats, int32_t path, void *stream)
{
    g_last_error.clear();
    DT_CHECK_ARG(ix != nullptr, "index must not be NULL");
    if (int r = check_k(k)) return r;
    DT_CHECK_ARG(nq >= 0 && nq < (1LL << 31), "nq out of range");
    DT_CHECK_ARG(n_seed >= 0 && n_seed <= 4096, "n_seed must be in [0, 4096]");
    DT_CHECK_ARG(path >= 0 && path <= 2, "path must be 0, 1 or 2");
    if (h_stats) std::memset(h_stats, 0, sizeof(*h_stats));
    if (nq == 0) return DT_OK;
    REQUIRE_DEV(d_q, "d_q");
    REQUIRE_DEV(d_idx, "d_idx");
    REQUIRE_DEV(d_score, "d_score");
    if (d_ab) REQUIRE_DEV(d_ab, "d_ab");
    if (n_seed > 0) REQUIRE_DEV(d_seed, "d_seed");
    else d_seed = nullptr;
    int dev = -1;
    DT_CUDA_TRY(cudaGetDevice(&dev));
    DT_CHECK_ARG(dev == ix->device, "the current device must be the index's device");
    cudaStream_t s = (cudaStream_t)stream;
    if (path == 2 || (path == 0 && (nq >= kBatchedMinQueries || ix->n >= kBatchedMinRows)))
        return launch_dt_search_batched(ix, d_q, nq, k, d_seed, n_seed, d_idx, d_score, d_ab,
                                        h_stats, s);
    if (d_seed)
        return launch_dt_search_seeded(ix, d_q, nq, k, d_seed, n_seed, d_idx, d_score, d_ab,
                                       h_stats, s);
    return launch_dt_search(ix, d_q, nq, k, d_idx, d_score, d_ab, h_stats, s);
}

int dt_search(const dt_index *ix, const uint64_t *d_q, int64_t nq, int32_t k, uint32_t *d_idx,
              float *d_score, uint16_t *d_ab, dt_stats *h_stats, void *stream)
{
    return search_any(ix, d_q, nq, k, nullptr, 0, d_idx, d_score, d_ab, h_stats, 0, stream);
}

int dt_search_seeded(const dt_index *ix, const uint64_t *d_q, int64_t nq, int32_t k,
                     const uint32_t *d_seed, int32_t n_seed, uint32_t *d_idx, float *d_score,
                     uint16_t *d_ab, dt_stats *h_stats, void *stream)
{
    return search_any(ix, d_q, nq, k, d_seed, n_seed, d_idx, d_score, d_ab, h_stats, 0, stream);
}

int dt_search_path(const dt_index *ix, const uint64_t *d_q, int64_t nq, int32_t k,
                   const uint32_t *d_seed, int32_t n_seed, uint32_t *d_idx, float *d_score,
                   uint16_t *d_ab, dt_stats *h_stats, int32_t path, void *stream)
{
    return search_any(ix, d_q, nq, k, d_seed, n_seed, d_idx, d_score, d_ab, h_stats, path, stream);
}

int bf_search(const uint64_t *d_db, int64_t n, const uint64_t *d_q, int64_t nq, int32_t k,
              uint32_t *d_idx, float *d_score, uint16_t *d_ab, int32_t path, void *stream)
{
    g_last_error.clear();
    if (int r = check_k(k)) return r;
    DT_CHECK_ARG(n >= 1 && n <= DT_MAX_N - 65536, "n out of range");
    DT_CHECK_ARG(nq >= 0 && nq < (1LL << 31), "nq out of range");
    DT_CHECK_ARG(path >= 0 && path <= 2, "path must be 0, 1 or 2");
    if (nq == 0) return DT_OK;
    REQUIRE_DEV(d_db, "d_db");
    REQUIRE_DEV(d_q, "d_q");
    REQUIRE_DEV(d_idx, "d_idx");
    REQUIRE_DEV(d_score, "d_score");
    if (d_ab) REQUIRE_DEV(d_ab, "d_ab");
    if (path == 2 || (path == 0 && nq >= 64))
        return launch_bf_tc(d_db, n, d_q, nq, k, d_idx, d_score, d_ab, (cudaStream_t)stream);
    return launch_bf_popc(d_db, n, d_q, nq, k, d_idx, d_score, d_ab, (cudaStream_t)stream);
}

// Same checks as bf_search; the size limit of the fixed scratch is checked
// before any CUDA call, and nothing here or below allocates.
int bf_search_noalloc(const uint64_t *d_db, int64_t n, const uint64_t *d_q, int64_t nq, int32_t k,
                      uint32_t *d_idx, float *d_score, uint16_t *d_ab, void *stream)
{
    g_last_error.clear();
    if (int r = check_k(k)) return r;
    DT_CHECK_ARG(n >= 1 && n <= DT_MAX_N - 65536, "n out of range");
    DT_CHECK_ARG(nq >= 0 && nq < (1LL << 31), "nq out of range");
    DT_CHECK_ARG((uint64_t)nq * (uint64_t)k * 8u <= (uint64_t)DT_NOALLOC_SCRATCH_BYTES,
                 "bf_search_noalloc: nq * k * 8 exceeds DT_NOALLOC_SCRATCH_BYTES; "
                 "search the queries in smaller batches");
    if (nq == 0) return DT_OK;
    REQUIRE_DEV(d_db, "d_db");
    REQUIRE_DEV(d_q, "d_q");
    REQUIRE_DEV(d_idx, "d_idx");
    REQUIRE_DEV(d_score, "d_score");
    if (d_ab) REQUIRE_DEV(d_ab, "d_ab");
    return launch_bf_popc_noalloc(d_db, n, d_q, nq, k, d_idx, d_score, d_ab, (cudaStream_t)stream);
}

int retrieve_objects(const dt_index *ix, const uint32_t *d_object_of_desc, int32_t n_objects,
                     const uint64_t *d_qdesc, const int64_t *d_qoffsets, int32_t nq,
                     int64_t n_qdesc, int32_t vote_threshold, uint64_t seed, uint32_t *d_votes,
                     int32_t *d_winner, int64_t *d_consumed, int32_t engine, void *stream)
{
    g_last_error.clear();
    DT_CHECK_ARG(ix != nullptr, "index must not be NULL");
    DT_CHECK_ARG(n_objects >= 1, "n_objects must be >= 1");
    DT_CHECK_ARG(nq >= 0, "nq must be >= 0");
    DT_CHECK_ARG(n_qdesc >= 0 && n_qdesc < (1LL << 31), "n_qdesc out of range");
    DT_CHECK_ARG(vote_threshold >= 0, "vote_threshold must be >= 0");
    DT_CHECK_ARG(engine >= 0 && engine <= 3, "engine must be 0, 1, 2 or 3");
    if (nq == 0) return DT_OK;
    REQUIRE_DEV(d_object_of_desc, "d_object_of_desc");
    REQUIRE_DEV(d_qdesc, "d_qdesc");
    REQUIRE_DEV(d_qoffsets, "d_qoffsets");
    REQUIRE_DEV(d_votes, "d_votes");
    REQUIRE_DEV(d_winner, "d_winner");
    if (d_consumed) REQUIRE_DEV(d_consumed, "d_consumed");
    return launch_retrieve(ix, d_object_of_desc, n_objects, d_qdesc, d_qoffsets, nq, n_qdesc,
                           vote_threshold, seed, d_votes, d_winner, d_consumed, engine,
                           (cudaStream_t)stream);
}

int dt_kernel_timing(int32_t on)
{
    g_last_error.clear();
    kernel_timing_clear();
    g_timing_on.store(on != 0);
    return DT_OK;
}

int dt_kernel_time(const char *name, double *ms, int64_t *launches)
{
    g_last_error.clear();
    DT_CHECK_ARG(name != nullptr && ms != nullptr && launches != nullptr,
                 "name, ms and launches must not be NULL");
    std::lock_guard<std::mutex> lock(g_timing_mu);
    double total = 0.0;
    int64_t count = 0;
    for (auto &e : g_timing) {
        if (e.first != name) continue;
        DT_CUDA_TRY(cudaEventSynchronize(e.second.second));
        float t = 0.f;
        DT_CUDA_TRY(cudaEventElapsedTime(&t, e.second.first, e.second.second));
        total += t;
        ++count;
    }
    *ms = total;
    *launches = count;
    return DT_OK;
}

void dt_debug_fail_allocation(int32_t nth) { g_fail_alloc.store(nth > 0 ? nth : 0); }

void dt_debug_inject_missing_copy(int32_t on) { set_drop_copy(on != 0); }

int dt_sync_status(void *stream)
{
    g_last_error.clear();
    DT_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    bool raised = false, raised_tc = false, raised_enc = false;
    if (int r = take_bf_error(&raised)) return r;
    if (int r = take_tc_error(&raised_tc)) return r;
    if (int r = take_enc_tc_error(&raised_enc)) return r;
    raised = raised || raised_tc || raised_enc;
    if (raised) {
        set_error("a tile copy or tensor-core stage did not arrive within the spin limit");
        return DT_ETIMEOUT;
    }
    return DT_OK;
}

void dt_free(dt_index *ix)
{
    if (!ix) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(ix->device);
    cudaDeviceSynchronize();
    cudaFree(ix->db_tree);
    cudaFree(ix->perm);
    cudaFree(ix->iperm);
    cudaFree(ix->or_img);
    cudaFree(ix->and_img);
    cudaFree(ix->node);
    cudaFree(ix->tile_or);
    cudaFree(ix->tile_kmask);
    cudaFree(ix->scan_exp);
    cudaFree(ix->scan_side);
    cudaSetDevice(cur);
    delete ix;
}

}  // extern "C"
