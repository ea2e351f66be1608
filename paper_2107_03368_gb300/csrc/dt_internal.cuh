// dt_internal.cuh — shared pieces of the CUDA library behind include/dt.h.
#pragma once

#include <cstdint>
#include <cstdio>
#include <algorithm>
#include <string>
#include <vector>
#include <cuda_runtime.h>

#include "dt.h"

namespace dtk {

constexpr int kWords = DT_WORDS;      // uint64 words per descriptor
constexpr int kBits = DT_BITS;
constexpr int kMaxK = DT_MAX_K;
constexpr uint64_t kEmpty = ~0ull;    // packed (key, idx) of a missing result

// ---------------------------------------------------------------------------
// Ranking key.  For a query with P = max(|q|,1), Z = max(4096-|q|,1), Eq. 1
// times P*Z is the integer A*Z + B*P < 2^24, which orders targets exactly.
// A result is packed as (key << 32) | idx so that one 64-bit comparison
// ranks by (distance, index).
// ---------------------------------------------------------------------------
struct QueryWeights {
    uint32_t pop, P, Z;
};

__host__ __device__ inline QueryWeights query_weights(uint32_t pop)
{
    QueryWeights w;
    w.pop = pop;
    w.P = pop > 1 ? pop : 1;
    w.Z = (uint32_t)kBits - pop > 1 ? (uint32_t)kBits - pop : 1;
    return w;
}

// A = |q| - O, B = |t| - O with O = popc(q & t).
__device__ __forceinline__ uint32_t pair_key(const QueryWeights &w, uint32_t overlap,
                                             uint32_t tpop)
{
    return (w.pop - overlap) * w.Z + (tpop - overlap) * w.P;
}

__device__ __forceinline__ uint64_t pack(uint32_t key, uint32_t idx)
{
    return ((uint64_t)key << 32) | idx;
}

// FP32 score: the exact rational key / (P*Z), correctly rounded (both
// operands are exact in FP32: key < 2^24, P*Z <= 2^22).
__device__ __forceinline__ float key_score(const QueryWeights &w, uint32_t key)
{
    return __fdiv_rn((float)key, (float)(w.P * w.Z));
}

// ---------------------------------------------------------------------------
// Warp helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t shfl_u64(uint64_t v, int src)
{
    return __shfl_sync(0xffffffffu, v, src);
}

__device__ __forceinline__ uint32_t warp_sum(uint32_t v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ uint64_t warp_min_u64(uint64_t v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        uint64_t u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u < v ? u : v;
    }
    return v;
}

// Sorted top-k list held across a warp: lane i holds the i-th smallest
// packed result (kEmpty past the end).  Inserting v keeps the k smallest.
__device__ __forceinline__ void warp_list_insert(uint64_t &slot, uint64_t v, int lane)
{
    uint64_t up = __shfl_up_sync(0xffffffffu, slot, 1);
    if (lane == 0) up = 0;                 // nothing is smaller than lane 0's predecessor
    if (slot > v) slot = (up > v) ? up : v;
}

// Merge the (lane-distributed, unsorted) candidates cand into the sorted
// list; only candidates below the current k-th entry are inserted.
__device__ __forceinline__ void warp_list_merge(uint64_t &slot, uint64_t cand, int k, int lane)
{
    uint64_t worst = shfl_u64(slot, k - 1);
    unsigned m = __ballot_sync(0xffffffffu, cand < worst);
    while (m) {
        int src = __ffs(m) - 1;
        m &= m - 1;
        uint64_t v = shfl_u64(cand, src);
        worst = shfl_u64(slot, k - 1);
        if (v < worst) warp_list_insert(slot, v, lane);
    }
}

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------
void set_error(const std::string &msg);

#define DT_CUDA_TRY(expr)                                                          \
    do {                                                                           \
        cudaError_t e_ = (expr);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            ::dtk::set_error(std::string(#expr) + ": " + cudaGetErrorString(e_));  \
            return e_ == cudaErrorMemoryAllocation ? DT_ENOMEM : DT_ECUDA;         \
        }                                                                          \
    } while (0)

#define DT_CHECK_ARG(cond, msg)                                                    \
    do {                                                                           \
        if (!(cond)) {                                                             \
            ::dtk::set_error(msg);                                                 \
            return DT_EINVAL;                                                      \
        }                                                                          \
    } while (0)

inline bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// Every scratch allocation of the library: stream-ordered, from the
// library's own pool (graph memory under stream capture), except that a
// test hook (dt_debug_fail_allocation) can make the n-th one report
// cudaErrorMemoryAllocation.
cudaError_t dt_malloc_async(void **p, size_t bytes, cudaStream_t s);

// Stream-ordered scratch of one call: every buffer it hands out is freed on
// the stream (after the work enqueued so far) when it goes out of scope, on
// success and on every early error return alike.
class Scratch {
  public:
    explicit Scratch(cudaStream_t s) : s_(s) {}
    Scratch(const Scratch &) = delete;
    Scratch &operator=(const Scratch &) = delete;
    ~Scratch()
    {
        for (int i = n_ - 1; i >= 0; --i) cudaFreeAsync(p_[i], s_);
    }
    template <class T> cudaError_t alloc(T **out, size_t bytes)
    {
        *out = nullptr;
        if (n_ == kMax) return cudaErrorMemoryAllocation;
        void *p = nullptr;
        const cudaError_t e = dt_malloc_async(&p, bytes, s_);
        if (e != cudaSuccess) return e;
        p_[n_++] = p;
        *out = static_cast<T *>(p);
        return cudaSuccess;
    }

  private:
    static constexpr int kMax = 32;
    cudaStream_t s_;
    void *p_[kMax] = {};
    int n_ = 0;
};

// Device buffer that grows by doubling, keeping its contents.
struct Grow {
    void *p = nullptr;
    size_t bytes = 0;
    int ensure(size_t need, cudaStream_t s)
    {
        if (need <= bytes) return DT_OK;
        size_t nb = std::max(need, bytes * 2);
        void *q = nullptr;
        DT_CUDA_TRY(dt_malloc_async(&q, nb, s));
        if (p) {
            DT_CUDA_TRY(cudaMemcpyAsync(q, p, bytes, cudaMemcpyDeviceToDevice, s));
            DT_CUDA_TRY(cudaFreeAsync(p, s));
        }
        p = q;
        bytes = nb;
        return DT_OK;
    }
    void release(cudaStream_t s)
    {
        if (p) cudaFreeAsync(p, s);
        p = nullptr;
        bytes = 0;
    }
};

int sm_count();

// Kernel timing (dt_kernel_timing / dt_kernel_time): while switched on, a
// KernelTimer around a launch records a CUDA event pair on its stream
// (nothing under stream capture, nothing while off), totalled per name.
bool kernel_timing_on();
void kernel_timing_add(const char *name, cudaEvent_t start, cudaEvent_t stop);
class KernelTimer {
  public:
    KernelTimer(const char *name, cudaStream_t s) : name_(name), s_(s)
    {
        if (!kernel_timing_on()) return;
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
            cudaGetLastError();
            return;
        }
        if (cudaEventCreate(&a_) != cudaSuccess || cudaEventCreate(&b_) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        on_ = cudaEventRecord(a_, s) == cudaSuccess;
    }
    ~KernelTimer()
    {
        if (on_ && cudaEventRecord(b_, s_) == cudaSuccess) {
            kernel_timing_add(name_, a_, b_);
            return;
        }
        if (a_) cudaEventDestroy(a_);
        if (b_) cudaEventDestroy(b_);
    }
    KernelTimer(const KernelTimer &) = delete;
    KernelTimer &operator=(const KernelTimer &) = delete;

  private:
    const char *name_;
    cudaStream_t s_;
    cudaEvent_t a_ = nullptr, b_ = nullptr;
    bool on_ = false;
};

// Let `func` use `bytes` of dynamic shared memory on the current device (a
// per-device setting, applied once per kernel and device).
cudaError_t allow_smem(const void *func, int bytes);

// ---------------------------------------------------------------------------
// Index
// ---------------------------------------------------------------------------
struct NodeRec {          // 16 bytes, one load per node
    int32_t first_child;  // similar child id (dissimilar = +1); -1 at a leaf
    int32_t begin;        // segment of the tree-ordered arrays
    int32_t count;
    int32_t level;
};

}  // namespace dtk

struct dt_index {
    int64_t n = 0;
    int64_t n_nodes = 0;
    int64_t n_leaves = 0;
    int32_t depth = 0;
    int32_t leaf_size = 32;
    int32_t use_and = 0;
    int device = 0;
    uint64_t *db_tree = nullptr;    // [n][64] descriptors in tree order
    uint32_t *perm = nullptr;       // [n] tree position -> original index
    uint32_t *iperm = nullptr;      // [n] original index -> tree position
    uint64_t *or_img = nullptr;     // [n_nodes][64]
    uint64_t *and_img = nullptr;    // [n_nodes][64] when use_and
    dtk::NodeRec *node = nullptr;   // [n_nodes]
    // Scan tiles of the batched search: tile i = tree positions
    // [128 i, 128 i + 128).  tile_or[i] is the OR image of its rows and
    // tile_kmask[i] has bit c set when that image has a bit in the 128-bit
    // chunk c (words 2c, 2c + 1).  ceil(n / 128) entries each.
    uint64_t *tile_or = nullptr;
    uint32_t *tile_kmask = nullptr;
    // Optional (dt_keep_widened): the tree-ordered rows as FP8 stage images
    // of the tensor-core scan, [scan tile][128-bit chunk][16 KB], and each
    // scan tile's |t| record; null when not kept.
    unsigned char *scan_exp = nullptr;
    uint32_t *scan_side = nullptr;
};

namespace dtk {
// Autotuner table (autotune.cu): a launch shape per kernel kind and problem size.
enum TuneKind { TUNE_TREE = 0, TUNE_POPC = 1, TUNE_TC = 2, TUNE_TREE_TC = 3, TUNE_RETRIEVE = 4 };
struct TuneCfg {
    int a;   // TREE: threads per block; POPC / TC / TREE_TC: database splits
    int b;   // TREE: resident blocks per SM; TC / TREE_TC: database rows widened
             // in the kernel (1) or beforehand into scratch (2), 0 = automatic;
             // RETRIEVE: a = engine (1-3), b = engine 1's resident blocks per SM
};
bool tune_lookup(TuneKind kind, int64_t n, int64_t nq, int k, TuneCfg *cfg);
void tune_store(TuneKind kind, int64_t n, int64_t nq, int k, const TuneCfg &cfg);

// Launchers implemented in the kernel files (stream-ordered, no sync unless noted).
// The *_cfg variants take an explicit launch shape (NULL: table or heuristic).
int launch_dt_search_cfg(const dt_index *ix, const uint64_t *q, int64_t nq, int k, uint32_t *idx,
                         float *score, uint16_t *ab, dt_stats *stats, cudaStream_t s,
                         const TuneCfg *cfg, const uint32_t *seeds, int n_seed);
int launch_dt_search_seeded(const dt_index *ix, const uint64_t *q, int64_t nq, int k,
                            const uint32_t *seeds, int n_seed, uint32_t *idx, float *score,
                            uint16_t *ab, dt_stats *stats, cudaStream_t s);
int launch_bf_popc_cfg(const uint64_t *db, int64_t n, const uint64_t *q, int64_t nq, int k,
                       uint32_t *idx, float *score, uint16_t *ab, cudaStream_t s,
                       const TuneCfg *cfg);
int launch_bf_tc_cfg(const uint64_t *db, int64_t n, const uint64_t *q, int64_t nq, int k,
                     uint32_t *idx, float *score, uint16_t *ab, cudaStream_t s,
                     const TuneCfg *cfg);
int pick_bf_splits(int64_t row_blocks, int64_t tiles, int concurrent);
// Merge per-split sorted top-k lists partial[split][q][k] into idx/score/(A,B).
int launch_merge_partials(const uint64_t *partial, int n_split, const uint64_t *db, int64_t n,
                          const uint64_t *q, int64_t nq, int k, uint32_t *idx, float *score,
                          uint16_t *ab, cudaStream_t s);
int launch_bf_tc(const uint64_t *db, int64_t n, const uint64_t *q, int64_t nq, int k,
                 uint32_t *idx, float *score, uint16_t *ab, cudaStream_t s);
int take_tc_error(bool *raised);
int take_bf_error(bool *raised);   // read and clear the brute-force timeout flag
void set_drop_copy(bool on);       // test hook of the popcount kernel (missing tile copy)
int launch_bf_popc_noalloc(const uint64_t *db, int64_t n, const uint64_t *q, int64_t nq, int k,
                           uint32_t *idx, float *score, uint16_t *ab, cudaStream_t s);
int launch_bf_popc(const uint64_t *db, int64_t n, const uint64_t *q, int64_t nq, int k,
                   uint32_t *idx, float *score, uint16_t *ab, cudaStream_t s);
int build_tree(const uint64_t *db, int64_t n, int leaf_size, int use_and, int fused_cap,
               cudaStream_t s, dt_index *ix);
// A node to split with all of its descendants (tree construction, §4.1).
struct BuildRoot {
    int32_t id, begin, count, level;
};
int grow_forest(const uint64_t *db, uint32_t *perm, int64_t n_rows, const std::vector<BuildRoot> &roots,
                int leaf_size, int use_and, int fused_cap, cudaStream_t s, Grow &g_or, Grow &g_and,
                std::vector<NodeRec> &recs, int64_t *n_leaves, int32_t *depth);
int insert_tree(dt_index *ix, const uint64_t *d_new, int64_t m, cudaStream_t s);
int fill_index_rows(const uint64_t *db, dt_index *ix, cudaStream_t s);
// Rows of a scan tile of the batched tree search (= the tensor-core tile N).
constexpr int kScanTileRows = 128;
// Tile images of n tree-ordered rows: *tile_or [ceil(n/128)][64] and
// *kmask [ceil(n/128)], both cudaMalloc'ed here (the caller owns them).
int make_tile_images(const uint64_t *db_tree, int64_t n, uint64_t **tile_or, uint32_t **kmask,
                     cudaStream_t s);
// Batched tree search (dt_search.cu): all queries' descents, then the
// tile-level bound pass and scan on the tensor cores.
int launch_dt_search_batched(const dt_index *ix, const uint64_t *q, int64_t nq, int k,
                             const uint32_t *seeds, int n_seed, uint32_t *idx, float *score,
                             uint16_t *ab, dt_stats *stats, cudaStream_t s);
// The tensor-core passes of the batched tree search (bf_tc.cu).  Queries
// sit in slots (slot i < nq holds query slot_q[i]; slot_q has
// n_mtiles * 128 entries, -1 past nq), each with a key cap cap_slot[slot]
// that is >= its exact k-th result's key (0xFFFFFFFF: none).  Pass 1 bounds
// every (pair of 128-slot tiles, scan tile) by the tile images and marks
// the scan tiles some query of the pair may need; pass 2 scans those
// tiles, skipping K chunks the tile has no bit in, into per-split sorted
// lists partial[split][slot][k] of (key, original index).  *need (host
// copy, n_mpairs x need_words words) is filled when need_host is non-null.
// dt_keep_widened: build (on) or release (off) ix->scan_exp / scan_side.
int index_keep_widened(dt_index *ix, bool on, cudaStream_t s);
int launch_tree_tc(const dt_index *ix, const uint64_t *q, int64_t nq, const int32_t *slot_q,
                   const uint32_t *cap_slot, int n_mtiles, int k, Scratch &scratch, cudaStream_t s,
                   uint64_t **partial_out, int *n_split_out, std::vector<uint32_t> *need_host,
                   int64_t *need_words_out);
int launch_quicci(const float *d_vertices, int64_t n_vertices, const int32_t *d_triangles,
                  int64_t n_triangles, const float *d_points, const float *d_normals,
                  int64_t n_points, float support_radius, int modified, uint64_t *d_out,
                  cudaStream_t s);
int launch_dt_search(const dt_index *ix, const uint64_t *q, int64_t nq, int k, uint32_t *idx,
                     float *score, uint16_t *ab, dt_stats *stats, cudaStream_t s);
// cfg (nullable): the engine (a, used when engine is 0) and engine 1's
// resident blocks per SM (b); NULL: the tuning table, else defaults.
int launch_retrieve(const dt_index *ix, const uint32_t *object_of, int n_objects,
                    const uint64_t *qdesc, const int64_t *qoffsets, int nq, int64_t total,
                    int threshold, uint64_t seed, uint32_t *votes, int32_t *winner,
                    int64_t *consumed, int engine, cudaStream_t s, const TuneCfg *cfg = nullptr);
// Work unit of the tensor-core scan in list mode: the query tiles a_tile0
// and a_tile1 (TM rows each, the first nvalid0 / nvalid1 of them real;
// a_tile1 < 0: none) against database rows [row0, row1).  Results go to
// partial[a_tile * TM + row][k].
struct TcUnit {
    int64_t row0, row1;
    int32_t a_tile0, a_tile1, nvalid0, nvalid1;
    int64_t out_base;    // added to the slot: results go to partial[out_base + slot][k]
};
// Tensor-core scan over a unit table built on the device: *n_units units
// covering *n_tiles query tiles (at most max_tiles); the row r of tile t is
// query slot_q[t * TM + r] (negative = padding).  Rows are reported through
// idx_map.  For k = 1 the slot's entry is merged with an atomic minimum
// (partial must start at all ones, as always).
int launch_tc_units(const uint64_t *db, int64_t n, const uint32_t *idx_map, const uint64_t *q,
                    const int32_t *slot_q, const TcUnit *units, const int64_t *n_units,
                    const int64_t *n_tiles, int64_t max_tiles, int k, uint64_t *partial,
                    cudaStream_t s);
constexpr int kTcTileM = 128;
// Queries -> pre-widened tensor-core tiles a_exp [ceil(nq/128)][32 chunks][16 KB]
// and |q| (qpop [ceil(nq/128) * 128]); both device buffers of the caller.
int launch_widen_queries(const uint64_t *q, int64_t nq, unsigned char *a_exp, uint32_t *qpop,
                         cudaStream_t s);
size_t tc_tile_bytes();      // bytes of one pre-widened 128-query tile
// Tensor-core scan over a unit table whose query tiles are already widened
// (a_exp, qpop as above); *n_units units, at most max_units.
int launch_tc_units_pre(const uint64_t *db, int64_t n, const uint32_t *idx_map,
                        const unsigned char *a_exp, const uint32_t *qpop, const TcUnit *units,
                        const int64_t *n_units, int64_t max_units, int k, uint64_t *partial,
                        cudaStream_t s);
// Exact top-1 of each query over db on the tensor cores; reported indices go
// through idx_map when given (ties are broken on the reported index).
int launch_tc_top1(const uint64_t *db, int64_t n, const uint32_t *idx_map, const uint64_t *q,
                   int64_t nq, uint32_t *nn, cudaStream_t s);
}  // namespace dtk
