// dt_search.cu — Dissimilarity Tree query (§4.2): persistent warps, one
// query at a time per warp, queries handed out by an atomic counter so that
// cheap and expensive queries balance across the GPU.
#include <algorithm>

#include "dt_internal.cuh"
#include "dt_traverse.cuh"
#include "sort_util.cuh"

namespace dtk {
namespace {


struct SearchCtl {
    unsigned long long next;      // next query to hand out
    unsigned long long stats[4];  // nodes, leaves, descs, bounds
    unsigned int error;           // 1 = stack overflow
};

template <bool USE_AND>
__device__ __forceinline__ void
dt_search_body(TreeView tv, const uint32_t *__restrict__ iperm, const uint64_t *__restrict__ qs,
               int64_t nq, int k, const uint32_t *__restrict__ seeds, int n_seed, int64_t n_db,
               uint64_t *__restrict__ stacks, int stack_cap, SearchCtl *ctl,
               uint32_t *__restrict__ idx, float *__restrict__ score, uint16_t *__restrict__ ab)
{
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint64_t *stack = stacks + gw * stack_cap;
    TraverseStats st{0, 0, 0, 0};
    for (;;) {
        unsigned long long qi = 0;
        if (lane == 0) qi = atomicAdd(&ctl->next, 1ull);
        qi = __shfl_sync(0xffffffffu, qi, 0);
        if (qi >= (unsigned long long)nq) break;
        const uint4 qv = __ldg(reinterpret_cast<const uint4 *>(qs + (int64_t)qi * kWords) + lane);
        const QueryWeights w = query_weights(warp_sum(popc4(qv)));
        uint64_t slot = kEmpty;
        uint32_t cap = ~0u;
        if (seeds) {   // warm start: exact keys of the caller's candidates
            uint64_t seeded = kEmpty;
            for (int j = 0; j < n_seed; ++j) {
                const uint32_t c = __ldg(seeds + (int64_t)qi * n_seed + j);
                if ((int64_t)c >= n_db) continue;          // 0xFFFFFFFF or out of range: none
                const uint32_t pos = __ldg(iperm + c);
                const uint4 t = ldg16(tv.db_tree + (int64_t)pos * kWords, lane);
                const uint32_t r = warp_sum(popc_and4(qv, t) | (popc4(t) << 16));
                const uint64_t v = pack(pair_key(w, r & 0xffffu, r >> 16), c);
                // a candidate listed twice must count once
                if (!__any_sync(0xffffffffu, seeded == v))
                    warp_list_merge(seeded, lane == 0 ? v : kEmpty, k, lane);
            }
            cap = (uint32_t)(shfl_u64(seeded, k - 1) >> 32);
        }
        if (!warp_tree_search<USE_AND>(tv, qv, w, k, stack, stack_cap, lane, slot, st, cap)) {
            if (lane == 0) atomicOr(&ctl->error, 1u);
        }
        // outputs: lane j < k writes result j
        const int64_t o = (int64_t)qi * k + lane;
        uint32_t ov = 0, tp = 0;
        const bool have = slot != kEmpty;
        if (ab) {   // (A, B) of each result: re-read its descriptor (k rows)
            for (int j = 0; j < k; ++j) {
                uint64_t v = shfl_u64(slot, j);
                if (v == kEmpty) break;
                const uint32_t pos = __ldg(iperm + (uint32_t)v);
                const uint4 t = ldg16(tv.db_tree + (int64_t)pos * kWords, lane);
                uint32_t r = warp_sum(popc_and4(qv, t) | (popc4(t) << 16));
                if (lane == j) { ov = r & 0xffffu; tp = r >> 16; }
            }
        }
        if (lane < k) {
            if (have) {
                idx[o] = (uint32_t)slot;
                score[o] = key_score(w, (uint32_t)(slot >> 32));
                if (ab) { ab[2 * o] = (uint16_t)(w.pop - ov); ab[2 * o + 1] = (uint16_t)(tp - ov); }
            } else {
                idx[o] = 0xFFFFFFFFu;
                score[o] = __int_as_float(0x7f800000);
                if (ab) { ab[2 * o] = 0xFFFF; ab[2 * o + 1] = 0xFFFF; }
            }
        }
    }
    if (lane == 0) {
        atomicAdd(&ctl->stats[0], st.nodes);
        atomicAdd(&ctl->stats[1], st.leaves);
        atomicAdd(&ctl->stats[2], st.descs);
        atomicAdd(&ctl->stats[3], st.bounds);
    }
}

#define DT_SEARCH_PARAMS                                                                     \
    TreeView tv, const uint32_t *__restrict__ iperm, const uint64_t *__restrict__ qs, int64_t nq, \
        int k, const uint32_t *__restrict__ seeds, int n_seed, int64_t n_db,                   \
        uint64_t *__restrict__ stacks, int stack_cap, SearchCtl *ctl, uint32_t *__restrict__ idx, \
        float *__restrict__ score, uint16_t *__restrict__ ab
#define DT_SEARCH_ARGS tv, iperm, qs, nq, k, seeds, n_seed, n_db, stacks, stack_cap, ctl, idx, score, ab

template <bool USE_AND, int NT>
__global__ void __launch_bounds__(NT) dt_search_kernel(DT_SEARCH_PARAMS)
{
    dt_search_body<USE_AND>(DT_SEARCH_ARGS);
}

// Registers capped so that 1024 threads fit per SM (more queries in flight,
// a few spills); used when more resident blocks are asked for than the
// uncapped kernel allows.
template <bool USE_AND, int NT>
__global__ void __launch_bounds__(NT, 1024 / NT) dt_search_kernel_tight(DT_SEARCH_PARAMS)
{
    dt_search_body<USE_AND>(DT_SEARCH_ARGS);
}

// ---------------------------------------------------------------------------
// Batched search (large batches).  A subtree may be skipped for a query only
// when its bound exceeds the query's k-th result (§4.2); on the GPU whole
// tiles of 256 queries share each scan of the tree-ordered database, so the
// same rule is applied per (tile of queries, tile of 128 tree-ordered rows):
//   1. each query descends greedily (the child with the smaller bound,
//      the similar one on ties) to one leaf and scans it: that leaf's k-th
//      key — or, with a warm start, the k-th of the leaf and the caller's
//      candidates — is a cap >= the query's exact k-th key, and the leaf's
//      position orders the queries so that neighbouring queries share
//      subtrees;
//   2. the queries are sorted by that position into slots (128 per tile);
//   3. the tensor cores bound every (query, scan tile) by the tile's OR
//      image and mark the scan tiles that some query of a tile pair may
//      need (bound <= cap: equality is kept, as in the per-query search);
//   4. the marked tiles are scanned exactly on the tensor cores, skipping
//      the 128-bit K chunks in which the tile's image has no bit (they add
//      nothing to any overlap); keys above the cap are not kept;
//   5. each query merges its per-split lists.
// Every exact top-k result has a key <= cap, so its tile's bound is <= cap
// and the tile is scanned: the result equals the per-query search's.
// ---------------------------------------------------------------------------

__global__ void descend_kernel(TreeView tv, const uint32_t *__restrict__ iperm,
                               const uint64_t *__restrict__ qs, int64_t nq, int k,
                               const uint32_t *__restrict__ seeds, int n_seed, int64_t n_db,
                               uint32_t *__restrict__ cap, uint32_t *__restrict__ pos,
                               uint32_t *__restrict__ ids, unsigned long long *__restrict__ stats)
{
    const int lane = threadIdx.x & 31;
    int64_t qi = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t stride = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long nodes = 0, bounds = 0, descs = 0;
    for (; qi < nq; qi += stride) {
        const uint4 qv = __ldg(reinterpret_cast<const uint4 *>(qs + qi * kWords) + lane);
        const QueryWeights w = query_weights(warp_sum(popc4(qv)));
        int nd = 0;
        NodeRec rec = tv.node[0];
        ++nodes;
        while (rec.first_child >= 0) {
            const int sc = rec.first_child, dc = sc + 1;
            const uint4 os = ldg16(tv.or_img + (int64_t)sc * kWords, lane);
            const uint4 od = ldg16(tv.or_img + (int64_t)dc * kWords, lane);
            const uint32_t ab = warp_sum(popc_andnot4(qv, os) | (popc_andnot4(qv, od) << 16));
            bounds += 2;
            nd = (ab & 0xffffu) <= (ab >> 16) ? sc : dc;
            rec = tv.node[nd];
            ++nodes;
        }
        uint64_t slot = kEmpty;
        scan_leaf(tv, qv, w, rec.begin, rec.count, k, lane, slot);
        descs += (unsigned long long)rec.count;
        for (int j = 0; j < n_seed; ++j) {      // warm start: the caller's candidates
            const uint32_t c = __ldg(seeds + qi * n_seed + j);
            if ((int64_t)c >= n_db) continue;
            const uint32_t p = __ldg(iperm + c);
            const uint4 t = ldg16(tv.db_tree + (int64_t)p * kWords, lane);
            const uint32_t r = warp_sum(popc_and4(qv, t) | (popc4(t) << 16));
            const uint64_t v = pack(pair_key(w, r & 0xffffu, r >> 16), c);
            // a descriptor met twice (in the leaf and among the seeds, or
            // twice among the seeds) must count once
            if (!__any_sync(0xffffffffu, slot == v)) warp_list_merge(slot, lane == 0 ? v : kEmpty, k, lane);
        }
        const uint64_t kth = shfl_u64(slot, k - 1);
        if (lane == 0) {
            cap[qi] = (uint32_t)(kth >> 32);   // 0xFFFFFFFF: fewer than k candidates
            pos[qi] = (uint32_t)rec.begin;
            ids[qi] = (uint32_t)qi;
        }
    }
    if (lane == 0) {
        atomicAdd(&stats[0], nodes);
        atomicAdd(&stats[1], bounds);
        atomicAdd(&stats[2], descs);
    }
}

// Slot i holds query order[i]; padding slots up to n_slots get -1.
__global__ void slots_kernel(const uint32_t *__restrict__ order, const uint32_t *__restrict__ cap,
                             int64_t nq, int64_t n_slots, int32_t *__restrict__ slot_q,
                             uint32_t *__restrict__ cap_slot, int32_t *__restrict__ slot_of)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_slots) return;
    if (i < nq) {
        const uint32_t q = order[i];
        slot_q[i] = (int32_t)q;
        cap_slot[i] = cap[q];
        slot_of[q] = (int32_t)i;
    } else {
        slot_q[i] = -1;
        cap_slot[i] = 0u;
    }
}

// One warp per query: merge the per-split lists of its slot, then write idx,
// score and (A, B) (the result rows re-read through iperm).
__global__ void tree_merge_kernel(const uint64_t *__restrict__ partial, int n_split, int64_t nq,
                                  int k, const int32_t *__restrict__ slot_of, TreeView tv,
                                  const uint32_t *__restrict__ iperm, const uint64_t *__restrict__ qs,
                                  uint32_t *__restrict__ idx, float *__restrict__ score,
                                  uint16_t *__restrict__ ab)
{
    const int lane = threadIdx.x & 31;
    const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (q >= nq) return;
    const int64_t sl = slot_of[q];
    uint64_t slot = kEmpty;
    for (int sp = 0; sp < n_split; ++sp) {
        const uint64_t c = lane < k ? partial[((int64_t)sp * nq + sl) * k + lane] : kEmpty;
        warp_list_merge(slot, c, k, lane);
    }
    const uint4 qv = __ldg(reinterpret_cast<const uint4 *>(qs + q * kWords) + lane);
    const QueryWeights w = query_weights(warp_sum(popc4(qv)));
    uint32_t ov = 0, tp = 0;
    if (ab) {
        for (int j = 0; j < k; ++j) {
            const uint64_t v = shfl_u64(slot, j);
            if (v == kEmpty) break;
            const uint32_t p = __ldg(iperm + (uint32_t)v);
            const uint4 t = ldg16(tv.db_tree + (int64_t)p * kWords, lane);
            const uint32_t r = warp_sum(popc_and4(qv, t) | (popc4(t) << 16));
            if (lane == j) { ov = r & 0xffffu; tp = r >> 16; }
        }
    }
    if (lane < k) {
        const int64_t o = q * k + lane;
        if (slot != kEmpty) {
            idx[o] = (uint32_t)slot;
            score[o] = key_score(w, (uint32_t)(slot >> 32));
            if (ab) { ab[2 * o] = (uint16_t)(w.pop - ov); ab[2 * o + 1] = (uint16_t)(tp - ov); }
        } else {
            idx[o] = 0xFFFFFFFFu;
            score[o] = __int_as_float(0x7f800000);
            if (ab) { ab[2 * o] = 0xFFFF; ab[2 * o + 1] = 0xFFFF; }
        }
    }
}

}  // namespace

int launch_dt_search_batched(const dt_index *ix, const uint64_t *q, int64_t nq, int k,
                             const uint32_t *seeds, int n_seed, uint32_t *idx, float *score,
                             uint16_t *ab, dt_stats *stats, cudaStream_t s)
{
    TreeView tv{ix->node, ix->or_img, ix->and_img, ix->db_tree, ix->perm};
    const int n_mtiles = (int)((nq + kTcTileM - 1) / kTcTileM);
    const int64_t n_slots = (int64_t)n_mtiles * kTcTileM;
    Scratch scratch(s);
    uint32_t *cap = nullptr, *pos = nullptr, *ids = nullptr, *pos2 = nullptr, *ids2 = nullptr,
             *hist = nullptr, *cap_slot = nullptr;
    int32_t *slot_q = nullptr, *slot_of = nullptr;
    unsigned long long *dstats = nullptr;
    DT_CUDA_TRY(scratch.alloc(&cap, (size_t)nq * 4));
    DT_CUDA_TRY(scratch.alloc(&pos, (size_t)nq * 4));
    DT_CUDA_TRY(scratch.alloc(&ids, (size_t)nq * 4));
    DT_CUDA_TRY(scratch.alloc(&pos2, (size_t)nq * 4));
    DT_CUDA_TRY(scratch.alloc(&ids2, (size_t)nq * 4));
    DT_CUDA_TRY(scratch.alloc(&hist, (size_t)radix_tiles(nq) * 256 * 4));
    DT_CUDA_TRY(scratch.alloc(&slot_q, (size_t)n_slots * 4));
    DT_CUDA_TRY(scratch.alloc(&cap_slot, (size_t)n_slots * 4));
    DT_CUDA_TRY(scratch.alloc(&slot_of, (size_t)nq * 4));
    DT_CUDA_TRY(scratch.alloc(&dstats, 3 * sizeof(unsigned long long)));
    DT_CUDA_TRY(cudaMemsetAsync(dstats, 0, 3 * sizeof(unsigned long long), s));

    // 1. descents (a warp per query)
    const int64_t warps_needed = nq;
    const int64_t dblocks = std::max<int64_t>(1, std::min<int64_t>((warps_needed + 7) / 8, (int64_t)sm_count() * 32));
    descend_kernel<<<(unsigned)dblocks, 256, 0, s>>>(tv, ix->iperm, q, nq, k, seeds, seeds ? n_seed : 0,
                                                     ix->n, cap, pos, ids, dstats);
    DT_CUDA_TRY(cudaGetLastError());
    // 2. queries in the order of their leaves (stable: ties keep query order)
    int bits = 1;
    while (bits < 32 && (ix->n >> bits) != 0) ++bits;
    DT_CUDA_TRY(radix_sort_pairs(&pos, &ids, &pos2, &ids2, nq, bits, hist, s));
    slots_kernel<<<(unsigned)((n_slots + 255) / 256), 256, 0, s>>>(ids, cap, nq, n_slots, slot_q,
                                                                   cap_slot, slot_of);
    DT_CUDA_TRY(cudaGetLastError());
    // 3, 4. bound pass and scan on the tensor cores
    uint64_t *partial = nullptr;
    int n_split = 0;
    int64_t need_words = 0;
    std::vector<uint32_t> need_host;
    if (int r = launch_tree_tc(ix, q, nq, slot_q, cap_slot, n_mtiles, k, scratch, s, &partial,
                               &n_split, stats ? &need_host : nullptr, &need_words))
        return r;
    // 5. per-query merge
    tree_merge_kernel<<<(unsigned)((nq + 7) / 8), 256, 0, s>>>(partial, n_split, nq, k, slot_of, tv,
                                                               ix->iperm, q, idx, score, ab);
    DT_CUDA_TRY(cudaGetLastError());
    if (stats) {
        unsigned long long h[3];
        DT_CUDA_TRY(cudaMemcpyAsync(h, dstats, sizeof(h), cudaMemcpyDeviceToHost, s));
        DT_CUDA_TRY(cudaStreamSynchronize(s));
        // scanned pairs: every valid query of a tile pair against every row
        // of each scan tile marked for the pair
        const int64_t n_tt = (ix->n + kScanTileRows - 1) / kScanTileRows;
        int64_t pairs = 0;
        const int64_t n_mpairs = (n_mtiles + 1) / 2;
        for (int64_t mp = 0; mp < n_mpairs; ++mp) {
            const int64_t rows_q = std::min<int64_t>(2 * kTcTileM, nq - mp * 2 * kTcTileM);
            int64_t rows_db = 0;
            for (int64_t wd = 0; wd < need_words; ++wd) {
                uint32_t m = need_host[(size_t)(mp * need_words + wd)];
                while (m) {
                    const int64_t t = wd * 32 + __builtin_ctz(m);
                    m &= m - 1;
                    rows_db += std::min<int64_t>(kScanTileRows, ix->n - t * kScanTileRows);
                }
            }
            pairs += rows_q * rows_db;
        }
        stats->nodes_visited = (int64_t)h[0];
        stats->leaves_visited = nq;
        stats->descs_scanned = (int64_t)h[2] + pairs;
        stats->bounds_evaluated = (int64_t)h[1] + nq * n_tt;
    }
    return DT_OK;
}

int launch_dt_search_cfg(const dt_index *ix, const uint64_t *q, int64_t nq, int k, uint32_t *idx,
                         float *score, uint16_t *ab, dt_stats *stats, cudaStream_t s,
                         const TuneCfg *cfg, const uint32_t *seeds, int n_seed)
{
    TreeView tv{ix->node, ix->or_img, ix->and_img, ix->db_tree, ix->perm};
    // default: 256 threads, 4 resident blocks per SM (the register-capped
    // kernel; measured ~9% faster than 3 uncapped blocks at 10M x 10k)
    TuneCfg c{256, 4};
    if (cfg) c = *cfg;
    else tune_lookup(TUNE_TREE, ix->n, nq, k, &c);
    const int nt = c.a == 128 ? 128 : 256;
    using Kern = void (*)(TreeView, const uint32_t *, const uint64_t *, int64_t, int,
                          const uint32_t *, int, int64_t, uint64_t *, int, SearchCtl *, uint32_t *,
                          float *, uint16_t *);
    auto pick = [&](bool tight) -> Kern {
        if (ix->use_and) {
            if (nt == 128) return tight ? dt_search_kernel_tight<true, 128> : dt_search_kernel<true, 128>;
            return tight ? dt_search_kernel_tight<true, 256> : dt_search_kernel<true, 256>;
        }
        if (nt == 128) return tight ? dt_search_kernel_tight<false, 128> : dt_search_kernel<false, 128>;
        return tight ? dt_search_kernel_tight<false, 256> : dt_search_kernel<false, 256>;
    };
    Kern kern = pick(false);
    int per_sm = 0;
    DT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, 0));
    per_sm = std::max(1, per_sm);
    if (c.b > per_sm) {                             // more in flight than the full kernel fits
        kern = pick(true);
        DT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, 0));
        per_sm = std::max(1, per_sm);
    }
    if (c.b > 0) per_sm = std::min(per_sm, c.b);   // fewer queries in flight than fit
    int64_t blocks = per_sm * (int64_t)sm_count();
    blocks = std::min<int64_t>(blocks, (nq + nt / 32 - 1) / (nt / 32));
    blocks = std::max<int64_t>(blocks, 1);
    const int stack_cap = ix->depth + 2;
    const int64_t nwarps = blocks * (nt / 32);

    Scratch scratch(s);
    SearchCtl *ctl = nullptr;
    uint64_t *stacks = nullptr;
    DT_CUDA_TRY(scratch.alloc(&ctl, sizeof(SearchCtl)));
    DT_CUDA_TRY(scratch.alloc(&stacks, (size_t)nwarps * stack_cap * 8));
    DT_CUDA_TRY(cudaMemsetAsync(ctl, 0, sizeof(SearchCtl), s));
    {
        KernelTimer timer("tree_warp", s);
        kern<<<(unsigned)blocks, nt, 0, s>>>(tv, ix->iperm, q, nq, k, seeds, n_seed, ix->n, stacks,
                                             stack_cap, ctl, idx, score, ab);
    }
    DT_CUDA_TRY(cudaGetLastError());
    int rc = DT_OK;
    if (stats) {
        SearchCtl h;
        DT_CUDA_TRY(cudaMemcpyAsync(&h, ctl, sizeof(h), cudaMemcpyDeviceToHost, s));
        DT_CUDA_TRY(cudaStreamSynchronize(s));
        stats->nodes_visited = (int64_t)h.stats[0];
        stats->leaves_visited = (int64_t)h.stats[1];
        stats->descs_scanned = (int64_t)h.stats[2];
        stats->bounds_evaluated = (int64_t)h.stats[3];
        if (h.error) {
            set_error("dt_search: traversal stack overflow");
            rc = DT_ECUDA;
        }
    }
    return rc;
}

int launch_dt_search(const dt_index *ix, const uint64_t *q, int64_t nq, int k, uint32_t *idx,
                     float *score, uint16_t *ab, dt_stats *stats, cudaStream_t s)
{
    return launch_dt_search_cfg(ix, q, nq, k, idx, score, ab, stats, s, nullptr, nullptr, 0);
}

int launch_dt_search_seeded(const dt_index *ix, const uint64_t *q, int64_t nq, int k,
                            const uint32_t *seeds, int n_seed, uint32_t *idx, float *score,
                            uint16_t *ab, dt_stats *stats, cudaStream_t s)
{
    return launch_dt_search_cfg(ix, q, nq, k, idx, score, ab, stats, s, nullptr, seeds, n_seed);
}

}  // namespace dtk
