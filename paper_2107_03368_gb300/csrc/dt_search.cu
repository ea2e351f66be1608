// dt_search.cu — Dissimilarity Tree query (§4.2): persistent warps, one
// query at a time per warp, queries handed out by an atomic counter so that
// cheap and expensive queries balance across the GPU.
#include <algorithm>

#include "dt_internal.cuh"
#include "dt_traverse.cuh"

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

}  // namespace

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
    kern<<<(unsigned)blocks, nt, 0, s>>>(tv, ix->iperm, q, nq, k, seeds, n_seed, ix->n, stacks,
                                         stack_cap, ctl, idx, score, ab);
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
