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

template <bool USE_AND, int NT>
__global__ void __launch_bounds__(NT)
dt_search_kernel(TreeView tv, const uint32_t *__restrict__ iperm, const uint64_t *__restrict__ qs,
                 int64_t nq, int k, uint64_t *__restrict__ stacks, int stack_cap,
                 SearchCtl *ctl, uint32_t *__restrict__ idx, float *__restrict__ score,
                 uint16_t *__restrict__ ab)
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
        if (!warp_tree_search<USE_AND>(tv, qv, w, k, stack, stack_cap, lane, slot, st)) {
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

}  // namespace

int launch_dt_search_cfg(const dt_index *ix, const uint64_t *q, int64_t nq, int k, uint32_t *idx,
                         float *score, uint16_t *ab, dt_stats *stats, cudaStream_t s,
                         const TuneCfg *cfg)
{
    TreeView tv{ix->node, ix->or_img, ix->and_img, ix->db_tree, ix->perm};
    TuneCfg c{256, 0};
    if (cfg) c = *cfg;
    else tune_lookup(TUNE_TREE, ix->n, nq, k, &c);
    const int nt = c.a == 128 ? 128 : 256;
    auto kern = ix->use_and ? (nt == 128 ? dt_search_kernel<true, 128> : dt_search_kernel<true, 256>)
                            : (nt == 128 ? dt_search_kernel<false, 128> : dt_search_kernel<false, 256>);
    int per_sm = 0;
    DT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, 0));
    per_sm = std::max(1, per_sm);
    if (c.b > 0) per_sm = std::min(per_sm, c.b);   // fewer queries in flight than fit
    int64_t blocks = per_sm * (int64_t)sm_count();
    blocks = std::min<int64_t>(blocks, (nq + nt / 32 - 1) / (nt / 32));
    blocks = std::max<int64_t>(blocks, 1);
    const int stack_cap = ix->depth + 2;
    const int64_t nwarps = blocks * (nt / 32);

    SearchCtl *ctl = nullptr;
    uint64_t *stacks = nullptr;
    DT_CUDA_TRY(cudaMallocAsync((void **)&ctl, sizeof(SearchCtl), s));
    DT_CUDA_TRY(cudaMallocAsync((void **)&stacks, (size_t)nwarps * stack_cap * 8, s));
    DT_CUDA_TRY(cudaMemsetAsync(ctl, 0, sizeof(SearchCtl), s));
    kern<<<(unsigned)blocks, nt, 0, s>>>(tv, ix->iperm, q, nq, k, stacks, stack_cap, ctl, idx,
                                         score, ab);
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
    DT_CUDA_TRY(cudaFreeAsync(stacks, s));
    DT_CUDA_TRY(cudaFreeAsync(ctl, s));
    return rc;
}

int launch_dt_search(const dt_index *ix, const uint64_t *q, int64_t nq, int k, uint32_t *idx,
                     float *score, uint16_t *ab, dt_stats *stats, cudaStream_t s)
{
    return launch_dt_search_cfg(ix, q, nq, k, idx, score, ab, stats, s, nullptr);
}

}  // namespace dtk
