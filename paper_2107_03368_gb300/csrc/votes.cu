// votes.cu — partial-object retrieval by voting (§3).
//
// Every descriptor of every partial query is one work item of a persistent
// launch (warps take items from an atomic counter; a binary search over the
// CSR offsets finds the item's query), so uneven queries of 500..10,000
// descriptors share one launch.  Each item's nearest database descriptor is
// found with the tree traversal of dt_search (k = 1).
//
// Threshold 0: every descriptor votes; the vote is an atomic increment of
// votes[query][object] straight from the traversal kernel, and a second
// kernel picks each query's winner.  Threshold T > 0: the nearest neighbours
// are kept, then one thread per query draws the query's descriptors in its
// Fisher-Yates / SplitMix64 order and replays the votes until an object
// reaches T.
#include <algorithm>

#include "dt_internal.cuh"
#include "dt_traverse.cuh"

namespace dtk {
namespace {

constexpr int VT = 256;

struct VoteCtl {
    unsigned long long next;
    unsigned int error;
};

__device__ __forceinline__ int find_query(const int64_t *__restrict__ off, int nq, int64_t i)
{
    int lo = 0, hi = nq - 1;          // largest j with off[j] <= i
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= i) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// mode 0: vote directly; mode 1: store the neighbour's original index.
template <bool USE_AND, int MODE>
__global__ void __launch_bounds__(VT)
retrieve_nn_kernel(TreeView tv, const uint32_t *__restrict__ object_of, int n_objects,
                   const uint64_t *__restrict__ qdesc, const int64_t *__restrict__ qoff, int nq,
                   uint64_t *__restrict__ stacks, int stack_cap, VoteCtl *ctl,
                   uint32_t *__restrict__ votes, uint32_t *__restrict__ nn_out)
{
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint64_t *stack = stacks + gw * stack_cap;
    const int64_t total = __ldg(qoff + nq);
    TraverseStats st{0, 0, 0, 0};
    for (;;) {
        unsigned long long it = 0;
        if (lane == 0) it = atomicAdd(&ctl->next, 1ull);
        it = __shfl_sync(0xffffffffu, it, 0);
        if ((int64_t)it >= total) break;
        const uint4 qv = __ldg(reinterpret_cast<const uint4 *>(qdesc + (int64_t)it * kWords) + lane);
        const QueryWeights w = query_weights(warp_sum(popc4(qv)));
        uint64_t slot = kEmpty;
        if (!warp_tree_search<USE_AND>(tv, qv, w, 1, stack, stack_cap, lane, slot, st))
            if (lane == 0) atomicOr(&ctl->error, 1u);
        if (lane == 0) {
            const uint32_t t = (uint32_t)slot;
            if (MODE == 0) {
                if (slot != kEmpty) {
                    const int j = find_query(qoff, nq, (int64_t)it);
                    const uint32_t o = __ldg(object_of + t);
                    if (o < (uint32_t)n_objects) atomicAdd(&votes[(int64_t)j * n_objects + o], 1u);
                }
            } else {
                nn_out[it] = slot != kEmpty ? t : 0xFFFFFFFFu;
            }
        }
    }
}

// Winner = most votes, lowest object id on ties, -1 without votes.
__global__ void winner_kernel(const uint32_t *__restrict__ votes, int n_objects,
                              const int64_t *__restrict__ qoff, int nq, int32_t *__restrict__ winner,
                              int64_t *__restrict__ consumed)
{
    const int lane = threadIdx.x & 31;
    const int j = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (j >= nq) return;
    uint64_t best = kEmpty;            // (~votes << 32 | object): min = most votes, lowest id
    const uint32_t *v = votes + (int64_t)j * n_objects;
    for (int o = lane; o < n_objects; o += 32) {
        uint32_t c = v[o];
        if (c) {
            uint64_t key = ((uint64_t)(~c) << 32) | (uint32_t)o;
            best = key < best ? key : best;
        }
    }
    best = warp_min_u64(best);
    if (lane == 0) {
        winner[j] = best == kEmpty ? -1 : (int32_t)(uint32_t)best;
        if (consumed) consumed[j] = qoff[j + 1] - qoff[j];
    }
}

__device__ __forceinline__ uint64_t splitmix_next(uint64_t &s)
{
    uint64_t z = (s += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// One thread per query: draw order (Fisher-Yates from the last position,
// SplitMix64 seeded with the (j+1)-th output of SplitMix64(seed)), then the
// vote replay of §3 up to the threshold.
__global__ void replay_kernel(const uint32_t *__restrict__ nn, const uint32_t *__restrict__ object_of,
                              int n_objects, const int64_t *__restrict__ qoff, int nq, int threshold,
                              uint64_t seed, uint32_t *__restrict__ order, uint32_t *__restrict__ votes,
                              int32_t *__restrict__ winner, int64_t *__restrict__ consumed)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nq) return;
    const int64_t b = qoff[j], m = max((int64_t)0, qoff[j + 1] - b);
    uint32_t *ord = order + b;
    uint64_t s0 = seed + (uint64_t)j * 0x9e3779b97f4a7c15ull;
    uint64_t state = splitmix_next(s0);
    for (int64_t i = 0; i < m; ++i) ord[i] = (uint32_t)i;
    for (int64_t i = m - 1; i > 0; --i) {
        const uint64_t r = splitmix_next(state) % (uint64_t)(i + 1);
        const uint32_t t = ord[i];
        ord[i] = ord[r];
        ord[r] = t;
    }
    uint32_t *v = votes + (int64_t)j * n_objects;
    int32_t win = -1;
    int64_t used = 0;
    for (int64_t i = 0; i < m; ++i) {
        const uint32_t t = nn[b + ord[i]];
        ++used;
        if (t == 0xFFFFFFFFu) continue;
        const uint32_t o = object_of[t];
        if (o >= (uint32_t)n_objects) continue;   // ids outside [0, n_objects) cast no vote
        const uint32_t c = ++v[o];
        if (c == (uint32_t)threshold) {
            win = (int32_t)o;
            break;
        }
    }
    if (win < 0) {
        uint32_t best = 0;
        for (int o = 0; o < n_objects; ++o)
            if (v[o] > best) { best = v[o]; win = o; }
    }
    winner[j] = win;
    if (consumed) consumed[j] = used;
}

}  // namespace

int launch_retrieve(const dt_index *ix, const uint32_t *object_of, int n_objects,
                    const uint64_t *qdesc, const int64_t *qoffsets, int nq, int threshold,
                    uint64_t seed, uint32_t *votes, int32_t *winner, int64_t *consumed,
                    cudaStream_t s)
{
    TreeView tv{ix->node, ix->or_img, ix->and_img, ix->db_tree, ix->perm};
    const bool use_and = ix->use_and != 0;
    DT_CUDA_TRY(cudaMemsetAsync(votes, 0, (size_t)nq * n_objects * 4, s));
    const int stack_cap = ix->depth + 2;

    int64_t total = -1;
    uint32_t *nn = nullptr, *order = nullptr;
    if (threshold > 0) {
        DT_CUDA_TRY(cudaMemcpyAsync(&total, qoffsets + nq, 8, cudaMemcpyDeviceToHost, s));
        DT_CUDA_TRY(cudaStreamSynchronize(s));
        if (total < 0) {
            set_error("retrieve_objects: negative descriptor total");
            return DT_EINVAL;
        }
        DT_CUDA_TRY(cudaMallocAsync((void **)&nn, (size_t)std::max<int64_t>(total, 1) * 4, s));
        DT_CUDA_TRY(cudaMallocAsync((void **)&order, (size_t)std::max<int64_t>(total, 1) * 4, s));
    }

    auto k0 = use_and ? retrieve_nn_kernel<true, 0> : retrieve_nn_kernel<false, 0>;
    auto k1 = use_and ? retrieve_nn_kernel<true, 1> : retrieve_nn_kernel<false, 1>;
    auto kern = threshold > 0 ? k1 : k0;
    int per_sm = 0;
    DT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, VT, 0));
    int64_t blocks = std::max(1, per_sm) * (int64_t)sm_count();
    if (total >= 0) blocks = std::max<int64_t>(1, std::min<int64_t>(blocks, (total + 7) / 8));
    const int64_t nwarps = blocks * (VT / 32);

    VoteCtl *ctl = nullptr;
    uint64_t *stacks = nullptr;
    DT_CUDA_TRY(cudaMallocAsync((void **)&ctl, sizeof(VoteCtl), s));
    DT_CUDA_TRY(cudaMallocAsync((void **)&stacks, (size_t)nwarps * stack_cap * 8, s));
    DT_CUDA_TRY(cudaMemsetAsync(ctl, 0, sizeof(VoteCtl), s));
    kern<<<(unsigned)blocks, VT, 0, s>>>(tv, object_of, n_objects, qdesc, qoffsets, nq, stacks,
                                         stack_cap, ctl, votes, nn);
    DT_CUDA_TRY(cudaGetLastError());
    if (threshold > 0) {
        replay_kernel<<<(nq + 127) / 128, 128, 0, s>>>(nn, object_of, n_objects, qoffsets, nq,
                                                      threshold, seed, order, votes, winner,
                                                      consumed);
    } else {
        winner_kernel<<<(nq + 7) / 8, 256, 0, s>>>(votes, n_objects, qoffsets, nq, winner, consumed);
    }
    DT_CUDA_TRY(cudaGetLastError());
    DT_CUDA_TRY(cudaFreeAsync(stacks, s));
    DT_CUDA_TRY(cudaFreeAsync(ctl, s));
    if (nn) DT_CUDA_TRY(cudaFreeAsync(nn, s));
    if (order) DT_CUDA_TRY(cudaFreeAsync(order, s));
    return DT_OK;
}

}  // namespace dtk
