// votes.cu — partial-object retrieval by voting (§3).
//
// Query j's descriptors are drawn in a random order (Fisher-Yates from the
// last position, SplitMix64 seeded with the (j+1)-th output of
// SplitMix64(seed)); each drawn descriptor's nearest database descriptor
// (exact top-1 of Eq. 1, ties by lowest original index) votes for its
// object; with a threshold T the first object to reach T votes wins.
//
// Two engines find the nearest neighbours; both are exact, so both give the
// same votes:
//  * tree: every descriptor is one work item of a persistent launch (warps
//    take items from an atomic counter, a binary search over the CSR
//    offsets finds the item's query) traversing the Dissimilarity Tree as in
//    dt_search.  With T = 0 the vote is an atomic increment straight from
//    the traversal kernel; with T > 0 all neighbours are kept and one thread
//    per query replays the draw order.
//  * tensor: batches of descriptors are scanned against the index's
//    tree-ordered database on the tensor cores (bf_tc.cu, rows reported as
//    original indices).  With T = 0 all descriptors form one batch.  With
//    T > 0 the draws are taken in rounds — the next T, 2T, 4T ... drawn
//    descriptors of every undecided query — and a replay kernel advances
//    each query's vote count in draw order, so only the descriptors the
//    loop of §3 actually consumes (plus the rest of their round) are searched.
#include <algorithm>
#include <vector>

#include "block_util.cuh"
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

__device__ __forceinline__ uint64_t splitmix_next(uint64_t &s)
{
    uint64_t z = (s += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// ---------------------------------------------------------------- tree engine
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

// Query j's draw order into order[qoff[j] ..].
__global__ void draw_order_kernel(const int64_t *__restrict__ qoff, int nq, uint64_t seed,
                                  uint32_t *__restrict__ order)
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
}

// One thread per query: the vote loop of §3 over all draws (tree engine, T > 0).
__global__ void replay_kernel(const uint32_t *__restrict__ nn, const uint32_t *__restrict__ object_of,
                              int n_objects, const int64_t *__restrict__ qoff, int nq, int threshold,
                              const uint32_t *__restrict__ order, uint32_t *__restrict__ votes,
                              int32_t *__restrict__ winner, int64_t *__restrict__ consumed)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nq) return;
    const int64_t b = qoff[j], m = max((int64_t)0, qoff[j + 1] - b);
    const uint32_t *ord = order + b;
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

// -------------------------------------------------------------- tensor engine
// T = 0: one vote per descriptor from its neighbour.
__global__ void vote_all_kernel(const uint32_t *__restrict__ nn, int64_t total,
                                const uint32_t *__restrict__ object_of, int n_objects,
                                const int64_t *__restrict__ qoff, int nq, uint32_t *__restrict__ votes)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; i < total; i += stride) {
        const uint32_t t = nn[i];
        if (t == 0xFFFFFFFFu) continue;
        const uint32_t o = __ldg(object_of + t);
        if (o >= (uint32_t)n_objects) continue;
        atomicAdd(&votes[(int64_t)find_query(qoff, nq, i) * n_objects + o], 1u);
    }
}

struct RoundState {
    int64_t *used;       // draws consumed so far
    int32_t *done;       // 1 once decided or out of draws
    int64_t *take;       // draws in this round
    int64_t *slot;       // first batch slot of this round (exclusive scan of take)
    int64_t *total;      // [1] batch size of this round
};

// take_j = undecided ? min(C, m_j - used_j) : 0, then an exclusive scan in one block.
__global__ void round_plan_kernel(const int64_t *__restrict__ qoff, int nq, int64_t C, RoundState st)
{
    __shared__ uint32_t scan_tmp[33];
    __shared__ unsigned long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nq; base += blockDim.x) {
        const int j = base + threadIdx.x;
        int64_t t = 0;
        if (j < nq && !st.done[j]) t = min(C, (qoff[j + 1] - qoff[j]) - st.used[j]);
        if (j < nq) st.take[j] = t;
        uint32_t tot;
        const uint32_t ex = block_excl_scan((uint32_t)t, scan_tmp, &tot);
        if (j < nq) st.slot[j] = (int64_t)carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) st.total[0] = (int64_t)carry;
}

// Warp per query: copy this round's drawn descriptors into the batch.
__global__ void round_gather_kernel(const uint64_t *__restrict__ qdesc, const int64_t *__restrict__ qoff,
                                    int nq, const uint32_t *__restrict__ order, RoundState st,
                                    uint64_t *__restrict__ batch)
{
    const int lane = threadIdx.x & 31;
    const int j = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (j >= nq) return;
    const int64_t take = st.take[j], b = qoff[j], u = st.used[j], s0 = st.slot[j];
    for (int64_t i = 0; i < take; ++i) {
        const int64_t src = b + order[b + u + i];
        reinterpret_cast<uint4 *>(batch + (s0 + i) * kWords)[lane] =
            __ldg(reinterpret_cast<const uint4 *>(qdesc + src * kWords) + lane);
    }
}

// Thread per query: advance the vote loop through this round's draws.
__global__ void round_replay_kernel(const uint32_t *__restrict__ nn, const uint32_t *__restrict__ object_of,
                                    int n_objects, const int64_t *__restrict__ qoff, int nq,
                                    int threshold, RoundState st, uint32_t *__restrict__ votes,
                                    int32_t *__restrict__ winner)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nq || st.done[j]) return;
    const int64_t take = st.take[j], s0 = st.slot[j], m = qoff[j + 1] - qoff[j];
    uint32_t *v = votes + (int64_t)j * n_objects;
    int64_t used = st.used[j];
    for (int64_t i = 0; i < take; ++i) {
        const uint32_t t = nn[s0 + i];
        ++used;
        if (t == 0xFFFFFFFFu) continue;
        const uint32_t o = object_of[t];
        if (o >= (uint32_t)n_objects) continue;
        if (++v[o] == (uint32_t)threshold) {
            winner[j] = (int32_t)o;
            st.done[j] = 1;
            break;
        }
    }
    st.used[j] = used;
    if (used >= m) st.done[j] = 1;
}

// Queries that ran out of draws: most votes, lowest id; report draws used.
__global__ void round_finish_kernel(const uint32_t *__restrict__ votes, int n_objects, int nq,
                                    RoundState st, int32_t *__restrict__ winner,
                                    int64_t *__restrict__ consumed)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nq) return;
    if (winner[j] < 0) {
        const uint32_t *v = votes + (int64_t)j * n_objects;
        uint32_t best = 0;
        int32_t win = -1;
        for (int o = 0; o < n_objects; ++o)
            if (v[o] > best) { best = v[o]; win = o; }
        winner[j] = win;
    }
    if (consumed) consumed[j] = st.used[j];
}

int retrieve_tree(const dt_index *ix, const uint32_t *object_of, int n_objects, const uint64_t *qdesc,
                  const int64_t *qoffsets, int nq, int64_t total, int threshold, uint64_t seed,
                  uint32_t *votes, int32_t *winner, int64_t *consumed, int blocks_per_sm,
                  cudaStream_t s)
{
    TreeView tv{ix->node, ix->or_img, ix->and_img, ix->db_tree, ix->perm};
    const bool use_and = ix->use_and != 0;
    const int stack_cap = ix->depth + 2;
    Scratch scratch(s);
    uint32_t *nn = nullptr, *order = nullptr;
    if (threshold > 0) {
        DT_CUDA_TRY(scratch.alloc(&nn, (size_t)std::max<int64_t>(total, 1) * 4));
        DT_CUDA_TRY(scratch.alloc(&order, (size_t)std::max<int64_t>(total, 1) * 4));
    }
    auto k0 = use_and ? retrieve_nn_kernel<true, 0> : retrieve_nn_kernel<false, 0>;
    auto k1 = use_and ? retrieve_nn_kernel<true, 1> : retrieve_nn_kernel<false, 1>;
    auto kern = threshold > 0 ? k1 : k0;
    int per_sm = 0;
    DT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, VT, 0));
    if (blocks_per_sm > 0) per_sm = std::min(per_sm, blocks_per_sm);   // fewer descriptors in flight
    int64_t blocks = std::max(1, per_sm) * (int64_t)sm_count();
    blocks = std::max<int64_t>(1, std::min<int64_t>(blocks, (total + 7) / 8));
    const int64_t nwarps = blocks * (VT / 32);
    VoteCtl *ctl = nullptr;
    uint64_t *stacks = nullptr;
    DT_CUDA_TRY(scratch.alloc(&ctl, sizeof(VoteCtl)));
    DT_CUDA_TRY(scratch.alloc(&stacks, (size_t)nwarps * stack_cap * 8));
    DT_CUDA_TRY(cudaMemsetAsync(ctl, 0, sizeof(VoteCtl), s));
    kern<<<(unsigned)blocks, VT, 0, s>>>(tv, object_of, n_objects, qdesc, qoffsets, nq, stacks,
                                         stack_cap, ctl, votes, nn);
    DT_CUDA_TRY(cudaGetLastError());
    if (threshold > 0) {
        draw_order_kernel<<<(nq + 127) / 128, 128, 0, s>>>(qoffsets, nq, seed, order);
        replay_kernel<<<(nq + 127) / 128, 128, 0, s>>>(nn, object_of, n_objects, qoffsets, nq,
                                                      threshold, order, votes, winner, consumed);
    } else {
        winner_kernel<<<(nq + 7) / 8, 256, 0, s>>>(votes, n_objects, qoffsets, nq, winner, consumed);
    }
    DT_CUDA_TRY(cudaGetLastError());
    return DT_OK;
}

// Nearest database descriptor (original index) of each of m query
// descriptors: the tensor-core brute force over the tree-ordered rows, or
// the batched tree search (top-1).  Both break ties by lowest index.
int nearest(const dt_index *ix, const uint64_t *q, int64_t m, uint32_t *nn, bool tree,
            cudaStream_t s)
{
    if (!tree) return launch_tc_top1(ix->db_tree, ix->n, ix->perm, q, m, nn, s);
    Scratch scratch(s);
    float *score = nullptr;
    DT_CUDA_TRY(scratch.alloc(&score, (size_t)m * 4));
    return launch_dt_search_batched(ix, q, m, 1, nullptr, 0, nn, score, nullptr, nullptr, s);
}

// Engines 2 (tree = false) and 3 (tree = true): every query descriptor's
// nearest neighbour in one batched search (T = 0), or in rounds of draws.
int retrieve_batched(const dt_index *ix, const uint32_t *object_of, int n_objects,
                     const uint64_t *qdesc, const int64_t *qoffsets, int nq, int64_t total,
                     int threshold, uint64_t seed, uint32_t *votes, int32_t *winner,
                     int64_t *consumed, bool tree, cudaStream_t s)
{
    Scratch scratch(s);
    if (threshold == 0) {
        uint32_t *nn = nullptr;
        DT_CUDA_TRY(scratch.alloc(&nn, (size_t)std::max<int64_t>(total, 1) * 4));
        if (total > 0) {
            if (int r = nearest(ix, qdesc, total, nn, tree, s)) return r;
            vote_all_kernel<<<(unsigned)std::min<int64_t>((total + 255) / 256, 4096), 256, 0, s>>>(
                nn, total, object_of, n_objects, qoffsets, nq, votes);
        }
        winner_kernel<<<(nq + 7) / 8, 256, 0, s>>>(votes, n_objects, qoffsets, nq, winner, consumed);
        DT_CUDA_TRY(cudaGetLastError());
        return DT_OK;
    }
    // rounds of draws
    uint32_t *order = nullptr;
    RoundState st;
    DT_CUDA_TRY(scratch.alloc(&order, (size_t)std::max<int64_t>(total, 1) * 4));
    DT_CUDA_TRY(scratch.alloc(&st.used, (size_t)nq * 8));
    DT_CUDA_TRY(scratch.alloc(&st.done, (size_t)nq * 4));
    DT_CUDA_TRY(scratch.alloc(&st.take, (size_t)nq * 8));
    DT_CUDA_TRY(scratch.alloc(&st.slot, (size_t)nq * 8));
    DT_CUDA_TRY(scratch.alloc(&st.total, 8));
    DT_CUDA_TRY(cudaMemsetAsync(st.used, 0, (size_t)nq * 8, s));
    DT_CUDA_TRY(cudaMemsetAsync(st.done, 0, (size_t)nq * 4, s));
    DT_CUDA_TRY(cudaMemsetAsync(winner, 0xFF, (size_t)nq * 4, s));   // -1
    draw_order_kernel<<<(nq + 127) / 128, 128, 0, s>>>(qoffsets, nq, seed, order);
    DT_CUDA_TRY(cudaGetLastError());
    int rc = DT_OK;
    // A query needs at least T draws to reach T votes, so the first round
    // takes exactly T; later rounds double.
    int64_t C = std::max<int64_t>(1, (int64_t)threshold);
    for (;;) {
        round_plan_kernel<<<1, 1024, 0, s>>>(qoffsets, nq, C, st);
        int64_t batch_n = 0;
        cudaError_t e = cudaMemcpyAsync(&batch_n, st.total, 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            set_error(std::string("retrieve_objects round: ") + cudaGetErrorString(e));
            rc = DT_ECUDA;
            break;
        }
        if (batch_n == 0) break;
        Scratch round(s);                      // this round's batch, freed at its end
        uint64_t *batch = nullptr;
        uint32_t *nn = nullptr;
        if (round.alloc(&batch, (size_t)batch_n * 512) != cudaSuccess ||
            round.alloc(&nn, (size_t)batch_n * 4) != cudaSuccess) {
            set_error("retrieve_objects: batch allocation failed");
            rc = DT_ENOMEM;
            break;
        }
        round_gather_kernel<<<(nq + 7) / 8, 256, 0, s>>>(qdesc, qoffsets, nq, order, st, batch);
        rc = nearest(ix, batch, batch_n, nn, tree, s);
        if (rc == DT_OK)
            round_replay_kernel<<<(nq + 127) / 128, 128, 0, s>>>(nn, object_of, n_objects, qoffsets,
                                                                nq, threshold, st, votes, winner);
        if (rc != DT_OK) break;
        C *= 2;
    }
    if (rc == DT_OK)
        round_finish_kernel<<<(nq + 127) / 128, 128, 0, s>>>(votes, n_objects, nq, st, winner, consumed);
    DT_CUDA_TRY(cudaGetLastError());
    return rc;
}

}  // namespace

int launch_retrieve(const dt_index *ix, const uint32_t *object_of, int n_objects,
                    const uint64_t *qdesc, const int64_t *qoffsets, int nq, int64_t total,
                    int threshold, uint64_t seed, uint32_t *votes, int32_t *winner,
                    int64_t *consumed, int engine, cudaStream_t s, const TuneCfg *cfg)
{
    DT_CUDA_TRY(cudaMemsetAsync(votes, 0, (size_t)nq * n_objects * 4, s));
    // the autotuner's choice for this database size and kind of threshold
    TuneCfg c{0, 0};
    if (cfg) c = *cfg;
    else tune_lookup(TUNE_RETRIEVE, ix->n, threshold > 0 ? 2 : 1, 1, &c);
    // untuned: the batched search from 256 query descriptors, or on a large
    // index, where a warp walking most of the rows per descriptor is slow
    // whatever the batch (as in dt_search)
    if (engine == 0)
        engine = c.a >= 1 && c.a <= 3 ? c.a : (total >= 256 || ix->n >= (int64_t(1) << 17) ? 3 : 1);
    if (engine >= 2)
        return retrieve_batched(ix, object_of, n_objects, qdesc, qoffsets, nq, total, threshold,
                                seed, votes, winner, consumed, engine == 3, s);
    return retrieve_tree(ix, object_of, n_objects, qdesc, qoffsets, nq, total, threshold, seed, votes,
                         winner, consumed, c.b, s);
}

}  // namespace dtk
