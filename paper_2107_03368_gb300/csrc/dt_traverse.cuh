// dt_traverse.cuh — one warp searches the Dissimilarity Tree for one query.
//
// The paper's query (§4.2) is best-first with a priority queue on the CPU.
// Any visit order gives the same exact result as long as a subtree is
// skipped only when its bound is strictly greater than the current k-th
// result, so on the GPU a warp runs a depth-first branch-and-bound: at an
// inner node it bounds both children (two 512-byte OR images, one 16-byte
// load per lane each), descends into the nearer one and stacks the farther
// one; a popped entry is re-checked against the k-th result, which only
// improves meanwhile.  The stack holds at most one entry per level.
//
// A lane owns 16 bytes (128 bits) of every image, so each node or
// descriptor is one coalesced 512-byte warp load.  Leaves are contiguous
// runs of the tree-ordered database; 32 descriptors are reduced at once by a
// butterfly transpose-add (31 shuffles) that leaves descriptor j's overlap
// and popcount in lane j.
#pragma once

#include "dt_internal.cuh"

namespace dtk {

struct TreeView {
    const NodeRec *node;
    const uint64_t *or_img;
    const uint64_t *and_img;
    const uint64_t *db_tree;
    const uint32_t *perm;
};

struct TraverseStats {
    unsigned long long nodes, leaves, descs, bounds;
};

__device__ __forceinline__ uint32_t popc4(uint4 v)
{
    return __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
}

__device__ __forceinline__ uint32_t popc_andnot4(uint4 q, uint4 t)   // popc(q & ~t)
{
    return __popc(q.x & ~t.x) + __popc(q.y & ~t.y) + __popc(q.z & ~t.z) + __popc(q.w & ~t.w);
}

__device__ __forceinline__ uint32_t popc_and4(uint4 q, uint4 t)
{
    return __popc(q.x & t.x) + __popc(q.y & t.y) + __popc(q.z & t.z) + __popc(q.w & t.w);
}

__device__ __forceinline__ uint4 ldg16(const uint64_t *row, int lane)
{
    return __ldg(reinterpret_cast<const uint4 *>(row) + lane);
}

// Scan one leaf's descriptors [begin, begin+count) and merge them into the
// warp's top-k list.
__device__ __forceinline__ void scan_leaf(const TreeView &tv, uint4 qv, const QueryWeights &w,
                                          int begin, int count, int k, int lane, uint64_t &slot)
{
    for (int b0 = 0; b0 < count; b0 += 32) {
        const int m = min(32, count - b0);
        uint32_t v[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            v[j] = 0;
            if (j < m) {
                uint4 t = ldg16(tv.db_tree + (int64_t)(begin + b0 + j) * kWords, lane);
                v[j] = popc_and4(qv, t) | (popc4(t) << 16);   // overlap | |t| << 16
            }
        }
        // butterfly transpose-add: lane j ends with descriptor j's totals
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
#pragma unroll
            for (int j = 0; j < o; ++j) {
                const bool hi = lane & o;
                uint32_t send = hi ? v[j] : v[j + o];
                uint32_t keep = hi ? v[j + o] : v[j];
                v[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
        }
        uint64_t cand = kEmpty;
        if (lane < m) {
            const uint32_t ov = v[0] & 0xffffu, tp = v[0] >> 16;
            cand = pack(pair_key(w, ov, tp), __ldg(tv.perm + begin + b0 + lane));
        }
        warp_list_merge(slot, cand, k, lane);
    }
}

template <bool USE_AND>
__device__ __forceinline__ uint32_t node_bound(const TreeView &tv, int nd, uint4 qv,
                                               const QueryWeights &w, int lane)
{
    uint4 o = ldg16(tv.or_img + (int64_t)nd * kWords, lane);
    uint32_t a = warp_sum(popc_andnot4(qv, o));
    uint32_t b = 0;
    if (USE_AND) {
        uint4 n = ldg16(tv.and_img + (int64_t)nd * kWords, lane);
        b = warp_sum(popc_andnot4(n, qv));
    }
    return a * w.Z + b * w.P;
}

// Search one query; `slot` is the warp's sorted top-k list (must start
// kEmpty).  `stack` is this warp's private stack of depth+1 entries.
// `cap` is a key known to be >= the exact k-th result's key (the k-th
// smallest key of k database descriptors found beforehand, or ~0u): a
// subtree is skipped when its bound exceeds min(cap, current k-th key), so
// a good cap prunes from the first node on and the result stays exact.
// Returns false if the stack would overflow (cannot happen for a stack of
// depth+1 entries; checked anyway).
template <bool USE_AND>
__device__ __forceinline__ bool warp_tree_search(const TreeView &tv, uint4 qv,
                                                 const QueryWeights &w, int k, uint64_t *stack,
                                                 int stack_cap, int lane, uint64_t &slot,
                                                 TraverseStats &st, uint32_t cap = ~0u)
{
    int sp = 0;
    {
        uint32_t lb = node_bound<USE_AND>(tv, 0, qv, w, lane);
        st.bounds += 1;
        if (lane == 0) stack[0] = ((uint64_t)lb << 32) | 0u;
        sp = 1;
    }
    while (sp > 0) {
        --sp;
        // only lane 0 touches the stack; the entry is broadcast
        uint64_t e = shfl_u64(lane == 0 ? stack[sp] : 0ull, 0);
        uint32_t lb = (uint32_t)(e >> 32);
        int nd = (int)(uint32_t)e;
        uint32_t worst = min(cap, (uint32_t)(shfl_u64(slot, k - 1) >> 32));
        if (lb > worst) continue;
        for (;;) {
            const NodeRec rec = tv.node[nd];
            st.nodes += 1;
            if (rec.first_child < 0) {
                st.leaves += 1;
                st.descs += (unsigned long long)rec.count;
                scan_leaf(tv, qv, w, rec.begin, rec.count, k, lane, slot);
                break;
            }
            const int s = rec.first_child, d = s + 1;
            const uint4 os = ldg16(tv.or_img + (int64_t)s * kWords, lane);
            const uint4 od = ldg16(tv.or_img + (int64_t)d * kWords, lane);
            uint32_t ab = warp_sum(popc_andnot4(qv, os) | (popc_andnot4(qv, od) << 16));
            uint32_t lbs = (ab & 0xffffu) * w.Z, lbd = (ab >> 16) * w.Z;
            if (USE_AND) {
                const uint4 ns = ldg16(tv.and_img + (int64_t)s * kWords, lane);
                const uint4 nd2 = ldg16(tv.and_img + (int64_t)d * kWords, lane);
                uint32_t bb = warp_sum(popc_andnot4(ns, qv) | (popc_andnot4(nd2, qv) << 16));
                lbs += (bb & 0xffffu) * w.P;
                lbd += (bb >> 16) * w.P;
            }
            st.bounds += 2;
            worst = min(cap, (uint32_t)(shfl_u64(slot, k - 1) >> 32));
            const bool sim_first = lbs <= lbd;
            const int near = sim_first ? s : d, far = sim_first ? d : s;
            const uint32_t lbn = sim_first ? lbs : lbd, lbf = sim_first ? lbd : lbs;
            if (lbf <= worst) {
                if (sp >= stack_cap) return false;
                if (lane == 0) stack[sp] = ((uint64_t)lbf << 32) | (uint32_t)far;
                ++sp;
            }
            if (lbn > worst) break;
            nd = near;
        }
    }
    return true;
}

}  // namespace dtk
