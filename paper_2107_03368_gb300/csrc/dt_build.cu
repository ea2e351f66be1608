// dt_build.cu — Dissimilarity Tree construction (§4.1) on the GPU.
//
// The split of a node with n descriptors: give bit b the key
// (popularity(b) << 12) | b, so keys order bits by ascending popularity with
// the lower bit first on ties — the position of b in the paper's bitOrder.
// The move loop of §4.1 has, after handling the bits up to key K, moved
// exactly the descriptors whose smallest set-bit key is <= K.  It stops at
// the first bit where ceil(n/2) have moved, so with minkey(d) = min over d's
// set bits of key(b):
//     K*  = the ceil(n/2)-th smallest minkey (descriptors with no set bit
//           never move; if fewer than ceil(n/2) can move, all of them do),
//     dissimilar = { d : minkey(d) <= K* },  similar = the rest,
// and a split that leaves a side empty falls back to cutting the node's list
// (ascending original index) at floor(n/2).  No 4096-entry sort per node is
// needed: one popularity histogram, one min per descriptor, one selection.
//
// Build schedule: level by level (breadth first).  Each level's nodes own
// contiguous segments of `perm` (tree position -> original index) holding
// their descriptors in ascending original index.
//   * nodes with at most fused_cap descriptors (and leaves): one CTA each,
//     everything in shared memory — histogram, minkeys, bitonic selection,
//     stable partition written back in place, OR / AND images;
//   * larger nodes: chunked multi-CTA kernels — global histogram and OR
//     images by atomics, a minkey pass that also histograms each
//     descriptor's argmin bit, a per-node selection over the 4096 sorted
//     bit keys (prefix sums of that histogram), a chunk-count / scan /
//     scatter stable partition.
// The host reads back one split size per node per level to number the next
// level (breadth first, similar child first) and never touches descriptors.
#include <algorithm>
#include <vector>

#include "block_util.cuh"
#include "dt_internal.cuh"

namespace dtk {
namespace {

constexpr int BT = 256;            // threads per build CTA
constexpr int kDefaultCap = 2048;  // largest node split by one CTA
constexpr int CHUNK = 4096;        // descriptors per chunk of a large node

struct NodeWork {
    int32_t id;     // global node id (breadth-first)
    int32_t begin;  // segment in perm
    int32_t count;
    int32_t slot;   // output slot in the level arrays
};

struct Chunk {
    int32_t slot;   // large-node slot
    int32_t begin;  // positions [begin, end) of perm
    int32_t end;
    int32_t node_begin;
};

__device__ __forceinline__ uint64_t bit_key(uint32_t count, int b)
{
    return ((uint64_t)count << 12) | (uint64_t)b;
}

// ---------------------------------------------------------------------------
// One CTA per node (count <= cap).  Leaves only get their images.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(BT)
small_node_kernel(const NodeWork *__restrict__ work, const uint64_t *__restrict__ db,
                  uint32_t *__restrict__ perm, uint64_t *__restrict__ or_img,
                  uint64_t *__restrict__ and_img, int leaf_size, int cap,
                  int32_t *__restrict__ n_sim_out)
{
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *counts = reinterpret_cast<uint32_t *>(smem);                 // [4096]
    unsigned long long *img_or = reinterpret_cast<unsigned long long *>(counts + kBits);  // [64]
    unsigned long long *img_and = img_or + kWords;                         // [64]
    uint64_t *mk = reinterpret_cast<uint64_t *>(img_and + kWords);         // [cap]
    uint64_t *sorted = mk + cap;                                           // [pow2 >= cap]
    uint32_t *seg = reinterpret_cast<uint32_t *>(sorted + cap);            // [cap] (cap is pow2)
    __shared__ uint32_t scan_tmp[33];
    __shared__ uint32_t s_misc[4];

    const NodeWork nw = work[blockIdx.x];
    const int cnt = nw.count, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const bool internal = cnt > leaf_size;

    for (int i = tid; i < cnt; i += BT) seg[i] = perm[nw.begin + i];
    if (internal)
        for (int b = tid; b < kBits; b += BT) counts[b] = 0;
    if (tid < kWords) {
        img_or[tid] = 0ull;
        img_and[tid] = ~0ull;
    }
    __syncthreads();

    // pass 1: images and bit popularity (16 bytes per lane, warp per descriptor)
    uint64_t o0 = 0, o1 = 0, a0 = ~0ull, a1 = ~0ull;
    for (int i = wid; i < cnt; i += BT / 32) {
        const uint4 v = reinterpret_cast<const uint4 *>(db + (int64_t)seg[i] * kWords)[lane];
        const uint64_t w0 = ((uint64_t)v.y << 32) | v.x, w1 = ((uint64_t)v.w << 32) | v.z;
        o0 |= w0; o1 |= w1; a0 &= w0; a1 &= w1;
        if (internal) {
            uint64_t x = w0;
            while (x) { atomicAdd(&counts[lane * 128 + __ffsll(x) - 1], 1u); x &= x - 1; }
            x = w1;
            while (x) { atomicAdd(&counts[lane * 128 + 64 + __ffsll(x) - 1], 1u); x &= x - 1; }
        }
    }
    atomicOr(&img_or[2 * lane], (unsigned long long)o0);
    atomicOr(&img_or[2 * lane + 1], (unsigned long long)o1);
    atomicAnd(&img_and[2 * lane], (unsigned long long)a0);
    atomicAnd(&img_and[2 * lane + 1], (unsigned long long)a1);
    __syncthreads();
    if (tid < kWords) {
        or_img[(int64_t)nw.id * kWords + tid] = img_or[tid];
        if (and_img) and_img[(int64_t)nw.id * kWords + tid] = img_and[tid];
    }
    if (!internal) {
        if (tid == 0) n_sim_out[nw.slot] = -1;
        return;
    }

    // pass 2: smallest set-bit key of every descriptor
    for (int i = wid; i < cnt; i += BT / 32) {
        const uint4 v = reinterpret_cast<const uint4 *>(db + (int64_t)seg[i] * kWords)[lane];
        const uint64_t w0 = ((uint64_t)v.y << 32) | v.x, w1 = ((uint64_t)v.w << 32) | v.z;
        uint64_t m = kEmpty, x = w0;
        while (x) {
            int b = lane * 128 + __ffsll(x) - 1;
            uint64_t key = bit_key(counts[b], b);
            m = key < m ? key : m;
            x &= x - 1;
        }
        x = w1;
        while (x) {
            int b = lane * 128 + 64 + __ffsll(x) - 1;
            uint64_t key = bit_key(counts[b], b);
            m = key < m ? key : m;
            x &= x - 1;
        }
        m = warp_min_u64(m);
        if (lane == 0) mk[i] = m;
    }
    __syncthreads();

    // selection of K*: sort a copy of the minkeys
    int p2 = 1;
    while (p2 < cnt) p2 <<= 1;
    for (int i = tid; i < p2; i += BT) sorted[i] = i < cnt ? mk[i] : kEmpty;
    __syncthreads();
    block_bitonic_sort(sorted, p2);
    uint32_t nf = 0;
    for (int i = tid; i < cnt; i += BT) nf += sorted[i] != kEmpty;
    const uint32_t n_finite = block_sum(nf, scan_tmp);
    const uint32_t half = (uint32_t)(cnt + 1) / 2;
    const uint64_t kstar = n_finite >= half ? sorted[half - 1]
                         : (n_finite > 0 ? sorted[n_finite - 1] : 0);
    uint32_t nd = 0;
    for (int i = tid; i < cnt; i += BT) nd += (n_finite > 0 && mk[i] <= kstar);
    const uint32_t n_dis_rule = block_sum(nd, scan_tmp);
    const bool degenerate = n_dis_rule == 0 || n_dis_rule == (uint32_t)cnt;
    const uint32_t n_dis = degenerate ? (uint32_t)(cnt - cnt / 2) : n_dis_rule;
    const uint32_t n_sim = (uint32_t)cnt - n_dis;

    // stable partition: similar first, then dissimilar, each in list order
    const int per = (cnt + BT - 1) / BT;
    const int i0 = tid * per, i1 = min(cnt, i0 + per);
    uint32_t mine = 0;
    for (int i = i0; i < i1; ++i)
        mine += degenerate ? (i >= cnt / 2) : (n_finite > 0 && mk[i] <= kstar);
    uint32_t tot;
    uint32_t rank_dis = block_excl_scan(mine, scan_tmp, &tot);
    // all reads of seg/mk are done before writes to perm (perm is global, seg is a copy)
    for (int i = i0; i < i1; ++i) {
        bool dis = degenerate ? (i >= cnt / 2) : (n_finite > 0 && mk[i] <= kstar);
        uint32_t dest = dis ? n_sim + rank_dis : (uint32_t)i - rank_dis;
        rank_dis += dis;
        if (dest < (uint32_t)cnt) perm[nw.begin + dest] = seg[i];
    }
    if (tid == 0) n_sim_out[nw.slot] = (int32_t)n_sim;
    (void)s_misc;
}

// ---------------------------------------------------------------------------
// Large nodes: chunked multi-CTA passes.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(BT)
large_count_kernel(const Chunk *__restrict__ chunks, const NodeWork *__restrict__ nodes,
                   const uint64_t *__restrict__ db, const uint32_t *__restrict__ perm,
                   uint32_t *__restrict__ gcounts, unsigned long long *__restrict__ or_img,
                   unsigned long long *__restrict__ and_img)
{
    __shared__ uint32_t counts[kBits];
    __shared__ unsigned long long s_or[kWords], s_and[kWords];
    const Chunk ch = chunks[blockIdx.x];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int b = tid; b < kBits; b += BT) counts[b] = 0;
    if (tid < kWords) { s_or[tid] = 0ull; s_and[tid] = ~0ull; }
    __syncthreads();
    uint64_t o0 = 0, o1 = 0, a0 = ~0ull, a1 = ~0ull;
    for (int p = ch.begin + wid; p < ch.end; p += BT / 32) {
        const uint4 v = reinterpret_cast<const uint4 *>(db + (int64_t)perm[p] * kWords)[lane];
        const uint64_t w0 = ((uint64_t)v.y << 32) | v.x, w1 = ((uint64_t)v.w << 32) | v.z;
        o0 |= w0; o1 |= w1; a0 &= w0; a1 &= w1;
        uint64_t x = w0;
        while (x) { atomicAdd(&counts[lane * 128 + __ffsll(x) - 1], 1u); x &= x - 1; }
        x = w1;
        while (x) { atomicAdd(&counts[lane * 128 + 64 + __ffsll(x) - 1], 1u); x &= x - 1; }
    }
    atomicOr(&s_or[2 * lane], (unsigned long long)o0);
    atomicOr(&s_or[2 * lane + 1], (unsigned long long)o1);
    atomicAnd(&s_and[2 * lane], (unsigned long long)a0);
    atomicAnd(&s_and[2 * lane + 1], (unsigned long long)a1);
    __syncthreads();
    uint32_t *gc = gcounts + (int64_t)ch.slot * kBits;
    for (int b = tid; b < kBits; b += BT)
        if (counts[b]) atomicAdd(&gc[b], counts[b]);
    const int64_t id = nodes[ch.slot].id;
    if (tid < kWords) {
        atomicOr(&or_img[id * kWords + tid], s_or[tid]);
        if (and_img) atomicAnd(&and_img[id * kWords + tid], s_and[tid]);
    }
}

__global__ void __launch_bounds__(BT)
large_minkey_kernel(const Chunk *__restrict__ chunks, const uint64_t *__restrict__ db,
                    const uint32_t *__restrict__ perm, const uint32_t *__restrict__ gcounts,
                    uint64_t *__restrict__ mk, uint32_t *__restrict__ ghist)
{
    __shared__ uint32_t counts[kBits];
    __shared__ uint32_t hist[kBits];
    const Chunk ch = chunks[blockIdx.x];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const uint32_t *gc = gcounts + (int64_t)ch.slot * kBits;
    for (int b = tid; b < kBits; b += BT) { counts[b] = gc[b]; hist[b] = 0; }
    __syncthreads();
    for (int p = ch.begin + wid; p < ch.end; p += BT / 32) {
        const uint4 v = reinterpret_cast<const uint4 *>(db + (int64_t)perm[p] * kWords)[lane];
        const uint64_t w0 = ((uint64_t)v.y << 32) | v.x, w1 = ((uint64_t)v.w << 32) | v.z;
        uint64_t m = kEmpty, x = w0;
        while (x) {
            int b = lane * 128 + __ffsll(x) - 1;
            uint64_t key = bit_key(counts[b], b);
            m = key < m ? key : m;
            x &= x - 1;
        }
        x = w1;
        while (x) {
            int b = lane * 128 + 64 + __ffsll(x) - 1;
            uint64_t key = bit_key(counts[b], b);
            m = key < m ? key : m;
            x &= x - 1;
        }
        m = warp_min_u64(m);
        if (lane == 0) {
            mk[p] = m;
            if (m != kEmpty) atomicAdd(&hist[(int)(m & 4095u)], 1u);
        }
    }
    __syncthreads();
    uint32_t *gh = ghist + (int64_t)ch.slot * kBits;
    for (int b = tid; b < kBits; b += BT)
        if (hist[b]) atomicAdd(&gh[b], hist[b]);
}

// One CTA (1024 threads) per large node: K* from the bit keys in bitOrder
// and the histogram of argmin bits.  Writes kstar, n_sim and the mode
// (0 = rule, 1 = positional fallback).
__global__ void __launch_bounds__(1024)
large_select_kernel(const NodeWork *__restrict__ nodes, const uint32_t *__restrict__ gcounts,
                    const uint32_t *__restrict__ ghist, uint64_t *__restrict__ kstar_out,
                    int32_t *__restrict__ mode_out, int32_t *__restrict__ n_sim_out)
{
    __shared__ uint64_t keys[kBits];
    __shared__ uint32_t scan_tmp[33];
    const int slot = blockIdx.x, tid = threadIdx.x;
    const NodeWork nw = nodes[slot];
    const uint32_t *gc = gcounts + (int64_t)slot * kBits;
    const uint32_t *gh = ghist + (int64_t)slot * kBits;
    for (int b = tid; b < kBits; b += blockDim.x) keys[b] = bit_key(gc[b], b);
    __syncthreads();
    block_bitonic_sort(keys, kBits);
    // inclusive prefix of hist in key order: 4 consecutive keys per thread
    uint32_t h[4], s = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) { h[j] = gh[keys[tid * 4 + j] & 4095u]; s += h[j]; }
    uint32_t total;
    uint32_t before = block_excl_scan(s, scan_tmp, &total);
    const uint32_t cnt = (uint32_t)nw.count, half = (cnt + 1) / 2;
    __shared__ uint64_t s_kstar;
    __shared__ uint32_t s_ndis;
    if (tid == 0) { s_kstar = 0; s_ndis = 0; }
    __syncthreads();
    uint32_t run = before;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        uint32_t prev = run;
        run += h[j];
        if (total >= half) {
            if (prev < half && run >= half) { s_kstar = keys[tid * 4 + j]; s_ndis = run; }
        } else if (total > 0) {
            if (h[j] > 0 && run == total) { s_kstar = keys[tid * 4 + j]; s_ndis = total; }
        }
    }
    __syncthreads();
    if (tid == 0) {
        uint32_t nd = s_ndis;
        bool degenerate = nd == 0 || nd == cnt;
        kstar_out[slot] = s_kstar;
        mode_out[slot] = degenerate ? 1 : 0;
        n_sim_out[nw.slot] = (int32_t)(degenerate ? cnt / 2 : cnt - nd);
    }
}

__device__ __forceinline__ bool goes_dissimilar(int mode, uint64_t key, uint64_t kstar, int pos,
                                                int node_begin, int node_count)
{
    return mode ? (pos - node_begin) >= node_count / 2 : (key != kEmpty && key <= kstar);
}

__global__ void __launch_bounds__(BT)
large_chunk_count_kernel(const Chunk *__restrict__ chunks, const NodeWork *__restrict__ nodes,
                         const uint64_t *__restrict__ mk, const uint64_t *__restrict__ kstar,
                         const int32_t *__restrict__ mode, uint32_t *__restrict__ chunk_dis)
{
    __shared__ uint32_t scan_tmp[33];
    const Chunk ch = chunks[blockIdx.x];
    const NodeWork nw = nodes[ch.slot];
    const int md = mode[ch.slot];
    const uint64_t ks = kstar[ch.slot];
    uint32_t c = 0;
    for (int p = ch.begin + threadIdx.x; p < ch.end; p += BT)
        c += goes_dissimilar(md, mk[p], ks, p, nw.begin, nw.count);
    uint32_t t = block_sum(c, scan_tmp);
    if (threadIdx.x == 0) chunk_dis[blockIdx.x] = t;
}

// Exclusive scan of chunk counts within each node (chunks of a node are
// consecutive; one thread per node walks them).
__global__ void large_chunk_scan_kernel(const int32_t *__restrict__ first_chunk, int n_large,
                                        const uint32_t *__restrict__ chunk_dis,
                                        uint32_t *__restrict__ chunk_off)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_large) return;
    uint32_t run = 0;
    for (int c = first_chunk[s]; c < first_chunk[s + 1]; ++c) {
        chunk_off[c] = run;
        run += chunk_dis[c];
    }
}

__global__ void __launch_bounds__(BT)
large_scatter_kernel(const Chunk *__restrict__ chunks, const NodeWork *__restrict__ nodes,
                     const uint64_t *__restrict__ mk, const uint64_t *__restrict__ kstar,
                     const int32_t *__restrict__ mode, const int32_t *__restrict__ n_sim_level,
                     const uint32_t *__restrict__ chunk_off, const uint32_t *__restrict__ perm,
                     uint32_t *__restrict__ tmp)
{
    __shared__ uint32_t scan_tmp[33];
    const Chunk ch = chunks[blockIdx.x];
    const NodeWork nw = nodes[ch.slot];
    const int md = mode[ch.slot];
    const uint64_t ks = kstar[ch.slot];
    const uint32_t n_sim = (uint32_t)n_sim_level[nw.slot];
    const uint32_t dis_before_chunk = chunk_off[blockIdx.x];
    const uint32_t sim_before_chunk = (uint32_t)(ch.begin - nw.begin) - dis_before_chunk;
    const int len = ch.end - ch.begin;
    const int per = (len + BT - 1) / BT;
    const int i0 = ch.begin + threadIdx.x * per, i1 = min(ch.end, i0 + per);
    uint32_t mine = 0;
    for (int p = i0; p < i1; ++p) mine += goes_dissimilar(md, mk[p], ks, p, nw.begin, nw.count);
    uint32_t tot;
    uint32_t rd = block_excl_scan(mine, scan_tmp, &tot);
    uint32_t rs = (uint32_t)(i0 - ch.begin) - rd;
    for (int p = i0; p < i1; ++p) {
        bool dis = goes_dissimilar(md, mk[p], ks, p, nw.begin, nw.count);
        uint32_t dest = dis ? n_sim + dis_before_chunk + rd : sim_before_chunk + rs;
        rd += dis;
        rs += !dis;
        if (dest < (uint32_t)nw.count) tmp[nw.begin + dest] = perm[p];
    }
}

__global__ void copy_back_kernel(const Chunk *__restrict__ chunks, const uint32_t *__restrict__ tmp,
                                 uint32_t *__restrict__ perm)
{
    const Chunk ch = chunks[blockIdx.x];
    for (int p = ch.begin + threadIdx.x; p < ch.end; p += blockDim.x) perm[p] = tmp[p];
}

// db_tree[pos] = db[perm[pos]]: one warp per 512-byte row.
__global__ void gather_rows_kernel(const uint64_t *__restrict__ db, const uint32_t *__restrict__ perm,
                                   int64_t n, uint64_t *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t stride = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (; r < n; r += stride)
        reinterpret_cast<uint4 *>(out + r * kWords)[lane] =
            reinterpret_cast<const uint4 *>(db + (int64_t)perm[r] * kWords)[lane];
}

__global__ void invert_kernel(const uint32_t *__restrict__ perm, int64_t n, uint32_t *__restrict__ iperm)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; i < n; i += stride) iperm[perm[i]] = (uint32_t)i;
}

__global__ void iota_kernel(uint32_t *p, int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; i < n; i += stride) p[i] = (uint32_t)i;
}


size_t small_smem_bytes(int cap)
{
    return kBits * 4 + 2 * kWords * 8 + (size_t)cap * 8 * 2 + (size_t)cap * 4;
}

}  // namespace

// Splits every root and, level by level, all of its descendants (§4.1).
// A root is a node whose descriptors occupy perm[begin, begin + count) in
// ascending original-index order; perm holds row numbers of `db`.  Children
// are numbered from recs.size() on, one level at a time, similar child
// first, and appended to recs; recs[root.id] gets the root's segment and
// first child.  Images of every processed node are written at its id in
// g_or / g_and (grown as needed, contents kept).  Counts the processed
// nodes that are leaves into *n_leaves and raises *depth to the deepest
// level reached.
int grow_forest(const uint64_t *db, uint32_t *perm, int64_t n_rows, const std::vector<BuildRoot> &roots,
                int leaf_size, int use_and, int fused_cap, cudaStream_t s, Grow &g_or, Grow &g_and,
                std::vector<NodeRec> &recs, int64_t *n_leaves, int32_t *depth)
{
    int cap = fused_cap > 0 ? fused_cap : kDefaultCap;
    int p2 = 1;
    while (p2 < cap) p2 <<= 1;
    cap = std::max(p2, 64);
    if (cap < leaf_size) {
        int c = 1;
        while (c < leaf_size) c <<= 1;
        cap = c;
    }
    const size_t ssmem = small_smem_bytes(cap);
    if (ssmem > 200 * 1024) {
        set_error("fused_cap too large for shared memory");
        return DT_EINVAL;
    }
    DT_CUDA_TRY(allow_smem((const void *)small_node_kernel, ssmem));

    int rc = DT_OK;
    uint32_t *tmp = nullptr;
    uint64_t *mk = nullptr;
    Grow g_work, g_chunks, g_counts, g_hist, g_kstar, g_mode, g_nsim, g_cdis, g_coff, g_first;
    std::vector<BuildRoot> lvl(roots);

    auto cleanup = [&]() {
        g_work.release(s); g_chunks.release(s); g_counts.release(s); g_hist.release(s);
        g_kstar.release(s); g_mode.release(s); g_nsim.release(s); g_cdis.release(s);
        g_coff.release(s); g_first.release(s);
        if (tmp) cudaFreeAsync(tmp, s);
        if (mk) cudaFreeAsync(mk, s);
    };
#define BUILD_TRY(expr)                 \
    do {                                \
        int r_ = (expr);                \
        if (r_ != DT_OK) {              \
            rc = r_;                    \
            goto fail;                  \
        }                               \
    } while (0)
#define BUILD_CUDA(expr)                                                             \
    do {                                                                             \
        cudaError_t e_ = (expr);                                                     \
        if (e_ != cudaSuccess) {                                                     \
            set_error(std::string(#expr) + ": " + cudaGetErrorString(e_));           \
            rc = e_ == cudaErrorMemoryAllocation ? DT_ENOMEM : DT_ECUDA;             \
            goto fail;                                                               \
        }                                                                            \
    } while (0)

    {
        BUILD_CUDA(dt_malloc_async((void **)&tmp, (size_t)n_rows * 4, s));
        BUILD_CUDA(dt_malloc_async((void **)&mk, (size_t)n_rows * 8, s));

        std::vector<NodeWork> small, large;
        std::vector<Chunk> chunks;
        std::vector<int32_t> first_chunk, n_sim;
        for (const BuildRoot &r : lvl) {
            NodeRec &rec = recs[(size_t)r.id];
            rec.first_child = -1;
            rec.begin = r.begin;
            rec.count = r.count;
            rec.level = r.level;
        }
        while (!lvl.empty()) {
            const int64_t m = (int64_t)lvl.size();
            const size_t n_ids = recs.size();
            BUILD_TRY(g_or.ensure(n_ids * kWords * 8, s));
            if (use_and) BUILD_TRY(g_and.ensure(n_ids * kWords * 8, s));
            small.clear();
            large.clear();
            chunks.clear();
            first_chunk.clear();
            for (int64_t i = 0; i < m; ++i) {
                const BuildRoot &r = lvl[(size_t)i];
                NodeWork w{r.id, r.begin, r.count, (int32_t)i};
                if (r.count <= cap || r.count <= leaf_size) {
                    small.push_back(w);
                } else {
                    first_chunk.push_back((int32_t)chunks.size());
                    const int32_t slot = (int32_t)large.size();
                    for (int32_t b = r.begin; b < r.begin + r.count; b += CHUNK)
                        chunks.push_back(Chunk{slot, b, std::min(b + CHUNK, r.begin + r.count), r.begin});
                    large.push_back(w);
                }
                if (r.count <= leaf_size) ++*n_leaves;
                *depth = std::max(*depth, r.level);
            }
            first_chunk.push_back((int32_t)chunks.size());
            BUILD_TRY(g_nsim.ensure((size_t)m * 4, s));
            int32_t *d_nsim = (int32_t *)g_nsim.p;
            uint64_t *d_or = (uint64_t *)g_or.p;
            uint64_t *d_and = use_and ? (uint64_t *)g_and.p : nullptr;

            // work lists: [small..., large...]
            const size_t nwork = small.size() + large.size();
            BUILD_TRY(g_work.ensure(nwork * sizeof(NodeWork), s));
            NodeWork *d_work = (NodeWork *)g_work.p;
            if (!small.empty())
                BUILD_CUDA(cudaMemcpyAsync(d_work, small.data(), small.size() * sizeof(NodeWork),
                                           cudaMemcpyHostToDevice, s));
            if (!large.empty())
                BUILD_CUDA(cudaMemcpyAsync(d_work + small.size(), large.data(),
                                           large.size() * sizeof(NodeWork), cudaMemcpyHostToDevice, s));
            if (!large.empty()) {
                const size_t L = large.size(), C = chunks.size();
                NodeWork *d_large = d_work + small.size();
                BUILD_TRY(g_chunks.ensure(C * sizeof(Chunk), s));
                BUILD_TRY(g_counts.ensure(L * kBits * 4, s));
                BUILD_TRY(g_hist.ensure(L * kBits * 4, s));
                BUILD_TRY(g_kstar.ensure(L * 8, s));
                BUILD_TRY(g_mode.ensure(L * 4, s));
                BUILD_TRY(g_cdis.ensure(C * 4, s));
                BUILD_TRY(g_coff.ensure(C * 4, s));
                BUILD_TRY(g_first.ensure((L + 1) * 4, s));
                Chunk *d_chunks = (Chunk *)g_chunks.p;
                BUILD_CUDA(cudaMemcpyAsync(d_chunks, chunks.data(), C * sizeof(Chunk),
                                           cudaMemcpyHostToDevice, s));
                BUILD_CUDA(cudaMemcpyAsync(g_first.p, first_chunk.data(), (L + 1) * 4,
                                           cudaMemcpyHostToDevice, s));
                BUILD_CUDA(cudaMemsetAsync(g_counts.p, 0, L * kBits * 4, s));
                BUILD_CUDA(cudaMemsetAsync(g_hist.p, 0, L * kBits * 4, s));
                for (const NodeWork &w : large) {
                    BUILD_CUDA(cudaMemsetAsync(d_or + (int64_t)w.id * kWords, 0, kWords * 8, s));
                    if (d_and)
                        BUILD_CUDA(cudaMemsetAsync(d_and + (int64_t)w.id * kWords, 0xFF, kWords * 8, s));
                }
                large_count_kernel<<<(unsigned)C, BT, 0, s>>>(
                    d_chunks, d_large, db, perm, (uint32_t *)g_counts.p,
                    (unsigned long long *)d_or, (unsigned long long *)d_and);
                large_minkey_kernel<<<(unsigned)C, BT, 0, s>>>(d_chunks, db, perm,
                                                              (const uint32_t *)g_counts.p, mk,
                                                              (uint32_t *)g_hist.p);
                large_select_kernel<<<(unsigned)L, 1024, 0, s>>>(
                    d_large, (const uint32_t *)g_counts.p, (const uint32_t *)g_hist.p,
                    (uint64_t *)g_kstar.p, (int32_t *)g_mode.p, d_nsim);
                large_chunk_count_kernel<<<(unsigned)C, BT, 0, s>>>(
                    d_chunks, d_large, mk, (const uint64_t *)g_kstar.p, (const int32_t *)g_mode.p,
                    (uint32_t *)g_cdis.p);
                large_chunk_scan_kernel<<<(unsigned)((L + 127) / 128), 128, 0, s>>>(
                    (const int32_t *)g_first.p, (int)L, (const uint32_t *)g_cdis.p,
                    (uint32_t *)g_coff.p);
                large_scatter_kernel<<<(unsigned)C, BT, 0, s>>>(
                    d_chunks, d_large, mk, (const uint64_t *)g_kstar.p, (const int32_t *)g_mode.p,
                    d_nsim, (const uint32_t *)g_coff.p, perm, tmp);
                copy_back_kernel<<<(unsigned)C, BT, 0, s>>>(d_chunks, tmp, perm);
                BUILD_CUDA(cudaGetLastError());
            }
            if (!small.empty()) {
                small_node_kernel<<<(unsigned)small.size(), BT, ssmem, s>>>(
                    d_work, db, perm, d_or, d_and, leaf_size, cap, d_nsim);
                BUILD_CUDA(cudaGetLastError());
            }
            n_sim.resize((size_t)m);
            BUILD_CUDA(cudaMemcpyAsync(n_sim.data(), d_nsim, (size_t)m * 4, cudaMemcpyDeviceToHost, s));
            BUILD_CUDA(cudaStreamSynchronize(s));

            // next level: children of internal nodes, in order, similar first
            std::vector<BuildRoot> next;
            for (int64_t i = 0; i < m; ++i) {
                const BuildRoot &r = lvl[(size_t)i];
                if (r.count <= leaf_size) continue;
                const int32_t ns = n_sim[(size_t)i];
                if (ns <= 0 || ns >= r.count) {
                    set_error("internal error: empty side after split");
                    rc = DT_ECUDA;
                    goto fail;
                }
                const int32_t c0 = (int32_t)recs.size();
                recs[(size_t)r.id].first_child = c0;
                const BuildRoot sim{c0, r.begin, ns, r.level + 1};
                const BuildRoot dis{c0 + 1, r.begin + ns, r.count - ns, r.level + 1};
                for (const BuildRoot &c : {sim, dis}) {
                    recs.push_back(NodeRec{-1, c.begin, c.count, c.level});
                    next.push_back(c);
                }
            }
            lvl.swap(next);
        }
        cleanup();
        return DT_OK;
    }
fail:
    cleanup();
    cudaStreamSynchronize(s);
    return rc;
#undef BUILD_TRY
#undef BUILD_CUDA
}

int build_tree(const uint64_t *db, int64_t n, int leaf_size, int use_and, int fused_cap,
               cudaStream_t s, dt_index *ix)
{
    Scratch scratch(s);
    uint32_t *perm = nullptr;
    DT_CUDA_TRY(scratch.alloc(&perm, (size_t)n * 4));
    iota_kernel<<<std::min<int64_t>((n + 255) / 256, 65535), 256, 0, s>>>(perm, n);
    DT_CUDA_TRY(cudaGetLastError());

    Grow g_or, g_and;
    struct Release {
        Grow &a, &b;
        cudaStream_t s;
        ~Release() { a.release(s); b.release(s); }
    } release{g_or, g_and, s};
    std::vector<NodeRec> recs{NodeRec{-1, 0, (int32_t)n, 0}};
    int64_t n_leaves = 0;
    int32_t depth = 0;
    int rc = grow_forest(db, perm, n, {BuildRoot{0, 0, (int32_t)n, 0}}, leaf_size, use_and, fused_cap,
                         s, g_or, g_and, recs, &n_leaves, &depth);
    if (rc != DT_OK) return rc;

    const int64_t n_nodes = (int64_t)recs.size();
    ix->n = n;
    ix->n_nodes = n_nodes;
    ix->n_leaves = n_leaves;
    ix->depth = depth;
    ix->leaf_size = leaf_size;
    ix->use_and = use_and;
    DT_CUDA_TRY(cudaMalloc((void **)&ix->or_img, (size_t)n_nodes * kWords * 8));
    DT_CUDA_TRY(cudaMemcpyAsync(ix->or_img, g_or.p, (size_t)n_nodes * kWords * 8,
                                cudaMemcpyDeviceToDevice, s));
    if (use_and) {
        DT_CUDA_TRY(cudaMalloc((void **)&ix->and_img, (size_t)n_nodes * kWords * 8));
        DT_CUDA_TRY(cudaMemcpyAsync(ix->and_img, g_and.p, (size_t)n_nodes * kWords * 8,
                                    cudaMemcpyDeviceToDevice, s));
    }
    DT_CUDA_TRY(cudaMalloc((void **)&ix->node, (size_t)n_nodes * sizeof(NodeRec)));
    DT_CUDA_TRY(cudaMemcpyAsync(ix->node, recs.data(), (size_t)n_nodes * sizeof(NodeRec),
                                cudaMemcpyHostToDevice, s));
    DT_CUDA_TRY(cudaMalloc((void **)&ix->db_tree, (size_t)n * kWords * 8));
    DT_CUDA_TRY(cudaMalloc((void **)&ix->perm, (size_t)n * 4));
    DT_CUDA_TRY(cudaMalloc((void **)&ix->iperm, (size_t)n * 4));
    gather_rows_kernel<<<std::min<int64_t>((n + 7) / 8, 8 * 152 * 8), 256, 0, s>>>(db, perm, n,
                                                                                   ix->db_tree);
    DT_CUDA_TRY(cudaGetLastError());
    DT_CUDA_TRY(cudaMemcpyAsync(ix->perm, perm, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
    invert_kernel<<<std::min<int64_t>((n + 255) / 256, 65535), 256, 0, s>>>(perm, n, ix->iperm);
    DT_CUDA_TRY(cudaGetLastError());
    if (int rc = make_tile_images(ix->db_tree, n, &ix->tile_or, &ix->tile_kmask, s)) return rc;
    DT_CUDA_TRY(cudaStreamSynchronize(s));
    return DT_OK;
}

// Tile images: a warp per run of kScanTileRows tree-ordered rows; lane l
// owns the 128-bit chunk l (words 2l, 2l + 1) of the running OR, so the
// chunk mask is one ballot.
__global__ void tile_images_kernel(const uint64_t *__restrict__ db_tree, int64_t n, int64_t n_tt,
                                   uint64_t *__restrict__ tile_or, uint32_t *__restrict__ kmask)
{
    const int lane = threadIdx.x & 31;
    int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t stride = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (; t < n_tt; t += stride) {
        const int64_t r0 = t * kScanTileRows, r1 = min(n, r0 + kScanTileRows);
        uint4 o = make_uint4(0u, 0u, 0u, 0u);
        for (int64_t r = r0; r < r1; ++r) {
            const uint4 v = __ldg(reinterpret_cast<const uint4 *>(db_tree + r * kWords) + lane);
            o.x |= v.x; o.y |= v.y; o.z |= v.z; o.w |= v.w;
        }
        reinterpret_cast<uint4 *>(tile_or + t * kWords)[lane] = o;
        const uint32_t m = __ballot_sync(0xffffffffu, (o.x | o.y | o.z | o.w) != 0u);
        if (lane == 0) kmask[t] = m;
    }
}

int make_tile_images(const uint64_t *db_tree, int64_t n, uint64_t **tile_or, uint32_t **kmask,
                     cudaStream_t s)
{
    *tile_or = nullptr;
    *kmask = nullptr;
    const int64_t n_tt = (n + kScanTileRows - 1) / kScanTileRows;
    uint64_t *o = nullptr;
    uint32_t *m = nullptr;
    cudaError_t e = cudaMalloc((void **)&o, (size_t)n_tt * kWords * 8);
    if (e == cudaSuccess) e = cudaMalloc((void **)&m, (size_t)n_tt * 4);
    if (e == cudaSuccess) {
        const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((n_tt + 7) / 8, (int64_t)sm_count() * 16));
        tile_images_kernel<<<(unsigned)blocks, 256, 0, s>>>(db_tree, n, n_tt, o, m);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        cudaFree(o);
        cudaFree(m);
        set_error(std::string("make_tile_images: ") + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? DT_ENOMEM : DT_ECUDA;
    }
    *tile_or = o;
    *kmask = m;
    return DT_OK;
}

// db_tree[pos] = db[perm[pos]] and iperm = perm^-1 for an index whose perm
// (device, n entries, a permutation of 0 .. n-1) is already in place;
// allocates both arrays.
int fill_index_rows(const uint64_t *db, dt_index *ix, cudaStream_t s)
{
    const int64_t n = ix->n;
    DT_CUDA_TRY(cudaMalloc((void **)&ix->db_tree, (size_t)n * kWords * 8));
    DT_CUDA_TRY(cudaMalloc((void **)&ix->iperm, (size_t)n * 4));
    gather_rows_kernel<<<std::min<int64_t>((n + 7) / 8, 8 * 152 * 8), 256, 0, s>>>(db, ix->perm, n,
                                                                                   ix->db_tree);
    invert_kernel<<<std::min<int64_t>((n + 255) / 256, 65535), 256, 0, s>>>(ix->perm, n, ix->iperm);
    DT_CUDA_TRY(cudaGetLastError());
    if (int rc = make_tile_images(ix->db_tree, n, &ix->tile_or, &ix->tile_kmask, s)) return rc;
    DT_CUDA_TRY(cudaStreamSynchronize(s));
    return DT_OK;
}

}  // namespace dtk
