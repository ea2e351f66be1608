// dt_insert.cu — incremental insertion into a built Dissimilarity Tree.
//
// §4.1 suggests that a tree can grow by redoing only the part of it that new
// descriptors touch.  A batch of m descriptors (original indices n .. n+m-1)
// goes in as follows; every step over descriptors or rows runs on the
// device, the host only numbers the nodes of rebuilt subtrees:
//   1. route: a warp per new descriptor descends from the root, against the
//      images as they were before the batch, into the child whose images it
//      widens least — popc(d & ~OR), plus popc(~d & AND) with AND images —
//      the similar child on ties (least-enlargement insertion, as in R-trees,
//      Guttman 1984), and records its leaf;
//   2. order: a stable LSD radix sort of the batch by the end position of
//      its leaf, so the new descriptors of one leaf keep ascending index;
//   3. widen: a warp per new descriptor walks its root-to-leaf path again
//      (by segment, never by image) and ORs / ANDs itself into a copy of the
//      images of every node on it;
//   4. shift: a tree-ordered row moves up by the number of new rows in the
//      leaves that end at or before it (one binary search per run of rows,
//      merge order after that); the new row of sorted rank t in a leaf that
//      ended at position e lands at e + t; every node's segment moves alike;
//   5. rebuild: every leaf now over leaf_size, in ascending id, is split by
//      the construction of §4.1 (grow_forest: the build's own kernels) as the
//      root of a subtree whose nodes are numbered after the old ones,
//      generation by generation; the rows of those segments are then
//      permuted through a scratch copy.
// The index is replaced only after every step has succeeded; on an error it
// is left as it was.
#include <algorithm>
#include <vector>

#include "dt_internal.cuh"
#include "sort_util.cuh"

namespace dtk {
namespace {

constexpr int kRun = 64;          // rows per warp in the shift
constexpr int kSegChunk = 4096;   // rows per block when permuting rebuilt segments

__device__ __forceinline__ uint64_t lo64(const uint4 v) { return ((uint64_t)v.y << 32) | v.x; }
__device__ __forceinline__ uint64_t hi64(const uint4 v) { return ((uint64_t)v.w << 32) | v.z; }

__device__ __forceinline__ int warp_sum(int v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// First index i of the non-decreasing a[0, len) with a[i] > x.
__device__ __forceinline__ int64_t upper_bound_u32(const uint32_t *__restrict__ a, int64_t len, int64_t x)
{
    int64_t lo = 0, hi = len;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if ((int64_t)a[mid] <= x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// 1. A warp per new descriptor: the leaf it joins, and that leaf's end.
__global__ void __launch_bounds__(256)
route_kernel(const uint64_t *__restrict__ d_new, int64_t m, const NodeRec *__restrict__ node,
             const uint64_t *__restrict__ or_img, const uint64_t *__restrict__ and_img,
             int max_steps, uint32_t *__restrict__ leaf_of, uint32_t *__restrict__ key,
             uint32_t *__restrict__ val, int *__restrict__ err)
{
    const int lane = threadIdx.x & 31;
    int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (; j < m; j += nw) {
        const uint4 v = reinterpret_cast<const uint4 *>(d_new + j * kWords)[lane];
        const uint64_t x0 = lo64(v), x1 = hi64(v);
        int32_t at = 0;
        NodeRec r = node[0];
        for (int step = 0; r.first_child >= 0 && step < max_steps; ++step) {
            const int32_t s = r.first_child;
            int g[2];
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const uint4 o = reinterpret_cast<const uint4 *>(or_img + (int64_t)(s + c) * kWords)[lane];
                int gl = __popcll(x0 & ~lo64(o)) + __popcll(x1 & ~hi64(o));
                if (and_img) {
                    const uint4 a =
                        reinterpret_cast<const uint4 *>(and_img + (int64_t)(s + c) * kWords)[lane];
                    gl += __popcll(~x0 & lo64(a)) + __popcll(~x1 & hi64(a));
                }
                g[c] = warp_sum(gl);
            }
            at = g[0] <= g[1] ? s : s + 1;
            r = node[at];
        }
        if (lane == 0) {
            if (r.first_child >= 0) atomicExch(err, 1);   // the depth bound was wrong
            leaf_of[j] = (uint32_t)at;
            key[j] = (uint32_t)(r.begin + r.count);
            val[j] = (uint32_t)j;
        }
    }
}

// 3. A warp per new descriptor: widen the images of every node on its path.
// A word is written only if it changes; images only gain (OR) or lose (AND)
// bits, so a stale read costs at most one needless atomic.
__global__ void __launch_bounds__(256)
widen_kernel(const uint64_t *__restrict__ d_new, int64_t m, const NodeRec *__restrict__ node,
             const uint32_t *__restrict__ leaf_of, int max_steps, unsigned long long *or_img,
             unsigned long long *and_img)
{
    const int lane = threadIdx.x & 31;
    int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (; j < m; j += nw) {
        const uint4 v = reinterpret_cast<const uint4 *>(d_new + j * kWords)[lane];
        const unsigned long long x[2] = {lo64(v), hi64(v)};
        const int32_t leaf = (int32_t)leaf_of[j];
        const int32_t target = node[leaf].begin;
        int32_t at = 0;
        for (int step = 0; step <= max_steps; ++step) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                unsigned long long *o = or_img + (int64_t)at * kWords + 2 * lane + h;
                const unsigned long long ov = __ldcg(o);
                if ((ov | x[h]) != ov) atomicOr(o, x[h]);
                if (and_img) {
                    unsigned long long *a = and_img + (int64_t)at * kWords + 2 * lane + h;
                    const unsigned long long av = __ldcg(a);
                    if ((av & x[h]) != av) atomicAnd(a, x[h]);
                }
            }
            if (at == leaf) break;
            const int32_t s = node[at].first_child;
            if (s < 0) break;                       // not on the path: nothing more to widen
            const NodeRec rs = node[s];
            at = target < rs.begin + rs.count ? s : s + 1;
        }
    }
}

// 4. A warp per run of kRun tree-ordered rows: row p moves to p + (number of
// sorted leaf ends <= p).
__global__ void __launch_bounds__(256)
shift_rows_kernel(const uint64_t *__restrict__ db_old, const uint32_t *__restrict__ perm_old,
                  int64_t n_old, const uint32_t *__restrict__ ends, int64_t m,
                  uint64_t *__restrict__ db_new, uint32_t *__restrict__ perm_new)
{
    const int lane = threadIdx.x & 31;
    int64_t run = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (; run * kRun < n_old; run += nw) {
        const int64_t r0 = run * kRun, r1 = std::min<int64_t>(r0 + kRun, n_old);
        int64_t t = upper_bound_u32(ends, m, r0);
        for (int64_t p = r0; p < r1; ++p) {
            if (t < m && (int64_t)ends[t] <= p) t += upper_bound_u32(ends + t, m - t, p);
            const int64_t np = p + t;
            reinterpret_cast<uint4 *>(db_new + np * kWords)[lane] =
                reinterpret_cast<const uint4 *>(db_old + p * kWords)[lane];
            if (lane == 0) perm_new[np] = perm_old[p];
        }
    }
}

// A warp per new row: sorted rank t in a leaf that ended at e goes to e + t.
__global__ void __launch_bounds__(256)
place_new_kernel(const uint64_t *__restrict__ d_new, int64_t m, const uint32_t *__restrict__ ends,
                 const uint32_t *__restrict__ order, int64_t n_old, uint64_t *__restrict__ db_new,
                 uint32_t *__restrict__ perm_new)
{
    const int lane = threadIdx.x & 31;
    int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (; t < m; t += nw) {
        const int64_t j = order[t], np = (int64_t)ends[t] + t;
        reinterpret_cast<uint4 *>(db_new + np * kWords)[lane] =
            reinterpret_cast<const uint4 *>(d_new + j * kWords)[lane];
        if (lane == 0) perm_new[np] = (uint32_t)(n_old + j);
    }
}

// A thread per node: its segment after the shift.
__global__ void node_shift_kernel(const NodeRec *__restrict__ in, int64_t n_nodes,
                                  const uint32_t *__restrict__ ends, int64_t m,
                                  NodeRec *__restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_nodes) return;
    NodeRec r = in[i];
    const int64_t b = r.begin, e = (int64_t)r.begin + r.count;
    const int64_t nb = b + upper_bound_u32(ends, m, b), ne = e + upper_bound_u32(ends, m, e);
    r.begin = (int32_t)nb;
    r.count = (int32_t)(ne - nb);
    out[i] = r;
}

__global__ void iota_u32_kernel(uint32_t *p, int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; i < n; i += stride) p[i] = (uint32_t)i;
}

__global__ void invert_u32_kernel(const uint32_t *__restrict__ perm, int64_t n, uint32_t *__restrict__ iperm)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; i < n; i += stride) iperm[perm[i]] = (uint32_t)i;
}

struct SegChunk {
    int64_t begin;   // first tree position of the chunk
    int64_t count;
    int64_t off;     // first row of the chunk in the scratch copy
};

// 5. Rows of rebuilt segments: out[off + i] = row at position pl[begin + i].
__global__ void __launch_bounds__(256)
segment_gather_kernel(const SegChunk *__restrict__ chunks, const uint64_t *__restrict__ db,
                      const uint32_t *__restrict__ perm, const uint32_t *__restrict__ pl,
                      uint64_t *__restrict__ tmp_rows, uint32_t *__restrict__ tmp_perm)
{
    const SegChunk c = chunks[blockIdx.x];
    const int lane = threadIdx.x & 31;
    for (int64_t i = threadIdx.x >> 5; i < c.count; i += blockDim.x >> 5) {
        const int64_t src = pl[c.begin + i];
        reinterpret_cast<uint4 *>(tmp_rows + (c.off + i) * kWords)[lane] =
            reinterpret_cast<const uint4 *>(db + src * kWords)[lane];
        if (lane == 0) tmp_perm[c.off + i] = perm[src];
    }
}

__global__ void __launch_bounds__(256)
segment_put_kernel(const SegChunk *__restrict__ chunks, const uint64_t *__restrict__ tmp_rows,
                   const uint32_t *__restrict__ tmp_perm, uint64_t *__restrict__ db,
                   uint32_t *__restrict__ perm)
{
    const SegChunk c = chunks[blockIdx.x];
    const int lane = threadIdx.x & 31;
    for (int64_t i = threadIdx.x >> 5; i < c.count; i += blockDim.x >> 5) {
        reinterpret_cast<uint4 *>(db + (c.begin + i) * kWords)[lane] =
            reinterpret_cast<const uint4 *>(tmp_rows + (c.off + i) * kWords)[lane];
        if (lane == 0) perm[c.begin + i] = tmp_perm[c.off + i];
    }
}

// A device array from cudaMalloc, freed unless handed over to the index.
struct Owned {
    void *p = nullptr;
    ~Owned()
    {
        if (p) cudaFree(p);
    }
    template <class T> T *as() const { return static_cast<T *>(p); }
    void *release()
    {
        void *q = p;
        p = nullptr;
        return q;
    }
};

unsigned warp_grid(int64_t warps)
{
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((warps + 7) / 8, (int64_t)sm_count() * 64));
}

}  // namespace

int insert_tree(dt_index *ix, const uint64_t *d_new, int64_t m, cudaStream_t s)
{
    const int64_t n_old = ix->n, n = n_old + m, nn = ix->n_nodes;
    const int max_steps = ix->depth + 1;
    Scratch scratch(s);
    uint32_t *leaf_of = nullptr, *keys = nullptr, *vals = nullptr, *keys2 = nullptr, *vals2 = nullptr,
             *hist = nullptr;
    int *err = nullptr;
    NodeRec *node_tmp = nullptr;
    const int64_t n_tiles = radix_tiles(m);
    DT_CUDA_TRY(scratch.alloc(&leaf_of, (size_t)m * 4));
    DT_CUDA_TRY(scratch.alloc(&keys, (size_t)m * 4));
    DT_CUDA_TRY(scratch.alloc(&vals, (size_t)m * 4));
    DT_CUDA_TRY(scratch.alloc(&keys2, (size_t)m * 4));
    DT_CUDA_TRY(scratch.alloc(&vals2, (size_t)m * 4));
    DT_CUDA_TRY(scratch.alloc(&hist, (size_t)n_tiles * 256 * 4));
    DT_CUDA_TRY(scratch.alloc(&err, sizeof(int)));
    DT_CUDA_TRY(scratch.alloc(&node_tmp, (size_t)nn * sizeof(NodeRec)));
    DT_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));

    // 1. route against the images as they were before the batch
    route_kernel<<<warp_grid(m), 256, 0, s>>>(d_new, m, ix->node, ix->or_img, ix->and_img, max_steps,
                                              leaf_of, keys, vals, err);
    DT_CUDA_TRY(cudaGetLastError());

    // 3. widen a copy of the images
    Grow g_or, g_and;
    struct Release {
        Grow &a, &b;
        cudaStream_t s;
        ~Release() { a.release(s); b.release(s); }
    } release{g_or, g_and, s};
    int rc = g_or.ensure((size_t)nn * kWords * 8, s);
    if (rc != DT_OK) return rc;
    DT_CUDA_TRY(cudaMemcpyAsync(g_or.p, ix->or_img, (size_t)nn * kWords * 8, cudaMemcpyDeviceToDevice, s));
    if (ix->use_and) {
        if ((rc = g_and.ensure((size_t)nn * kWords * 8, s)) != DT_OK) return rc;
        DT_CUDA_TRY(cudaMemcpyAsync(g_and.p, ix->and_img, (size_t)nn * kWords * 8,
                                    cudaMemcpyDeviceToDevice, s));
    }
    widen_kernel<<<warp_grid(m), 256, 0, s>>>(d_new, m, ix->node, leaf_of, max_steps,
                                              (unsigned long long *)g_or.p,
                                              ix->use_and ? (unsigned long long *)g_and.p : nullptr);
    DT_CUDA_TRY(cudaGetLastError());

    // 2. stable sort by leaf end (keys <= n_old)
    int bits = 1;
    while (bits < 32 && (n_old >> bits) != 0) ++bits;
    DT_CUDA_TRY(radix_sort_pairs(&keys, &vals, &keys2, &vals2, m, bits, hist, s));

    // 4. shifted rows and segments
    Owned db_new, perm_new, iperm_new, node_new, or_new, and_new;
    DT_CUDA_TRY(cudaMalloc(&db_new.p, (size_t)n * kWords * 8));
    DT_CUDA_TRY(cudaMalloc(&perm_new.p, (size_t)n * 4));
    shift_rows_kernel<<<warp_grid((n_old + kRun - 1) / kRun), 256, 0, s>>>(
        ix->db_tree, ix->perm, n_old, keys, m, db_new.as<uint64_t>(), perm_new.as<uint32_t>());
    place_new_kernel<<<warp_grid(m), 256, 0, s>>>(d_new, m, keys, vals, n_old, db_new.as<uint64_t>(),
                                                  perm_new.as<uint32_t>());
    node_shift_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(ix->node, nn, keys, m, node_tmp);
    DT_CUDA_TRY(cudaGetLastError());
    std::vector<NodeRec> recs((size_t)nn);
    int h_err = 0;
    DT_CUDA_TRY(cudaMemcpyAsync(recs.data(), node_tmp, (size_t)nn * sizeof(NodeRec),
                                cudaMemcpyDeviceToHost, s));
    DT_CUDA_TRY(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    DT_CUDA_TRY(cudaStreamSynchronize(s));
    if (h_err) {
        set_error("internal error: a routed descriptor did not reach a leaf");
        return DT_ECUDA;
    }

    // 5. rebuild the leaves over leaf_size
    std::vector<BuildRoot> roots;
    for (int64_t i = 0; i < nn; ++i) {
        const NodeRec &r = recs[(size_t)i];
        if (r.first_child < 0 && r.count > ix->leaf_size)
            roots.push_back(BuildRoot{(int32_t)i, r.begin, r.count, r.level});
    }
    int64_t n_leaves = ix->n_leaves - (int64_t)roots.size();
    int32_t depth = ix->depth;
    if (!roots.empty()) {
        uint32_t *pl = nullptr;
        DT_CUDA_TRY(scratch.alloc(&pl, (size_t)n * 4));
        iota_u32_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 65535), 256, 0, s>>>(pl, n);
        DT_CUDA_TRY(cudaGetLastError());
        if ((rc = grow_forest(db_new.as<uint64_t>(), pl, n, roots, ix->leaf_size, ix->use_and, 0, s,
                              g_or, g_and, recs, &n_leaves, &depth)) != DT_OK)
            return rc;
        std::vector<SegChunk> chunks;
        int64_t total = 0;
        for (const BuildRoot &r : roots)
            for (int64_t b = r.begin; b < (int64_t)r.begin + r.count; b += kSegChunk) {
                const int64_t c = std::min<int64_t>(kSegChunk, (int64_t)r.begin + r.count - b);
                chunks.push_back(SegChunk{b, c, total});
                total += c;
            }
        SegChunk *d_chunks = nullptr;
        uint64_t *tmp_rows = nullptr;
        uint32_t *tmp_perm = nullptr;
        DT_CUDA_TRY(scratch.alloc(&d_chunks, chunks.size() * sizeof(SegChunk)));
        DT_CUDA_TRY(scratch.alloc(&tmp_rows, (size_t)total * kWords * 8));
        DT_CUDA_TRY(scratch.alloc(&tmp_perm, (size_t)total * 4));
        DT_CUDA_TRY(cudaMemcpyAsync(d_chunks, chunks.data(), chunks.size() * sizeof(SegChunk),
                                    cudaMemcpyHostToDevice, s));
        segment_gather_kernel<<<(unsigned)chunks.size(), 256, 0, s>>>(
            d_chunks, db_new.as<uint64_t>(), perm_new.as<uint32_t>(), pl, tmp_rows, tmp_perm);
        segment_put_kernel<<<(unsigned)chunks.size(), 256, 0, s>>>(
            d_chunks, tmp_rows, tmp_perm, db_new.as<uint64_t>(), perm_new.as<uint32_t>());
        DT_CUDA_TRY(cudaGetLastError());
        // the host copy of `chunks` must outlive the upload
        DT_CUDA_TRY(cudaStreamSynchronize(s));
    }

    // the new index arrays
    const int64_t nn2 = (int64_t)recs.size();
    DT_CUDA_TRY(cudaMalloc(&node_new.p, (size_t)nn2 * sizeof(NodeRec)));
    DT_CUDA_TRY(cudaMemcpyAsync(node_new.p, recs.data(), (size_t)nn2 * sizeof(NodeRec),
                                cudaMemcpyHostToDevice, s));
    DT_CUDA_TRY(cudaMalloc(&or_new.p, (size_t)nn2 * kWords * 8));
    DT_CUDA_TRY(cudaMemcpyAsync(or_new.p, g_or.p, (size_t)nn2 * kWords * 8, cudaMemcpyDeviceToDevice, s));
    if (ix->use_and) {
        DT_CUDA_TRY(cudaMalloc(&and_new.p, (size_t)nn2 * kWords * 8));
        DT_CUDA_TRY(cudaMemcpyAsync(and_new.p, g_and.p, (size_t)nn2 * kWords * 8,
                                    cudaMemcpyDeviceToDevice, s));
    }
    DT_CUDA_TRY(cudaMalloc(&iperm_new.p, (size_t)n * 4));
    invert_u32_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 65535), 256, 0, s>>>(
        perm_new.as<uint32_t>(), n, iperm_new.as<uint32_t>());
    DT_CUDA_TRY(cudaGetLastError());
    Owned tor_new, tmask_new;
    {
        uint64_t *to = nullptr;
        uint32_t *tm = nullptr;
        if ((rc = make_tile_images(db_new.as<uint64_t>(), n, &to, &tm, s)) != DT_OK) return rc;
        tor_new.p = to;
        tmask_new.p = tm;
    }
    DT_CUDA_TRY(cudaStreamSynchronize(s));

    cudaFree(ix->db_tree);
    cudaFree(ix->perm);
    cudaFree(ix->iperm);
    cudaFree(ix->node);
    cudaFree(ix->or_img);
    cudaFree(ix->and_img);
    cudaFree(ix->tile_or);
    cudaFree(ix->tile_kmask);
    ix->tile_or = static_cast<uint64_t *>(tor_new.release());
    ix->tile_kmask = static_cast<uint32_t *>(tmask_new.release());
    ix->db_tree = static_cast<uint64_t *>(db_new.release());
    ix->perm = static_cast<uint32_t *>(perm_new.release());
    ix->iperm = static_cast<uint32_t *>(iperm_new.release());
    ix->node = static_cast<NodeRec *>(node_new.release());
    ix->or_img = static_cast<uint64_t *>(or_new.release());
    ix->and_img = ix->use_and ? static_cast<uint64_t *>(and_new.release()) : nullptr;
    ix->n = n;
    ix->n_nodes = nn2;
    ix->n_leaves = n_leaves;
    ix->depth = depth;
    return DT_OK;
}

}  // namespace dtk
