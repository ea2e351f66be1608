// objects.cu — object distance scores (§6.4): for a query object (a set of
// descriptors) and a database object, the sum over the query's descriptors
// of each one's Eq. 1 distance to its nearest descriptor of that object.
//
// Every (query descriptor, database descriptor) pair is needed, so the work
// is the brute force's, with a per-object minimum in place of the top-k:
//   1. the database rows are grouped by object (counting sort, one copy);
//   2. the query descriptors are widened once into tensor-core tiles;
//   3. a unit table pairs every object's row range with every pair of query
//      tiles, and the tensor-core scan (bf_tc.cu, list mode, k = 1) leaves
//      the smallest key of every (object, query descriptor) in
//      partial[object][descriptor];
//   4. a warp per (query object, database object) turns those keys into
//      exact FP64 distances key / (P Z) and sums them.
// Query descriptors are processed in chunks of whole query objects, so the
// per-object minima of one chunk fit a bounded buffer.
#include <algorithm>
#include <cmath>
#include <vector>

#include "block_util.cuh"
#include "dt_internal.cuh"

namespace dtk {
namespace {

__global__ void object_count_kernel(const uint32_t *__restrict__ object_of, int64_t n,
                                    int n_objects, int32_t *__restrict__ counts)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; i < n; i += stride) {
        const uint32_t o = object_of[i];
        if (o < (uint32_t)n_objects) atomicAdd(&counts[o], 1);
    }
}

// One block: exclusive prefix sum of the per-object counts.
__global__ void object_offsets_kernel(const int32_t *__restrict__ counts, int n_objects,
                                      int64_t *__restrict__ offsets)
{
    __shared__ uint32_t tmp[33];
    uint32_t run = 0;
    for (int c0 = 0; c0 < n_objects; c0 += blockDim.x) {
        const int c = c0 + threadIdx.x;
        uint32_t tot;
        const uint32_t before = block_excl_scan(c < n_objects ? (uint32_t)counts[c] : 0u, tmp, &tot);
        if (c < n_objects) offsets[c] = (int64_t)run + before;
        run += tot;
    }
    if (threadIdx.x == 0) offsets[n_objects] = run;
}

// A warp per database row: copy it into its object's segment.
__global__ void object_scatter_kernel(const uint64_t *__restrict__ db, int64_t n,
                                      const uint32_t *__restrict__ object_of, int n_objects,
                                      const int64_t *__restrict__ offsets, int32_t *__restrict__ fill,
                                      uint64_t *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (; w < n; w += nw) {
        const uint32_t o = object_of[w];
        if (o >= (uint32_t)n_objects) continue;
        int pos = 0;
        if (lane == 0) pos = atomicAdd(&fill[o], 1);
        pos = __shfl_sync(0xffffffffu, pos, 0);
        reinterpret_cast<uint4 *>(out + (offsets[o] + pos) * kWords)[lane] =
            reinterpret_cast<const uint4 *>(db + w * kWords)[lane];
    }
}

// Unit (o, p): object o's rows against query tiles 2p and 2p + 1 of the chunk.
__global__ void object_units_kernel(const int64_t *__restrict__ offsets, int n_objects,
                                    int64_t m, int n_pairs, int64_t slots_per_object,
                                    TcUnit *__restrict__ units)
{
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= (int64_t)n_objects * n_pairs) return;
    const int o = (int)(u / n_pairs), p = (int)(u % n_pairs);
    TcUnit t;
    t.row0 = offsets[o];
    t.row1 = offsets[o + 1];
    t.a_tile0 = 2 * p;
    t.nvalid0 = (int32_t)std::min<int64_t>(kTcTileM, m - (int64_t)(2 * p) * kTcTileM);
    const bool two = (int64_t)(2 * p + 1) * kTcTileM < m;
    t.a_tile1 = two ? 2 * p + 1 : -1;
    t.nvalid1 = two ? (int32_t)std::min<int64_t>(kTcTileM, m - (int64_t)(2 * p + 1) * kTcTileM) : 0;
    t.out_base = (int64_t)o * slots_per_object;
    units[u] = t;
}

// A warp per (query object j of the chunk, database object o): the sum of
// key / (P Z) in FP64 over j's descriptors; +inf if o has no descriptor.
__global__ void object_sum_kernel(const uint64_t *__restrict__ partial, int64_t slots_per_object,
                                  const uint32_t *__restrict__ qpop, const int64_t *__restrict__ qoff,
                                  int j0, int nq_chunk, int64_t d0, int n_objects,
                                  double *__restrict__ scores)
{
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= (int64_t)nq_chunk * n_objects) return;
    const int j = (int)(w / n_objects), o = (int)(w % n_objects);
    const int64_t b = qoff[j0 + j] - d0, e = qoff[j0 + j + 1] - d0;
    double sum = 0.0;
    bool missing = false;
    for (int64_t i = b + lane; i < e; i += 32) {
        const uint64_t v = partial[(int64_t)o * slots_per_object + i];
        if (v == kEmpty) {
            missing = true;
            continue;
        }
        const uint32_t pop = qpop[i];
        const double P = pop > 1 ? (double)pop : 1.0;
        const double Z = (uint32_t)kBits - pop > 1 ? (double)(kBits - pop) : 1.0;
        sum += (double)(uint32_t)(v >> 32) / (P * Z);
    }
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, s);
    missing = __any_sync(0xffffffffu, missing);
    if (lane == 0) scores[(int64_t)(j0 + j) * n_objects + o] = missing ? INFINITY : sum;
}

constexpr size_t kPartialBudget = (size_t)1 << 30;   // bytes of per-object minima per chunk

}  // namespace
}  // namespace dtk

using namespace dtk;

extern "C" {

int object_scores(const uint64_t *d_db, int64_t n, const uint32_t *d_object_of, int32_t n_objects,
                  const uint64_t *d_qdesc, const int64_t *d_qoffsets, int32_t nq, int64_t n_qdesc,
                  double *d_scores, void *stream)
{
    DT_CHECK_ARG(d_db && d_object_of && d_scores && n >= 1 && n_objects >= 1 && nq >= 0 &&
                 n_qdesc >= 0 && (nq == 0 || d_qoffsets), "bad arguments");
    DT_CHECK_ARG(n <= DT_MAX_N - 65536, "n out of range");
    if (nq == 0) return DT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int64_t> off((size_t)nq + 1);
    DT_CUDA_TRY(cudaMemcpyAsync(off.data(), d_qoffsets, off.size() * 8, cudaMemcpyDeviceToHost, s));
    DT_CUDA_TRY(cudaStreamSynchronize(s));
    DT_CHECK_ARG(off[0] == 0 && off[nq] == n_qdesc, "qoffsets must run from 0 to n_qdesc");
    for (int32_t j = 0; j < nq; ++j) DT_CHECK_ARG(off[j + 1] >= off[j], "qoffsets must not decrease");

    Scratch scratch(s);
    int32_t *counts = nullptr;
    int64_t *obj_off = nullptr, *n_units = nullptr;
    uint64_t *db_obj = nullptr;
    DT_CUDA_TRY(scratch.alloc(&counts, (size_t)n_objects * 4 * 2));
    DT_CUDA_TRY(scratch.alloc(&obj_off, (size_t)(n_objects + 1) * 8));
    DT_CUDA_TRY(scratch.alloc(&db_obj, (size_t)n * 512));
    DT_CUDA_TRY(scratch.alloc(&n_units, 8));
    int32_t *fill = counts + n_objects;
    DT_CUDA_TRY(cudaMemsetAsync(counts, 0, (size_t)n_objects * 4 * 2, s));
    const unsigned gb = (unsigned)std::min<int64_t>((n + 255) / 256, 8192);
    object_count_kernel<<<gb, 256, 0, s>>>(d_object_of, n, n_objects, counts);
    object_offsets_kernel<<<1, 1024, 0, s>>>(counts, n_objects, obj_off);
    object_scatter_kernel<<<(unsigned)std::min<int64_t>((n + 7) / 8, 8192), 256, 0, s>>>(
        d_db, n, d_object_of, n_objects, obj_off, fill, db_obj);
    DT_CUDA_TRY(cudaGetLastError());

    // chunks of whole query objects whose per-object minima fit the budget
    // (a query object larger than the budget forms a chunk of its own)
    const int64_t budget_desc =
        std::max<int64_t>(kTcTileM, (int64_t)(kPartialBudget / 8 / (size_t)n_objects));
    int rc = DT_OK;
    for (int32_t j0 = 0; j0 < nq && rc == DT_OK;) {
        int32_t j1 = j0 + 1;
        while (j1 < nq && off[j1 + 1] - off[j0] <= budget_desc) ++j1;
        const int64_t d0 = off[j0], m = off[j1] - off[j0];
        if (m == 0) {                         // query objects without descriptors score 0
            DT_CUDA_TRY(cudaMemsetAsync(d_scores + (int64_t)j0 * n_objects, 0,
                                        (size_t)(j1 - j0) * n_objects * 8, s));
            j0 = j1;
            continue;
        }
        Scratch chunk(s);
        const int64_t tiles = (m + kTcTileM - 1) / kTcTileM;
        const int n_pairs = (int)((tiles + 1) / 2);
        const int64_t slots = tiles * kTcTileM;
        const int64_t n_u = (int64_t)n_objects * n_pairs;
        unsigned char *a_exp = nullptr;
        uint32_t *qpop = nullptr;
        TcUnit *units = nullptr;
        uint64_t *partial = nullptr;
        DT_CUDA_TRY(chunk.alloc(&a_exp, (size_t)tiles * tc_tile_bytes()));
        DT_CUDA_TRY(chunk.alloc(&qpop, (size_t)slots * 4));
        DT_CUDA_TRY(chunk.alloc(&units, (size_t)n_u * sizeof(TcUnit)));
        DT_CUDA_TRY(chunk.alloc(&partial, (size_t)n_objects * slots * 8));
        DT_CUDA_TRY(cudaMemsetAsync(partial, 0xFF, (size_t)n_objects * slots * 8, s));
        DT_CUDA_TRY(cudaMemcpyAsync(n_units, &n_u, 8, cudaMemcpyHostToDevice, s));
        if ((rc = launch_widen_queries(d_qdesc + d0 * kWords, m, a_exp, qpop, s)) != DT_OK) break;
        object_units_kernel<<<(unsigned)((n_u + 255) / 256), 256, 0, s>>>(obj_off, n_objects, m,
                                                                            n_pairs, slots, units);
        DT_CUDA_TRY(cudaGetLastError());
        if ((rc = launch_tc_units_pre(db_obj, n, nullptr, a_exp, qpop, units, n_units, n_u, 1,
                                      partial, s)) != DT_OK)
            break;
        const int64_t warps = (int64_t)(j1 - j0) * n_objects;
        object_sum_kernel<<<(unsigned)((warps + 7) / 8), 256, 0, s>>>(
            partial, slots, qpop, d_qoffsets, j0, j1 - j0, d0, n_objects, d_scores);
        DT_CUDA_TRY(cudaGetLastError());
        // the host value behind n_units must outlive the copy
        DT_CUDA_TRY(cudaStreamSynchronize(s));
        j0 = j1;
    }
    return rc;
}

}  // extern "C"
