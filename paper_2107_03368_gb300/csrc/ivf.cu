// ivf.cu — learned proposal: an inverted file over encoder embeddings, with
// an exact Eq. 1 rerank of every proposed candidate (the paper has no
// learned component; its exact search remains the reference for recall).
//
// Build (ivf_build): embed the database with the encoder (BF16), run k-means
// on the unit-length embeddings (cosine assignment, centroid = normalised
// mean), then lay the database out list by list: a cluster-ordered copy of
// the descriptor bits, the original index of each row and list offsets.
//
// Search (ivf_search): embed the queries; one CTA per query scores every
// centroid, keeps the n_probe best lists, and scans all of their rows
// exactly (A, B counts of Eq. 1, ranked by A*Z + B*P, ties by original
// index) — the candidates come from the learned embedding, the ranking is
// exact, so the answer equals the exact one whenever the true neighbours
// lie in the probed lists.
#include <algorithm>
#include <cmath>
#include <vector>

#include <cuda_bf16.h>

#include "block_util.cuh"
#include "dt_internal.cuh"
#include "dt_traverse.cuh"

struct dt_encoder;
extern "C" int enc_embed(const dt_encoder *e, const uint64_t *d_bits, int64_t n, uint16_t *d_out_bf16,
                         float *d_out_f32, int32_t path, void *stream);

namespace dtk {
namespace {

constexpr int D = 128;

// ------------------------------------------------ k-means assignment
// 32 points x 32 centroids per tile, 256 threads, 2 x 2 dot products each.
constexpr int KT = 32;

__global__ void __launch_bounds__(256)
assign_kernel(const __nv_bfloat16 *__restrict__ emb, int64_t n, const float *__restrict__ cent,
              int K, int32_t *__restrict__ assign)
{
    __shared__ float ps[KT][D + 1];
    __shared__ float cs[KT][D + 1];
    __shared__ unsigned long long best[KT];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t p0 = (int64_t)blockIdx.x * KT;
    for (int i = tid; i < KT * D; i += 256) {
        const int r = i / D, c = i % D;
        ps[r][c] = p0 + r < n ? __bfloat162float(emb[(p0 + r) * D + c]) : 0.f;
    }
    if (tid < KT) best[tid] = 0ull;
    __syncthreads();
    for (int c0 = 0; c0 < K; c0 += KT) {
        for (int i = tid; i < KT * D; i += 256) {
            const int r = i / D, c = i % D;
            cs[r][c] = c0 + r < K ? cent[(int64_t)(c0 + r) * D + c] : 0.f;
        }
        __syncthreads();
        float acc[2][2] = {};
        for (int d = 0; d < D; ++d) {
            float a[2], b[2];
#pragma unroll
            for (int i = 0; i < 2; ++i) a[i] = ps[ty + 16 * i][d];
#pragma unroll
            for (int j = 0; j < 2; ++j) b[j] = cs[tx + 16 * j][d];
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 2; ++j) acc[i][j] += a[i] * b[j];
        }
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int c = c0 + tx + 16 * j;
                if (c >= K) continue;
                // larger dot first, lower centroid id on ties: order-preserving
                // float bits in the high word, inverted id in the low word
                uint32_t fb = __float_as_uint(acc[i][j]);
                fb = (fb & 0x80000000u) ? ~fb : (fb | 0x80000000u);
                const unsigned long long key = ((unsigned long long)fb << 32) | (0xFFFFFFFFu - (uint32_t)c);
                atomicMax(&best[ty + 16 * i], key);
            }
        __syncthreads();
    }
    if (tid < KT && p0 + tid < n) assign[p0 + tid] = (int32_t)(0xFFFFFFFFu - (uint32_t)(best[tid] & 0xFFFFFFFFu));
}

// Centroid sums in fixed point: each component (|x| <= 1, the embeddings
// are unit length) scaled by 2^30 and rounded to an integer, so that the
// sums, integer additions, do not depend on the order of the atomics and the
// build is the same on every run.  2^30 * n stays below 2^63 for n < 2^32.
constexpr float kSumScale = 1073741824.f;   // 2^30

// sums[c] += emb[i] for assign[i] = c; counts[c] += 1
__global__ void accumulate_kernel(const __nv_bfloat16 *__restrict__ emb, int64_t n,
                                  const int32_t *__restrict__ assign,
                                  unsigned long long *__restrict__ sums, int32_t *__restrict__ counts)
{
    const int lane = threadIdx.x & 31;
    int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t stride = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (; i < n; i += stride) {
        const int c = assign[i];
#pragma unroll
        for (int j = 0; j < 4; ++j)
            atomicAdd(&sums[(int64_t)c * D + lane + 32 * j],
                      (unsigned long long)__float2ll_rn(__bfloat162float(emb[i * D + lane + 32 * j]) * kSumScale));
        if (lane == 0) atomicAdd(&counts[c], 1);
    }
}

// centroid = normalised sum (kept when its cluster is empty); warp per centroid
__global__ void update_kernel(const unsigned long long *__restrict__ sums, const int32_t *__restrict__ counts,
                              int K, float *__restrict__ cent)
{
    const int lane = threadIdx.x & 31;
    const int c = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (c >= K || counts[c] == 0) return;
    float v[4], ss = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        v[j] = __ll2float_rn((long long)sums[(int64_t)c * D + lane + 32 * j]) / kSumScale;
        ss += v[j] * v[j];
    }
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    const float inv = 1.f / fmaxf(sqrtf(ss), 1e-12f);
#pragma unroll
    for (int j = 0; j < 4; ++j) cent[(int64_t)c * D + lane + 32 * j] = v[j] * inv;
}

__global__ void init_centroids_kernel(const __nv_bfloat16 *__restrict__ emb, int64_t n, int K,
                                      float *__restrict__ cent)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)K * D) return;
    const int64_t c = i / D, d = i % D;
    const int64_t src = (c * n) / K;                 // evenly spaced rows
    cent[i] = __bfloat162float(emb[src * D + d]);
}

// rows of list c go to [offsets[c], offsets[c+1]); order inside a list is
// irrelevant to the results (ties are broken by original index)
__global__ void scatter_kernel(const uint64_t *__restrict__ db, int64_t n,
                               const int32_t *__restrict__ assign, const int64_t *__restrict__ offsets,
                               int32_t *__restrict__ cursor, uint64_t *__restrict__ ivf_db,
                               uint32_t *__restrict__ ivf_ids)
{
    const int lane = threadIdx.x & 31;
    int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t stride = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (; i < n; i += stride) {
        const int c = assign[i];
        int pos = 0;
        if (lane == 0) pos = atomicAdd(&cursor[c], 1);
        pos = __shfl_sync(0xffffffffu, pos, 0);
        const int64_t dst = offsets[c] + pos;
        reinterpret_cast<uint4 *>(ivf_db + dst * kWords)[lane] =
            reinterpret_cast<const uint4 *>(db + i * kWords)[lane];
        if (lane == 0) ivf_ids[dst] = (uint32_t)i;
    }
}

__global__ void count_kernel(const int32_t *__restrict__ assign, int64_t n, int32_t *__restrict__ counts)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; i < n; i += stride) atomicAdd(&counts[assign[i]], 1);
}

__global__ void offsets_kernel(const int32_t *__restrict__ counts, int K, int64_t *__restrict__ offsets)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int64_t run = 0;
        for (int c = 0; c < K; ++c) {
            offsets[c] = run;
            run += counts[c];
        }
        offsets[K] = run;
    }
}

// ------------------------------------------------ search: one CTA per query
constexpr int ST = 256;
constexpr int MAX_PROBE = 256;

__global__ void __launch_bounds__(ST)
ivf_search_kernel(const float *__restrict__ qemb, const uint64_t *__restrict__ qs, int64_t nq,
                  const float *__restrict__ cent, int K, const int64_t *__restrict__ offsets,
                  const uint64_t *__restrict__ ivf_db, const uint32_t *__restrict__ ivf_ids,
                  int n_probe, int k, uint32_t *__restrict__ idx, float *__restrict__ score,
                  uint16_t *__restrict__ ab, int64_t *__restrict__ scanned,
                  int32_t *__restrict__ probe_out)
{
    extern __shared__ float csc[];                   // [K] centroid scores
    __shared__ float qe[D];
    __shared__ int probe[MAX_PROBE];
    __shared__ unsigned long long red[ST / 32];
    __shared__ uint64_t lists[ST / 32][kMaxK];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t q = blockIdx.x;
    if (tid < D) qe[tid] = qemb[q * D + tid];
    __syncthreads();
    for (int c = tid; c < K; c += ST) {       // centroids stored [D][K]: coalesced
        float s = 0.f;
        for (int d = 0; d < D; ++d) s = fmaf(qe[d], __ldg(cent + (int64_t)d * K + c), s);
        csc[c] = s;
    }
    __syncthreads();
    // n_probe best lists by repeated block-wide argmax (higher score, lower id)
    for (int p = 0; p < n_probe; ++p) {
        unsigned long long b = 0ull;
        for (int c = tid; c < K; c += ST) {
            uint32_t fb = __float_as_uint(csc[c]);
            fb = (fb & 0x80000000u) ? ~fb : (fb | 0x80000000u);
            const unsigned long long key = ((unsigned long long)fb << 32) | (0xFFFFFFFFu - (uint32_t)c);
            b = key > b ? key : b;
        }
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long u = __shfl_xor_sync(0xffffffffu, b, o);
            b = u > b ? u : b;
        }
        if (lane == 0) red[wid] = b;
        __syncthreads();
        if (tid == 0) {
            unsigned long long m = 0ull;
            for (int w = 0; w < ST / 32; ++w) m = red[w] > m ? red[w] : m;
            const int c = (int)(0xFFFFFFFFu - (uint32_t)(m & 0xFFFFFFFFu));
            probe[p] = c;
            csc[c] = -INFINITY;
        }
        __syncthreads();
    }
    if (probe_out) {                          // list-major path: hand the lists over
        if (tid < n_probe) probe_out[q * n_probe + tid] = probe[tid];
        if (tid == 0 && scanned) {
            int64_t rows = 0;
            for (int p = 0; p < n_probe; ++p) rows += offsets[probe[p] + 1] - offsets[probe[p]];
            scanned[q] = rows;
        }
        return;
    }
    // exact scan of the probed lists: warps take 32-row blocks in turn
    const uint4 qv = __ldg(reinterpret_cast<const uint4 *>(qs + q * kWords) + lane);
    const QueryWeights w = query_weights(warp_sum(popc4(qv)));
    uint64_t slot = kEmpty;
    int64_t rows = 0;
    for (int p = 0; p < n_probe; ++p) {
        const int c = probe[p];
        const int64_t b0 = offsets[c], b1 = offsets[c + 1];
        rows += b1 - b0;
        for (int64_t r0 = b0 + (int64_t)wid * 32; r0 < b1; r0 += ST) {
            const int m = (int)(b1 - r0 < 32 ? b1 - r0 : 32);
            uint32_t v[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                v[j] = 0;
                if (j < m) {
                    const uint4 t = __ldg(reinterpret_cast<const uint4 *>(ivf_db + (r0 + j) * kWords) + lane);
                    v[j] = popc_and4(qv, t) | (popc4(t) << 16);
                }
            }
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) {
#pragma unroll
                for (int j = 0; j < o; ++j) {
                    const bool hi = lane & o;
                    const uint32_t send = hi ? v[j] : v[j + o];
                    const uint32_t keep = hi ? v[j + o] : v[j];
                    v[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
                }
            }
            uint64_t cand = kEmpty;
            if (lane < m)
                cand = pack(pair_key(w, v[0] & 0xffffu, v[0] >> 16), __ldg(ivf_ids + r0 + lane));
            warp_list_merge(slot, cand, k, lane);
        }
    }
    if (lane < k) lists[wid][lane] = slot;
    __syncthreads();
    if (wid == 0) {
        uint64_t fin = kEmpty;
        for (int w2 = 0; w2 < ST / 32; ++w2)
            warp_list_merge(fin, lane < k ? lists[w2][lane] : kEmpty, k, lane);
        // (A, B) of each result from the candidate rows is not kept; recompute
        // them from the query and the result's row, found again by a scan of
        // the probed lists only when asked for.
        if (lane < k) {
            const int64_t o = q * k + lane;
            if (fin == kEmpty) {
                idx[o] = 0xFFFFFFFFu;
                score[o] = __int_as_float(0x7f800000);
            } else {
                idx[o] = (uint32_t)fin;
                score[o] = key_score(w, (uint32_t)(fin >> 32));
            }
        }
        if (lane == 0 && scanned) scanned[q] = rows;
    }
    (void)ab;
}

// Probes only, QB queries per block (QB <= 8): every centroid load feeds
// QB dot products; then warp w chooses query w's n_probe lists from the
// scores in shared memory (no block barriers).  Lane l holds the centroids
// l, l + 32, ...; it keeps its four best (score, -index) keys in registers,
// and the warp merges the lanes' sorted heads, one warp-wide maximum per
// pick; a lane whose four have all been taken finds its next four below the
// last one.  The picks and their order are those of a full warp-wide argmax
// per pick, as in ivf_search_kernel.
template <int QB>
__global__ void __launch_bounds__(ST)
ivf_probe_kernel(const float *__restrict__ qemb, int64_t nq, const float *__restrict__ cent, int K,
                 const int64_t *__restrict__ offsets, int n_probe, int32_t *__restrict__ probe_out,
                 int64_t *__restrict__ scanned)
{
    static_assert(QB <= ST / 32, "one warp per query");
    extern __shared__ float csc[];                   // [QB][K]
    __shared__ __align__(16) float qe[D][QB];        // dimension-major: a dimension's QB values together
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t q0 = (int64_t)blockIdx.x * QB;
    for (int i = tid; i < QB * D; i += ST) {
        const int64_t q = q0 + i / D;
        qe[i % D][i / D] = q < nq ? qemb[q * D + i % D] : 0.f;
    }
    __syncthreads();
    // a thread scores four adjacent centroids for the QB queries (4 x QB
    // accumulators, one 16-byte load of centroid values per dimension when
    // K is a multiple of 4); the loads run PF dimensions ahead of the FMAs
    // (L2 latency).  Each score is the same FMA chain over the dimensions in
    // order as in ivf_search_kernel.
    constexpr int PF = 8;
    static_assert(D % PF == 0, "whole prefetch groups");
    const bool vec = (K & 3) == 0;
    for (int c0 = 4 * tid; c0 < K; c0 += 4 * ST) {
        auto load4 = [&](int d) {
            const float *row = cent + (int64_t)d * K + c0;
            if (vec) return __ldg(reinterpret_cast<const float4 *>(row));
            return make_float4(__ldg(row), c0 + 1 < K ? __ldg(row + 1) : 0.f,
                               c0 + 2 < K ? __ldg(row + 2) : 0.f, c0 + 3 < K ? __ldg(row + 3) : 0.f);
        };
        float sc[QB][4];
#pragma unroll
        for (int i = 0; i < QB; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) sc[i][j] = 0.f;
        float4 nx[PF];
#pragma unroll
        for (int e = 0; e < PF; ++e) nx[e] = load4(e);
        for (int d0 = 0; d0 < D; d0 += PF) {
            float4 cu[PF];
#pragma unroll
            for (int e = 0; e < PF; ++e) cu[e] = nx[e];
            if (d0 + PF < D) {
#pragma unroll
                for (int e = 0; e < PF; ++e) nx[e] = load4(d0 + PF + e);
            }
#pragma unroll
            for (int e = 0; e < PF; ++e) {
                const float w[4] = {cu[e].x, cu[e].y, cu[e].z, cu[e].w};
#pragma unroll
                for (int i = 0; i < QB; ++i) {
                    const float qv = qe[d0 + e][i];
#pragma unroll
                    for (int j = 0; j < 4; ++j) sc[i][j] = fmaf(qv, w[j], sc[i][j]);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < QB; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (c0 + j < K) csc[i * K + c0 + j] = sc[i][j];
    }
    __syncthreads();
    const int64_t q = q0 + wid;
    if (wid >= QB || q >= nq) return;
    const float *sc = csc + (int64_t)wid * K;
    // key of centroid c: larger is better; every key is nonzero, so 0 marks
    // an empty register slot
    auto key_of = [&](int c) {
        uint32_t fb = __float_as_uint(sc[c]);
        fb = (fb & 0x80000000u) ? ~fb : (fb | 0x80000000u);
        return ((unsigned long long)fb << 32) | (0xFFFFFFFFu - (uint32_t)c);
    };
    // this lane's four best keys below `below`, in descending order
    unsigned long long t0, t1, t2, t3;
    auto best4 = [&](unsigned long long below) {
        t0 = t1 = t2 = t3 = 0ull;
        for (int c = lane; c < K; c += 32) {
            unsigned long long x = key_of(c);
            if (x >= below || x <= t3) continue;
            t3 = x;
            if (t3 > t2) { x = t2; t2 = t3; t3 = x; }
            if (t2 > t1) { x = t1; t1 = t2; t2 = x; }
            if (t1 > t0) { x = t0; t0 = t1; t1 = x; }
        }
    };
    best4(~0ull);
    int64_t rows = 0;
    for (int p = 0; p < n_probe; ++p) {
        unsigned long long b = t0;
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long u = __shfl_xor_sync(0xffffffffu, b, o);
            b = u > b ? u : b;
        }
        if (b == t0) {                 // this lane's head was taken (keys are distinct)
            t0 = t1;
            t1 = t2;
            t2 = t3;
            t3 = 0ull;
            if (t0 == 0ull) best4(b);
        }
        const int c = (int)(0xFFFFFFFFu - (uint32_t)(b & 0xFFFFFFFFu));
        if (lane == 0) {
            probe_out[q * n_probe + p] = c;
            rows += offsets[c + 1] - offsets[c];
        }
    }
    if (lane == 0 && scanned) scanned[q] = rows;
}

// ------------------------------------------------ list-major search on the tensor cores
// The (query, probed list) pairs are regrouped by list; each list's rows
// are then scanned once for all the queries that probe it, 128 queries per
// tensor-core tile (launch_tc_units), and every query merges the top-k
// lists of its pairs.
__global__ void pair_count_kernel(const int32_t *__restrict__ probe, int64_t pairs,
                                  int32_t *__restrict__ counts)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; i < pairs; i += stride) atomicAdd(&counts[probe[i]], 1);
}

// One block: per list, ceil(count / 128) query tiles (numbered list by
// list from tile_base) and ceil(tiles / 2) units of up to two tiles each.
__global__ void unit_plan_kernel(const int32_t *__restrict__ counts, int K,
                                 const int64_t *__restrict__ offsets, int64_t *__restrict__ tile_base,
                                 TcUnit *__restrict__ units, int64_t *__restrict__ n_units,
                                 int64_t *__restrict__ n_tiles)
{
    __shared__ uint32_t tmp[33];
    uint32_t run_t = 0, run_u = 0;
    for (int c0 = 0; c0 < K; c0 += blockDim.x) {
        const int c = c0 + threadIdx.x;
        const uint32_t cnt = c < K ? (uint32_t)counts[c] : 0u;
        const uint32_t nt = (cnt + kTcTileM - 1) / kTcTileM;
        const uint32_t nu = (nt + 1) / 2;
        uint32_t tot_t, tot_u;
        const uint32_t bt = block_excl_scan(nt, tmp, &tot_t);
        const uint32_t bu = block_excl_scan(nu, tmp, &tot_u);
        if (c < K) {
            const int64_t t0 = (int64_t)run_t + bt, u0 = (int64_t)run_u + bu;
            tile_base[c] = t0;
            for (uint32_t i = 0; i < nu; ++i) {
                TcUnit u;
                u.row0 = offsets[c];
                u.row1 = offsets[c + 1];
                u.a_tile0 = (int32_t)(t0 + 2 * i);
                u.nvalid0 = (int32_t)min(cnt - 2 * i * kTcTileM, (uint32_t)kTcTileM);
                const bool two = 2 * i + 1 < nt;
                u.a_tile1 = two ? (int32_t)(t0 + 2 * i + 1) : -1;
                u.nvalid1 = two ? (int32_t)min(cnt - (2 * i + 1) * kTcTileM, (uint32_t)kTcTileM) : 0;
                u.out_base = 0;
                units[u0 + i] = u;
            }
        }
        run_t += tot_t;
        run_u += tot_u;
    }
    if (threadIdx.x == 0) {
        *n_units = run_u;
        *n_tiles = run_t;
    }
}

// Pair (q, p) -> a row of one of its list's query tiles.
__global__ void pair_scatter_kernel(const int32_t *__restrict__ probe, int64_t nq, int n_probe,
                                    const int64_t *__restrict__ tile_base, int32_t *__restrict__ fill,
                                    int32_t *__restrict__ slot_q, int64_t *__restrict__ slot_of)
{
    const int64_t pairs = nq * n_probe;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (; i < pairs; i += stride) {
        const int c = probe[i];
        const int r = atomicAdd(&fill[c], 1);
        const int64_t slot = (tile_base[c] + r / kTcTileM) * kTcTileM + r % kTcTileM;
        slot_q[slot] = (int32_t)(i / n_probe);
        slot_of[i] = slot;
    }
}

// One warp per query: merge the lists of its pairs; write idx and score.
__global__ void pair_merge_kernel(const uint64_t *__restrict__ partial,
                                  const int64_t *__restrict__ slot_of, int n_probe,
                                  const uint64_t *__restrict__ qs, int64_t nq, int k,
                                  uint32_t *__restrict__ idx, float *__restrict__ score)
{
    const int lane = threadIdx.x & 31;
    const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (q >= nq) return;
    uint64_t slot = kEmpty;
    for (int p = 0; p < n_probe; ++p) {
        const int64_t sl = slot_of[q * n_probe + p];
        const uint64_t c = lane < k ? partial[sl * k + lane] : kEmpty;
        warp_list_merge(slot, c, k, lane);
    }
    const uint4 qv = __ldg(reinterpret_cast<const uint4 *>(qs + q * kWords) + lane);
    const QueryWeights w = query_weights(warp_sum(popc4(qv)));
    if (lane < k) {
        const int64_t o = q * k + lane;
        if (slot == kEmpty) {
            idx[o] = 0xFFFFFFFFu;
            score[o] = __int_as_float(0x7f800000);
        } else {
            idx[o] = (uint32_t)slot;
            score[o] = key_score(w, (uint32_t)(slot >> 32));
        }
    }
}

__global__ void transpose_centroids_kernel(const float *__restrict__ cent, int K,
                                           float *__restrict__ cent_t)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)K * D) return;
    const int64_t c = i / D, d = i % D;
    cent_t[d * K + c] = cent[i];
}

}  // namespace
}  // namespace dtk

struct dt_ivf {
    int device = 0;
    int64_t n = 0;
    int K = 0;
    float *cent = nullptr;          // [K][128]
    float *cent_t = nullptr;        // [128][K] (search reads it coalesced)
    int64_t *offsets = nullptr;     // [K+1]
    uint64_t *db = nullptr;         // [n][64] cluster order
    uint32_t *ids = nullptr;        // [n] original index
};

using namespace dtk;

extern "C" {

int ivf_build(const dt_encoder *enc, const uint64_t *d_db, int64_t n, int32_t n_lists, int32_t iters,
              void *stream, dt_ivf **out)
{
    DT_CHECK_ARG(enc && d_db && out && n >= 1 && n < (int64_t(1) << 32) && n_lists >= 1 &&
                     n_lists <= n && iters >= 0,
                 "bad arguments");
    *out = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    const int K = n_lists;
    dt_ivf *ix = new dt_ivf();
    cudaGetDevice(&ix->device);
    ix->n = n;
    ix->K = K;
    __nv_bfloat16 *emb = nullptr;
    int32_t *assign = nullptr, *counts = nullptr;
    unsigned long long *sums = nullptr;
    int rc = DT_OK;
    auto fail = [&](const char *what) {
        set_error(std::string("ivf_build: ") + what);
        rc = DT_ECUDA;
    };
    if (dt_malloc_async((void **)&emb, (size_t)n * D * 2, s) != cudaSuccess ||
        dt_malloc_async((void **)&assign, (size_t)n * 4, s) != cudaSuccess ||
        dt_malloc_async((void **)&counts, (size_t)K * 4, s) != cudaSuccess ||
        dt_malloc_async((void **)&sums, (size_t)K * D * 8, s) != cudaSuccess ||
        cudaMalloc((void **)&ix->cent, (size_t)K * D * 4) != cudaSuccess ||
        cudaMalloc((void **)&ix->cent_t, (size_t)K * D * 4) != cudaSuccess ||
        cudaMalloc((void **)&ix->offsets, (size_t)(K + 1) * 8) != cudaSuccess ||
        cudaMalloc((void **)&ix->db, (size_t)n * 512) != cudaSuccess ||
        cudaMalloc((void **)&ix->ids, (size_t)n * 4) != cudaSuccess) {
        set_error("ivf_build: allocation failed");
        rc = DT_ENOMEM;
    }
    if (rc == DT_OK) rc = enc_embed(enc, d_db, n, reinterpret_cast<uint16_t *>(emb), nullptr, 0, s);
    if (rc == DT_OK) {
        init_centroids_kernel<<<(unsigned)(((int64_t)K * D + 255) / 256), 256, 0, s>>>(emb, n, K, ix->cent);
        const unsigned ablocks = (unsigned)((n + KT - 1) / KT);
        for (int it = 0; it <= iters; ++it) {
            assign_kernel<<<ablocks, 256, 0, s>>>(emb, n, ix->cent, K, assign);
            if (it == iters) break;
            cudaMemsetAsync(sums, 0, (size_t)K * D * 8, s);
            cudaMemsetAsync(counts, 0, (size_t)K * 4, s);
            accumulate_kernel<<<(unsigned)std::min<int64_t>((n + 7) / 8, 8192), 256, 0, s>>>(emb, n, assign, sums, counts);
            update_kernel<<<(unsigned)((K + 7) / 8), 256, 0, s>>>(sums, counts, K, ix->cent);
        }
        cudaMemsetAsync(counts, 0, (size_t)K * 4, s);
        count_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 8192), 256, 0, s>>>(assign, n, counts);
        offsets_kernel<<<1, 32, 0, s>>>(counts, K, ix->offsets);
        cudaMemsetAsync(counts, 0, (size_t)K * 4, s);
        scatter_kernel<<<(unsigned)std::min<int64_t>((n + 7) / 8, 8192), 256, 0, s>>>(
            d_db, n, assign, ix->offsets, counts, ix->db, ix->ids);
        transpose_centroids_kernel<<<(unsigned)(((int64_t)K * D + 255) / 256), 256, 0, s>>>(
            ix->cent, K, ix->cent_t);
        if (cudaGetLastError() != cudaSuccess) fail("kernel launch");
    }
    cudaFreeAsync(sums, s);
    cudaFreeAsync(counts, s);
    cudaFreeAsync(assign, s);
    cudaFreeAsync(emb, s);
    if (cudaStreamSynchronize(s) != cudaSuccess && rc == DT_OK) fail("stream");
    if (rc != DT_OK) {
        cudaFree(ix->cent); cudaFree(ix->cent_t); cudaFree(ix->offsets); cudaFree(ix->db);
        cudaFree(ix->ids);
        delete ix;
        return rc;
    }
    *out = ix;
    return DT_OK;
}

void ivf_free(dt_ivf *ix)
{
    if (!ix) return;
    cudaDeviceSynchronize();
    cudaFree(ix->cent); cudaFree(ix->cent_t); cudaFree(ix->offsets); cudaFree(ix->db);
    cudaFree(ix->ids);
    delete ix;
}

// List sizes (host copy of the K+1 offsets).
int ivf_offsets(const dt_ivf *ix, int64_t *h_offsets)
{
    DT_CHECK_ARG(ix && h_offsets, "bad arguments");
    DT_CUDA_TRY(cudaMemcpy(h_offsets, ix->offsets, (size_t)(ix->K + 1) * 8, cudaMemcpyDeviceToHost));
    return DT_OK;
}

int ivf_search(const dt_ivf *ix, const dt_encoder *enc, const uint64_t *d_q, int64_t nq, int32_t k,
               int32_t n_probe, uint32_t *d_idx, float *d_score, int64_t *d_scanned, int32_t path,
               void *stream)
{
    DT_CHECK_ARG(ix && enc && d_q && d_idx && d_score && nq >= 0, "bad arguments");
    DT_CHECK_ARG(k >= 1 && k <= DT_MAX_K, "k must be in [1, DT_MAX_K]");
    DT_CHECK_ARG(n_probe >= 1 && n_probe <= MAX_PROBE && n_probe <= ix->K, "n_probe out of range");
    DT_CHECK_ARG(path >= 0 && path <= 2, "path must be 0, 1 or 2");
    DT_CHECK_ARG(nq <= (1LL << 31) / MAX_PROBE, "nq out of range");
    if (nq == 0) return DT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    // the list-major scan multiplies whole 128-query tiles: worth it from
    // about 10 queries per list on average (measured crossover)
    const bool tensor = path == 2 || (path == 0 && nq * n_probe >= 10LL * ix->K);
    Scratch scratch(s);
    float *qemb = nullptr;
    DT_CUDA_TRY(scratch.alloc(&qemb, (size_t)nq * D * 4));
    if (int r = enc_embed(enc, d_q, nq, nullptr, qemb, 0, s)) return r;
    const size_t smem = (size_t)ix->K * 4;
    if (smem > 48 * 1024)
        DT_CUDA_TRY(cudaFuncSetAttribute(ivf_search_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem));
    if (!tensor) {
        ivf_search_kernel<<<(unsigned)nq, ST, smem, s>>>(qemb, d_q, nq, ix->cent_t, ix->K,
                                                         ix->offsets, ix->db, ix->ids, n_probe, k,
                                                         d_idx, d_score, nullptr, d_scanned, nullptr);
        DT_CUDA_TRY(cudaGetLastError());
        return DT_OK;
    }
    // list-major: probes -> pairs grouped by list -> tensor-core units -> merge
    const int64_t pairs = nq * n_probe;
    const int64_t max_tiles = std::min<int64_t>(pairs, (pairs + kTcTileM - 1) / kTcTileM + ix->K);
    const int64_t max_units = max_tiles;
    int32_t *probe = nullptr, *counts = nullptr, *slot_q = nullptr;
    int64_t *tile_base = nullptr, *n_units = nullptr, *slot_of = nullptr;
    TcUnit *units = nullptr;
    uint64_t *partial = nullptr;
    DT_CUDA_TRY(scratch.alloc(&probe, (size_t)pairs * 4));
    DT_CUDA_TRY(scratch.alloc(&counts, (size_t)ix->K * 4 * 2));
    DT_CUDA_TRY(scratch.alloc(&tile_base, (size_t)ix->K * 8));
    DT_CUDA_TRY(scratch.alloc(&n_units, 16));
    DT_CUDA_TRY(scratch.alloc(&units, (size_t)max_units * sizeof(TcUnit)));
    DT_CUDA_TRY(scratch.alloc(&slot_q, (size_t)max_tiles * kTcTileM * 4));
    DT_CUDA_TRY(scratch.alloc(&slot_of, (size_t)pairs * 8));
    DT_CUDA_TRY(scratch.alloc(&partial, (size_t)max_tiles * kTcTileM * k * 8));
    int32_t *fill = counts + ix->K;
    int64_t *n_tiles = n_units + 1;
    DT_CUDA_TRY(cudaMemsetAsync(counts, 0, (size_t)ix->K * 4 * 2, s));
    DT_CUDA_TRY(cudaMemsetAsync(slot_q, 0xFF, (size_t)max_tiles * kTcTileM * 4, s));
    DT_CUDA_TRY(cudaMemsetAsync(partial, 0xFF, (size_t)max_tiles * kTcTileM * k * 8, s));
    {   // probes: up to eight queries per block, as many as their scores fit in shared memory
        const size_t per_q = (size_t)ix->K * 4, room = 200 * 1024;
        const int qb = per_q * 8 <= room ? 8 : per_q * 4 <= room ? 4 : per_q * 2 <= room ? 2 : 1;
        const size_t psmem = (size_t)qb * per_q;
        auto kern = qb == 8 ? ivf_probe_kernel<8> : qb == 4 ? ivf_probe_kernel<4>
                  : qb == 2 ? ivf_probe_kernel<2> : ivf_probe_kernel<1>;
        if (psmem > 48 * 1024)
            DT_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)psmem));
        kern<<<(unsigned)((nq + qb - 1) / qb), ST, psmem, s>>>(qemb, nq, ix->cent_t, ix->K,
                                                               ix->offsets, n_probe, probe, d_scanned);
    }
    const unsigned pb = (unsigned)std::min<int64_t>((pairs + 255) / 256, 8192);
    pair_count_kernel<<<pb, 256, 0, s>>>(probe, pairs, counts);
    unit_plan_kernel<<<1, 1024, 0, s>>>(counts, ix->K, ix->offsets, tile_base, units, n_units,
                                        n_tiles);
    pair_scatter_kernel<<<pb, 256, 0, s>>>(probe, nq, n_probe, tile_base, fill, slot_q, slot_of);
    DT_CUDA_TRY(cudaGetLastError());
    int rc = launch_tc_units(ix->db, ix->n, ix->ids, d_q, slot_q, units, n_units, n_tiles,
                             max_tiles, k, partial, s);
    if (rc == DT_OK) {
        pair_merge_kernel<<<(unsigned)((nq + 7) / 8), 256, 0, s>>>(partial, slot_of, n_probe, d_q,
                                                                   nq, k, d_idx, d_score);
        DT_CUDA_TRY(cudaGetLastError());
    }
    return rc;
}

}  // extern "C"
