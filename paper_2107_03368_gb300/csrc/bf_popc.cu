// bf_popc.cu — sequential (brute-force) search of §6.2 on CUDA cores.
//
// For each query/database pair the overlap O = popc(q & t) is counted over
// the 4096 bits; with A = |q| - O and B = |t| - O (the type A and type B
// errors of Eq. 1) the pair's exact rank key is A*Z + B*P.  Each query keeps
// its k smallest (key, index) pairs.
//
// Layout and schedule
//   * A CTA owns a block of 64 queries (staged once in shared memory) and a
//     contiguous range of database tiles (64 descriptors = 32 KB each).
//     Tiles are brought in by the bulk-copy (TMA) engine, double buffered,
//     one 512-byte row per cp.async.bulk into a 528-byte padded row so that
//     the 128-bit shared loads of eight threads hit 32 distinct banks.
//   * 256 threads; thread (tq, tt) computes the 4 x 4 pairs of queries
//     tq + 16i and descriptors tt + 16j, 128 bits per step: 8 LDS.128 feed
//     64 AND + 64 POPC.  The kernel is bound by the POPC pipe.
//   * Per query, a sorted top-k list lives in shared memory; the 16 threads
//     that own the query insert candidates that beat its k-th entry.
//   * The grid is (query blocks) x (database splits) with the query block
//     fastest, so every CTA of one split streams the same tiles together and
//     the database is read from HBM about once per split wave.  A second
//     kernel merges the per-split lists and writes idx / score / (A, B).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <mutex>
#include <vector>

#include "dt_internal.cuh"
#include "ptx_util.cuh"

namespace dtk {
namespace {

constexpr int QB = 64;           // queries per CTA
constexpr int TB = 64;           // database descriptors per tile
constexpr int ROW = 132;         // padded row, uint32 words (528 B)
constexpr int THREADS = 256;

struct BfSmem {
    uint32_t q[QB * ROW];
    uint32_t t[2][TB * ROW];
    uint32_t tpop[2][TB];
    uint32_t qpop[QB];
    uint64_t bar[2];
    // followed by uint64 lists[QB * k]
};

// Set when a tile copy did not arrive within the spin limit (DT_ETIMEOUT).
__device__ uint32_t g_bf_error;

__global__ void __launch_bounds__(THREADS, 2)
bf_popc_kernel(const uint64_t *__restrict__ db, int64_t n, const uint64_t *__restrict__ qs,
               int64_t nq, int k, int64_t tiles_per_split, uint64_t *__restrict__ partial,
               uint32_t *err, uint32_t spin_limit = kSpinLimit, int drop_rel_tile = -1)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    BfSmem &sm = *reinterpret_cast<BfSmem *>(smem_raw);
    uint64_t *lists = reinterpret_cast<uint64_t *>(smem_raw + sizeof(BfSmem));

    const int tid = threadIdx.x, lane = tid & 31;
    const int tq = tid >> 4, tt = tid & 15;
    const int64_t q0 = (int64_t)blockIdx.x * QB;
    const int64_t n_tiles = (n + TB - 1) / TB;
    const int64_t tile_begin = (int64_t)blockIdx.y * tiles_per_split;
    const int64_t tile_end = min(n_tiles, tile_begin + tiles_per_split);
    const int64_t n_split = (int64_t)gridDim.y;

    // queries -> shared (zero rows past nq), lists -> empty
    for (int i = tid; i < QB * 32; i += THREADS) {
        int r = i >> 5, c = i & 31;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (q0 + r < nq) v = reinterpret_cast<const uint4 *>(qs + (q0 + r) * kWords)[c];
        *reinterpret_cast<uint4 *>(&sm.q[r * ROW + 4 * c]) = v;
    }
    for (int i = tid; i < QB * k; i += THREADS) lists[i] = kEmpty;
    if (tid == 0) {
        mbar_init(&sm.bar[0], 1);
        mbar_init(&sm.bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid < QB) {
        uint32_t s = 0;
        for (int c = 0; c < 128; ++c) s += __popc(sm.q[tid * ROW + c]);
        sm.qpop[tid] = s;
    }

    auto issue = [&](int64_t tile, int buf) {
        if (tile - tile_begin == drop_rel_tile) return;   // test hook: a copy that never comes
        int64_t base = tile * TB;
        int rows = (int)(n - base < (int64_t)TB ? n - base : (int64_t)TB);
        mbar_arrive_expect_tx(&sm.bar[buf], (uint32_t)rows * 512u);
        for (int r = 0; r < rows; ++r)
            bulk_g2s(&sm.t[buf][r * ROW], db + (base + r) * kWords, 512u, &sm.bar[buf]);
    };

    if (tid == 0 && tile_begin < tile_end) issue(tile_begin, 0);
    __syncthreads();

    QueryWeights w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) w[i] = query_weights(sm.qpop[tq + 16 * i]);
    const uint32_t half_mask = (lane < 16) ? 0x0000ffffu : 0xffff0000u;

    for (int64_t tile = tile_begin, it = 0; tile < tile_end; ++tile, ++it) {
        const int buf = (int)(it & 1);
        if (tid == 0 && tile + 1 < tile_end) issue(tile + 1, buf ^ 1);
        const bool arrived = mbar_wait(&sm.bar[buf], (uint32_t)((it >> 1) & 1), spin_limit);
        if (__syncthreads_or(!arrived)) {      // give up together, after our copies land
            if (tid == 0) {
                atomicOr(err, 1u);
                // A copy that was issued but is only slow could still write
                // shared memory after the block exits: wait for it again
                // (bounded), and for the next tile's copy issued above.
                if (tile - tile_begin != drop_rel_tile)
                    mbar_wait(&sm.bar[buf], (uint32_t)((it >> 1) & 1));
                if (tile + 1 < tile_end) mbar_wait(&sm.bar[buf ^ 1], (uint32_t)(((it + 1) >> 1) & 1));
            }
            return;
        }
        const uint32_t *T = sm.t[buf];
        // |t| of the 64 rows: 4 threads per row, staggered to spread banks
        {
            int r = tid >> 2, p = tid & 3;
            uint32_t s = 0;
#pragma unroll
            for (int v = 0; v < 8; ++v) {
                int vv = (v + p) & 7;
                uint4 x = *reinterpret_cast<const uint4 *>(&T[r * ROW + p * 32 + vv * 4]);
                s += __popc(x.x) + __popc(x.y) + __popc(x.z) + __popc(x.w);
            }
            s += __shfl_xor_sync(0xffffffffu, s, 1);
            s += __shfl_xor_sync(0xffffffffu, s, 2);
            if (p == 0) sm.tpop[buf][r] = s;
        }
        uint32_t acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0;
#pragma unroll 4
        for (int s = 0; s < 32; ++s) {
            uint4 qv[4], tv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
                qv[i] = *reinterpret_cast<const uint4 *>(&sm.q[(tq + 16 * i) * ROW + 4 * s]);
#pragma unroll
            for (int j = 0; j < 4; ++j)
                tv[j] = *reinterpret_cast<const uint4 *>(&T[(tt + 16 * j) * ROW + 4 * s]);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    acc[i][j] += __popc(qv[i].x & tv[j].x) + __popc(qv[i].y & tv[j].y) +
                                 __popc(qv[i].z & tv[j].z) + __popc(qv[i].w & tv[j].w);
        }
        __syncthreads();  // tpop visible
        const int64_t base = tile * TB;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int qi = tq + 16 * i;
            uint64_t *L = lists + qi * k;
            uint64_t cand[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                int64_t t = base + tt + 16 * j;
                cand[j] = (t < n) ? pack(pair_key(w[i], acc[i][j], sm.tpop[buf][tt + 16 * j]),
                                         (uint32_t)t)
                                  : kEmpty;
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                uint64_t c = cand[j];
                for (;;) {
                    uint64_t thr = L[k - 1];
                    unsigned m = __ballot_sync(half_mask, c < thr) & half_mask;
                    if (!m) break;
                    if (lane == __ffs(m) - 1) {
                        int p = k - 1;
                        while (p > 0 && L[p - 1] > c) {
                            L[p] = L[p - 1];
                            --p;
                        }
                        L[p] = c;
                        c = kEmpty;
                    }
                    __syncwarp(half_mask);
                }
            }
        }
        __syncthreads();  // buffer `buf` and lists free for the next round
    }
    // partial[split][q][k]
    for (int i = tid; i < QB * k; i += THREADS) {
        int qi = i / k, j = i % k;
        if (q0 + qi < nq) partial[((int64_t)blockIdx.y * nq + q0 + qi) * k + j] = lists[i];
    }
    (void)n_split;
}

// One warp per query: merge the split lists, then write idx, score, (A, B).
__global__ void bf_merge_kernel(const uint64_t *__restrict__ partial, int n_split,
                                const uint64_t *__restrict__ db, int64_t n, const uint64_t *__restrict__ qs,
                                int64_t nq, int k, uint32_t *__restrict__ idx,
                                float *__restrict__ score, uint16_t *__restrict__ ab)
{
    const int lane = threadIdx.x & 31;
    const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (q >= nq) return;
    uint64_t slot = kEmpty;
    for (int s = 0; s < n_split; ++s) {
        uint64_t c = lane < k ? partial[((int64_t)s * nq + q) * k + lane] : kEmpty;
        if (c != kEmpty && (int64_t)(uint32_t)c >= n) c = kEmpty;   // never index past the database
        warp_list_merge(slot, c, k, lane);
    }
    // |q| with the warp, 16 bytes a lane
    const uint4 qv = reinterpret_cast<const uint4 *>(qs + q * kWords)[lane];
    uint32_t qp = warp_sum(__popc(qv.x) + __popc(qv.y) + __popc(qv.z) + __popc(qv.w));
    QueryWeights w = query_weights(qp);
    for (int j = 0; j < k; ++j) {
        uint64_t v = shfl_u64(slot, j);
        uint32_t o = 0, tp = 0;
        if (v != kEmpty) {
            const uint4 tv = reinterpret_cast<const uint4 *>(db + (int64_t)(uint32_t)v * kWords)[lane];
            o = warp_sum(__popc(qv.x & tv.x) + __popc(qv.y & tv.y) + __popc(qv.z & tv.z) +
                         __popc(qv.w & tv.w));
            tp = warp_sum(__popc(tv.x) + __popc(tv.y) + __popc(tv.z) + __popc(tv.w));
        }
        if (lane == 0) {
            const int64_t o_ = q * k + j;
            if (v == kEmpty) {
                idx[o_] = 0xFFFFFFFFu;
                score[o_] = __int_as_float(0x7f800000);
                if (ab) ab[2 * o_] = ab[2 * o_ + 1] = 0xFFFF;
            } else {
                uint32_t key = (uint32_t)(v >> 32);
                idx[o_] = (uint32_t)v;
                score[o_] = key_score(w, key);
                if (ab) {
                    ab[2 * o_] = (uint16_t)(qp - o);
                    ab[2 * o_ + 1] = (uint16_t)(tp - o);
                }
            }
        }
    }
}

int pick_splits(int64_t qblocks, int64_t tiles, int concurrent)
{
    int best = 1;
    double best_eff = -1.0;
    int max_s = (int)std::min<int64_t>(tiles, 512);
    for (int s = 1; s <= max_s; ++s) {
        double ctas = (double)qblocks * s;
        double waves = ctas / concurrent;
        double eff = waves / std::ceil(waves);
        // prefer at least two waves for tail balance, and then fewer splits
        if (waves >= 2.0 && eff >= 0.92) return s;
        if (eff > best_eff + 1e-9 && waves >= 1.0) {
            best_eff = eff;
            best = s;
        }
    }
    return best;
}

}  // namespace

int pick_bf_splits(int64_t row_blocks, int64_t tiles, int concurrent)
{
    return pick_splits(row_blocks, tiles, concurrent);
}

int launch_merge_partials(const uint64_t *partial, int n_split, const uint64_t *db, int64_t n,
                          const uint64_t *q, int64_t nq, int k, uint32_t *idx, float *score,
                          uint16_t *ab, cudaStream_t s)
{
    const int wpb = 8;
    bf_merge_kernel<<<(unsigned)((nq + wpb - 1) / wpb), wpb * 32, 0, s>>>(partial, n_split, db, n,
                                                                           q, nq, k, idx, score, ab);
    DT_CUDA_TRY(cudaGetLastError());
    return DT_OK;
}

int take_bf_error(bool *raised)
{
    uint32_t v = 0, zero = 0;
    DT_CUDA_TRY(cudaMemcpyFromSymbol(&v, g_bf_error, sizeof(v)));
    if (v) DT_CUDA_TRY(cudaMemcpyToSymbol(g_bf_error, &zero, sizeof(zero)));
    *raised = v != 0;
    return DT_OK;
}

int launch_bf_popc(const uint64_t *db, int64_t n, const uint64_t *q, int64_t nq, int k,
                   uint32_t *idx, float *score, uint16_t *ab, cudaStream_t s)
{
    return launch_bf_popc_cfg(db, n, q, nq, k, idx, score, ab, s, nullptr);
}

// Test hook (dt_debug_inject_missing_copy): the next popcount launches skip
// the copy of each CTA's first tile and give up waiting for it after a few
// thousand polls, so the timeout path runs and reports DT_ETIMEOUT.
static std::atomic<int> g_drop_copy{0};

int launch_bf_popc_cfg(const uint64_t *db, int64_t n, const uint64_t *q, int64_t nq, int k,
                       uint32_t *idx, float *score, uint16_t *ab, cudaStream_t s,
                       const TuneCfg *cfg)
{
    const size_t smem = sizeof(BfSmem) + (size_t)QB * k * sizeof(uint64_t);
    DT_CUDA_TRY(allow_smem((const void *)bf_popc_kernel,
                           (int)(sizeof(BfSmem) + QB * kMaxK * sizeof(uint64_t))));
    const int64_t qblocks = (nq + QB - 1) / QB;
    const int64_t tiles = (n + TB - 1) / TB;
    int per_sm = 0;
    DT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bf_popc_kernel, THREADS, smem));
    const int concurrent = std::max(1, per_sm) * sm_count();
    TuneCfg c{0, 0};
    if (cfg) c = *cfg;
    else tune_lookup(TUNE_POPC, n, nq, k, &c);
    const int splits = c.a > 0 ? (int)std::min<int64_t>(c.a, tiles) : pick_splits(qblocks, tiles, concurrent);
    const int64_t tiles_per_split = (tiles + splits - 1) / splits;
    const int n_split = (int)((tiles + tiles_per_split - 1) / tiles_per_split);

    Scratch scratch(s);
    uint64_t *partial = nullptr;
    uint32_t *err = nullptr;
    DT_CUDA_TRY(scratch.alloc(&partial, (size_t)n_split * nq * k * sizeof(uint64_t)));
    // every list starts empty, so a block that gives up leaves valid (empty) lists
    DT_CUDA_TRY(cudaMemsetAsync(partial, 0xFF, (size_t)n_split * nq * k * sizeof(uint64_t), s));
    DT_CUDA_TRY(cudaGetSymbolAddress((void **)&err, g_bf_error));
    dim3 grid((unsigned)qblocks, (unsigned)n_split);
    const bool drop = g_drop_copy.load() != 0;
    {
        KernelTimer timer("popc_scan", s);
        bf_popc_kernel<<<grid, THREADS, smem, s>>>(db, n, q, nq, k, tiles_per_split, partial, err,
                                                   drop ? 4096u : kSpinLimit, drop ? 0 : -1);
    }
    DT_CUDA_TRY(cudaGetLastError());
    const int wpb = 8;
    bf_merge_kernel<<<(unsigned)((nq + wpb - 1) / wpb), wpb * 32, 0, s>>>(partial, n_split, db, n,
                                                                           q, nq, k, idx, score, ab);
    DT_CUDA_TRY(cudaGetLastError());
    return DT_OK;
}

void set_drop_copy(bool on) { g_drop_copy.store(on ? 1 : 0); }

// ---------------------------------------------------------------------------
// Brute force without any allocation (bf_search_noalloc).
//
// The only scratch the brute force needs is the per-split top-k lists that
// the merge kernel combines.  Here they live in one fixed array compiled into
// the library, so the call makes no cudaMalloc / cudaMallocAsync / cudaFree.
// The array is shared by every call on a device; each call first fills the
// lists it uses with the empty pattern (a stream-ordered memset), so a block
// that gives up on a wait still leaves valid lists for the merge.  Two calls
// whose work overlaps on the GPU (different streams, no ordering between
// them) use the same array and race.
// ---------------------------------------------------------------------------
namespace {

static __device__ __align__(256) uint64_t g_noalloc_partial[DT_NOALLOC_SCRATCH_BYTES / 8];

struct NoallocDevice {
    bool ready = false;
    uint64_t *partial = nullptr;   // device address of g_noalloc_partial
    uint32_t *err = nullptr;       // device address of g_bf_error
};

std::mutex g_noalloc_mu;
NoallocDevice g_noalloc_dev[64];

// Per-device set-up on the current device: resolve the device addresses of
// the static arrays (a host-side name of a __device__ array is not a device
// address) and set the kernel's shared-memory limit.
int noalloc_setup(NoallocDevice **out)
{
    int dev = 0;
    DT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        set_error("bf_search_noalloc: device ordinal out of range");
        return DT_EUNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoallocDevice &d = g_noalloc_dev[dev];
    if (!d.ready) {
        void *p = nullptr, *e = nullptr;
        DT_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_partial));
        DT_CUDA_TRY(cudaGetSymbolAddress(&e, g_bf_error));
        DT_CUDA_TRY(allow_smem((const void *)bf_popc_kernel,
                               (int)(sizeof(BfSmem) + QB * kMaxK * sizeof(uint64_t))));
        d.partial = static_cast<uint64_t *>(p);
        d.err = static_cast<uint32_t *>(e);
        d.ready = true;
    }
    *out = &d;
    return DT_OK;
}

}  // namespace

int launch_bf_popc_noalloc(const uint64_t *db, int64_t n, const uint64_t *q, int64_t nq, int k,
                           uint32_t *idx, float *score, uint16_t *ab, cudaStream_t s)
{
    const uint64_t list_bytes = (uint64_t)nq * (uint64_t)k * sizeof(uint64_t);
    if (list_bytes > DT_NOALLOC_SCRATCH_BYTES) {
        set_error("bf_search_noalloc: nq * k * 8 bytes exceeds the fixed scratch of "
                  "DT_NOALLOC_SCRATCH_BYTES; split the queries into smaller batches");
        return DT_EINVAL;
    }
    NoallocDevice *d = nullptr;
    if (int r = noalloc_setup(&d)) return r;
    const size_t smem = sizeof(BfSmem) + (size_t)QB * k * sizeof(uint64_t);
    const int64_t qblocks = (nq + QB - 1) / QB;
    const int64_t tiles = (n + TB - 1) / TB;
    int per_sm = 0;
    DT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bf_popc_kernel, THREADS, smem));
    const int concurrent = std::max(1, per_sm) * sm_count();
    // as many database splits as the fixed scratch holds lists for
    const int64_t fit = (int64_t)(DT_NOALLOC_SCRATCH_BYTES / list_bytes);
    const int splits = (int)std::max<int64_t>(1, std::min<int64_t>(pick_splits(qblocks, tiles, concurrent), fit));
    const int64_t tiles_per_split = (tiles + splits - 1) / splits;
    const int n_split = (int)((tiles + tiles_per_split - 1) / tiles_per_split);
    dim3 grid((unsigned)qblocks, (unsigned)n_split);
    DT_CUDA_TRY(cudaMemsetAsync(d->partial, 0xFF, (size_t)n_split * list_bytes, s));
    bf_popc_kernel<<<grid, THREADS, smem, s>>>(db, n, q, nq, k, tiles_per_split, d->partial, d->err);
    DT_CUDA_TRY(cudaGetLastError());
    const int wpb = 8;
    bf_merge_kernel<<<(unsigned)((nq + wpb - 1) / wpb), wpb * 32, 0, s>>>(d->partial, n_split, db, n,
                                                                           q, nq, k, idx, score, ab);
    DT_CUDA_TRY(cudaGetLastError());
    return DT_OK;
}

}  // namespace dtk
