// bf_tc.cu — sequential search (§6.2) with the overlap counted on the
// tensor cores.
//
// O[q][t] = popc(q & t) is the dot product of two 0/1 vectors of length
// 4096, i.e. one row of a dense Q x N x 4096 contraction.  Bits are widened
// to FP8 E4M3 (1.0 = 0x38, 0.0 = 0x00) and multiplied by tcgen05.mma
// (kind::f8f6f4) with FP32 accumulation in tensor memory; every partial sum
// is an integer <= 4096 < 2^24, so the result is exact.  The epilogue turns
// O into the Eq. 1 key (A = |q| - O, B = |t| - O) and keeps per-query top-k.
//
// Kernel organisation (one persistent CTA per SM, 9 warps):
//   * warps 4-7 (producers): for each 128-bit K chunk, widen the chunk of
//     256 database descriptors into a 32 KB shared-memory stage (K-major
//     8x16-byte core matrices); the first lane of warp 4 also brings the
//     matching 16 KB chunk of the 128 pre-widened queries with one bulk copy;
//   * warp 8 (one thread): 4 MMAs of 128 x 256 x 32 per chunk into one of two
//     TMEM accumulators (256 columns each), then commits to free the stage;
//   * warps 0-3 (epilogue, one thread per query row = TMEM lane): read the
//     finished accumulator in 32-column slices while the next tile is being
//     multiplied into the other accumulator, rank candidates, keep top-k.
// A four-stage mbarrier ring connects producers and MMA; all waits are
// bounded and a shared abort flag makes every role leave together.
// Work units are (128-query tile, database split); per-split lists are merged
// by the same kernel as the popcount path.
#include <algorithm>
#include <mutex>

#include "dt_internal.cuh"
#include "tc_util.cuh"

namespace dtk {
namespace {

constexpr int TM = 128;                 // queries per tile (MMA M)
constexpr int TN = 256;                 // descriptors per tile (MMA N)
constexpr int KC = 128;                 // K bytes (= bits) per chunk
constexpr int NCHUNK = kBits / KC;      // 32
constexpr int STAGES = 4;
constexpr int A_STAGE = TM * KC;        // 16 KB
constexpr int B_STAGE = TN * KC;        // 32 KB
constexpr uint32_t LBO = 128;           // next core matrix along K
constexpr uint32_t SBO = (KC / 16) * 128;  // next 8-row group (1024 B)
constexpr int EPI_WARPS = 4, PROD_WARPS = 4;
constexpr int THREADS = (EPI_WARPS + PROD_WARPS + 1) * 32;
constexpr uint32_t TMEM_COLS = 512;     // two 256-column FP32 accumulators
constexpr uint32_t IDESC = idesc_e4m3_f32(TM, TN);

struct TcCtl {
    uint64_t full[STAGES];
    uint64_t empty[STAGES];
    uint64_t acc_full[2];
    uint64_t acc_empty[2];
    uint64_t final_bar;
    uint32_t tmem_base;
    volatile uint32_t abort;
};

constexpr size_t SMEM_BYTES = (size_t)STAGES * (A_STAGE + B_STAGE) + sizeof(TcCtl) + 1024;

__device__ uint32_t g_tc_error;  // a bounded wait gave up (DT_ETIMEOUT)

// 4 bits -> 4 E4M3 bytes: byte i = 0x38 if bit i else 0.
__device__ __forceinline__ uint32_t nib_e4m3(uint32_t nib)
{
    return ((nib * 0x00204081u) & 0x01010101u) * 0x38u;
}

// 32 bits -> 32 E4M3 bytes as two 16-byte pieces.
__device__ __forceinline__ void widen32(uint32_t w, uint4 &lo, uint4 &hi)
{
    lo = make_uint4(nib_e4m3(w & 15u), nib_e4m3((w >> 4) & 15u), nib_e4m3((w >> 8) & 15u),
                    nib_e4m3((w >> 12) & 15u));
    hi = make_uint4(nib_e4m3((w >> 16) & 15u), nib_e4m3((w >> 20) & 15u),
                    nib_e4m3((w >> 24) & 15u), nib_e4m3(w >> 28));
}

// Byte offset of (row, 16-byte piece j of the chunk) in a K-major stage.
__device__ __forceinline__ uint32_t core_off(int row, int j)
{
    return (uint32_t)(row >> 3) * SBO + (uint32_t)j * LBO + (uint32_t)(row & 7) * 16u;
}

// Write 128 bits of one row as 128 E4M3 bytes into a stage.
__device__ __forceinline__ void store_row_chunk(unsigned char *stage, int row, uint4 bits)
{
    const uint32_t w[4] = {bits.x, bits.y, bits.z, bits.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        uint4 lo, hi;
        widen32(w[i], lo, hi);
        *reinterpret_cast<uint4 *>(stage + core_off(row, 2 * i)) = lo;
        *reinterpret_cast<uint4 *>(stage + core_off(row, 2 * i + 1)) = hi;
    }
}

// Queries -> pre-widened tiles a_exp[m_tile][chunk][16 KB stage image], plus |q|.
__global__ void widen_queries_kernel(const uint64_t *__restrict__ q, int64_t nq, int n_mtiles,
                                     unsigned char *__restrict__ a_exp, uint32_t *__restrict__ qpop)
{
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // (m_tile, row, chunk)
    const int64_t total = (int64_t)n_mtiles * TM * NCHUNK;
    if (id >= total) return;
    const int c = (int)(id % NCHUNK);
    const int row = (int)((id / NCHUNK) % TM);
    const int64_t mt = id / ((int64_t)NCHUNK * TM);
    const int64_t qi = mt * TM + row;
    uint4 bits = make_uint4(0, 0, 0, 0);
    if (qi < nq) bits = __ldg(reinterpret_cast<const uint4 *>(q + qi * kWords) + c);
    store_row_chunk(a_exp + ((size_t)mt * NCHUNK + c) * A_STAGE, row, bits);
    if (qi < nq && c == 0) {
        uint32_t s = 0;
        const uint4 *r = reinterpret_cast<const uint4 *>(q + qi * kWords);
        for (int j = 0; j < 32; ++j) {
            uint4 v = __ldg(r + j);
            s += __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
        }
        qpop[qi] = s;
    }
}

// |t| of every database descriptor (warp per row).
__global__ void row_popcount_kernel(const uint64_t *__restrict__ db, int64_t n,
                                    uint32_t *__restrict__ tpop)
{
    const int lane = threadIdx.x & 31;
    int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t stride = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (; r < n; r += stride) {
        uint4 v = __ldg(reinterpret_cast<const uint4 *>(db + r * kWords) + lane);
        uint32_t s = warp_sum(__popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w));
        if (lane == 0) tpop[r] = s;
    }
}

// Bounded wait that also gives up when another role aborted.
__device__ __forceinline__ bool wait_or_abort(uint64_t *bar, uint32_t parity, TcCtl *ctl,
                                              uint32_t *err)
{
    for (uint32_t i = 0; i < kSpinLimit; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (ctl->abort) return false;
    }
    ctl->abort = 1u;
    atomicOr(err, 1u);
    return false;
}

__global__ void __launch_bounds__(THREADS, 1)
bf_tc_kernel(const uint64_t *__restrict__ db, int64_t n, const unsigned char *__restrict__ a_exp,
             const uint32_t *__restrict__ qpop, const uint32_t *__restrict__ tpop, int64_t nq,
             int k, int n_mtiles, int64_t n_ntiles, int64_t tiles_per_split, int n_split,
             uint64_t *__restrict__ partial, uint32_t *err)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        ((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char *stageA = smem;                                   // [STAGES][A_STAGE]
    unsigned char *stageB = smem + (size_t)STAGES * A_STAGE;        // [STAGES][B_STAGE]
    TcCtl *ctl = reinterpret_cast<TcCtl *>(smem + (size_t)STAGES * (A_STAGE + B_STAGE));

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&ctl->full[s], 1 + PROD_WARPS);   // A bytes + one arrival per producer warp
            mbar_init(&ctl->empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&ctl->acc_full[a], 1);
            mbar_init(&ctl->acc_empty[a], EPI_WARPS);
        }
        mbar_init(&ctl->final_bar, 1);
        ctl->abort = 0u;
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(&ctl->tmem_base, TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = ctl->tmem_base;

    const int64_t total_units = (int64_t)n_mtiles * n_split;

    if (warp >= EPI_WARPS && warp < EPI_WARPS + PROD_WARPS) {
        // ------------------------------------------------ producers
        const int pw = warp - EPI_WARPS;
        uint32_t g = 0;
        for (int64_t u = blockIdx.x; u < total_units; u += gridDim.x) {
            const int64_t mt = u % n_mtiles, sp = u / n_mtiles;
            const int64_t t0 = sp * tiles_per_split, t1 = min(n_ntiles, t0 + tiles_per_split);
            for (int64_t nt = t0; nt < t1; ++nt) {
                for (int c = 0; c < NCHUNK; ++c, ++g) {
                    const int s = (int)(g % STAGES);
                    const uint32_t r = g / STAGES;
                    bool ok = true;
                    if (lane == 0) ok = wait_or_abort(&ctl->empty[s], (r & 1u) ^ 1u, ctl, err);
                    ok = __shfl_sync(0xffffffffu, ok, 0);
                    if (!ok) goto done;
                    if (pw == 0 && lane == 0) {
                        mbar_arrive_expect_tx(&ctl->full[s], (uint32_t)A_STAGE);
                        bulk_g2s(stageA + (size_t)s * A_STAGE,
                                 a_exp + ((size_t)mt * NCHUNK + c) * A_STAGE, (uint32_t)A_STAGE,
                                 &ctl->full[s]);
                    }
                    unsigned char *B = stageB + (size_t)s * B_STAGE;
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        const int row = pw * 64 + i * 32 + lane;
                        const int64_t t = nt * TN + row;
                        uint4 bits = make_uint4(0, 0, 0, 0);
                        if (t < n) bits = __ldg(reinterpret_cast<const uint4 *>(db + t * kWords) + c);
                        store_row_chunk(B, row, bits);
                    }
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&ctl->full[s]);
                }
            }
        }
    } else if (warp == EPI_WARPS + PROD_WARPS) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            uint32_t g = 0, t = 0;
            for (int64_t u = blockIdx.x; u < total_units && !ctl->abort; u += gridDim.x) {
                const int64_t sp = u / n_mtiles;
                const int64_t t0 = sp * tiles_per_split, t1 = min(n_ntiles, t0 + tiles_per_split);
                for (int64_t nt = t0; nt < t1; ++nt, ++t) {
                    const uint32_t acc = t & 1u, ra = t >> 1;
                    if (!wait_or_abort(&ctl->acc_empty[acc], (ra & 1u) ^ 1u, ctl, err)) goto mma_done;
                    tc_fence_after();
                    const uint32_t d_tmem = tmem + acc * (uint32_t)TN;
                    for (int c = 0; c < NCHUNK; ++c, ++g) {
                        const int s = (int)(g % STAGES);
                        const uint32_t r = g / STAGES;
                        if (!wait_or_abort(&ctl->full[s], r & 1u, ctl, err)) goto mma_done;
                        tc_fence_after();
                        const uint32_t a_base = smem_u32(stageA + (size_t)s * A_STAGE);
                        const uint32_t b_base = smem_u32(stageB + (size_t)s * B_STAGE);
#pragma unroll
                        for (int kk = 0; kk < KC / 32; ++kk) {
                            const uint64_t ad = smem_desc_kmajor(a_base + kk * 2 * LBO, LBO, SBO);
                            const uint64_t bd = smem_desc_kmajor(b_base + kk * 2 * LBO, LBO, SBO);
                            mma_e4m3(d_tmem, ad, bd, IDESC, (c | kk) != 0 ? 1u : 0u);
                        }
                        mma_commit(&ctl->empty[s]);
                    }
                    mma_commit(&ctl->acc_full[acc]);
                }
            }
        mma_done:
            mma_commit(&ctl->final_bar);          // every MMA issued here has completed
            wait_or_abort(&ctl->final_bar, 0u, ctl, err);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------ epilogue (warps 0-3)
        const int row = warp * 32 + lane;            // TMEM lane = query row of the tile
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        uint64_t L[kMaxK];
        uint32_t t = 0;
        for (int64_t u = blockIdx.x; u < total_units; u += gridDim.x) {
            const int64_t mt = u % n_mtiles, sp = u / n_mtiles;
            const int64_t t0 = sp * tiles_per_split, t1 = min(n_ntiles, t0 + tiles_per_split);
            const int64_t qi = mt * TM + row;
            const QueryWeights w = query_weights(qi < nq ? qpop[qi] : 0u);
            for (int j = 0; j < k; ++j) L[j] = kEmpty;
            uint64_t worst = kEmpty;
            for (int64_t nt = t0; nt < t1; ++nt, ++t) {
                const uint32_t acc = t & 1u, ra = t >> 1;
                bool ok = true;
                if (lane == 0) ok = wait_or_abort(&ctl->acc_full[acc], ra & 1u, ctl, err);
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) goto done;
                tc_fence_after();
                const int64_t base = nt * TN;
                for (int cb = 0; cb < TN / 32; ++cb) {
                    uint32_t v[32];
                    tmem_ld_32x32b_x32(lane_base + acc * (uint32_t)TN + cb * 32, v);
                    tmem_ld_wait();
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int64_t ti = base + cb * 32 + j;
                        if (ti >= n) break;
                        // exact integer held in an FP32: add 2^23, read the mantissa
                        const uint32_t o = __float_as_uint(__uint_as_float(v[j]) + 8388608.0f) - 0x4B000000u;
                        const uint64_t cand = pack(pair_key(w, o, __ldg(tpop + ti)), (uint32_t)ti);
                        if (cand < worst) {
                            int p = k - 1;
                            while (p > 0 && L[p - 1] > cand) {
                                L[p] = L[p - 1];
                                --p;
                            }
                            L[p] = cand;
                            worst = L[k - 1];
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&ctl->acc_empty[acc]);
            }
            if (qi < nq)
                for (int j = 0; j < k; ++j) partial[((int64_t)sp * nq + qi) * k + j] = L[j];
        }
    }
done:
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, TMEM_COLS);
    }
}

}  // namespace

int take_tc_error(bool *raised)
{
    uint32_t v = 0, zero = 0;
    DT_CUDA_TRY(cudaMemcpyFromSymbol(&v, g_tc_error, sizeof(v)));
    if (v) DT_CUDA_TRY(cudaMemcpyToSymbol(g_tc_error, &zero, sizeof(zero)));
    *raised = v != 0;
    return DT_OK;
}

int launch_bf_tc(const uint64_t *db, int64_t n, const uint64_t *q, int64_t nq, int k,
                 uint32_t *idx, float *score, uint16_t *ab, cudaStream_t s)
{
    static std::once_flag attr_once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(attr_once, [] {
        attr_err = cudaFuncSetAttribute(bf_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)SMEM_BYTES);
    });
    DT_CUDA_TRY(attr_err);
    const int n_mtiles = (int)((nq + TM - 1) / TM);
    const int64_t n_ntiles = (n + TN - 1) / TN;
    const int sms = sm_count();
    const int splits = pick_bf_splits(n_mtiles, n_ntiles, sms);
    const int64_t tiles_per_split = (n_ntiles + splits - 1) / splits;
    const int n_split = (int)((n_ntiles + tiles_per_split - 1) / tiles_per_split);
    const int64_t units = (int64_t)n_mtiles * n_split;
    const int grid = (int)std::min<int64_t>(units, sms);

    unsigned char *a_exp = nullptr;
    uint32_t *qpop = nullptr, *tpop = nullptr, *err = nullptr;
    uint64_t *partial = nullptr;
    const size_t a_bytes = (size_t)n_mtiles * NCHUNK * A_STAGE;
    DT_CUDA_TRY(cudaMallocAsync((void **)&a_exp, a_bytes, s));
    DT_CUDA_TRY(cudaMallocAsync((void **)&qpop, (size_t)nq * 4, s));
    DT_CUDA_TRY(cudaMallocAsync((void **)&tpop, (size_t)n * 4, s));
    DT_CUDA_TRY(cudaMallocAsync((void **)&partial, (size_t)n_split * nq * k * 8, s));
    DT_CUDA_TRY(cudaGetSymbolAddress((void **)&err, g_tc_error));
    {
        const int64_t items = (int64_t)n_mtiles * TM * NCHUNK;
        widen_queries_kernel<<<(unsigned)((items + 255) / 256), 256, 0, s>>>(q, nq, n_mtiles, a_exp, qpop);
        row_popcount_kernel<<<(unsigned)std::min<int64_t>((n + 7) / 8, 32 * 152), 256, 0, s>>>(db, n, tpop);
        DT_CUDA_TRY(cudaGetLastError());
    }
    bf_tc_kernel<<<grid, THREADS, SMEM_BYTES, s>>>(db, n, a_exp, qpop, tpop, nq, k, n_mtiles,
                                                   n_ntiles, tiles_per_split, n_split, partial, err);
    DT_CUDA_TRY(cudaGetLastError());
    int rc = launch_merge_partials(partial, n_split, db, q, nq, k, idx, score, ab, s);
    cudaFreeAsync(partial, s);
    cudaFreeAsync(tpop, s);
    cudaFreeAsync(qpop, s);
    cudaFreeAsync(a_exp, s);
    return rc;
}

}  // namespace dtk
