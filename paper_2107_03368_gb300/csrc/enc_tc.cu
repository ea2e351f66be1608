// enc_tc.cu — encoder inference on the tensor cores: the two stride-2
// convolutions as implicit GEMMs and the two dense layers as GEMMs, BF16
// operands with FP32 accumulation in tensor memory (tcgen05, kind::f16).
// The network and its parameters are those of encoder.cu; this path rounds
// activations and weights to BF16, so its embeddings agree with the FP32
// path to about 1e-2 (the inverted file stores BF16 embeddings anyway).
//
// Per batch of images:
//   conv1 (CUDA cores; its input is 0/1 pixels) -> a1 [img][32x32 pos][32 ch] BF16
//   conv2: D[img*256 + pos][co] = sum over (tap, ci) of a1[img][in(pos,tap)][ci] W2[co][ci][tap]
//          -> ReLU -> a2 [img][16x16 pos][64 ch] BF16
//   conv3: rows ordered (image, pooled position, member of the 2x2 window) so
//          that a pooling window is four adjacent TMEM lanes; the epilogue adds
//          the bias, applies ReLU and averages the window -> feat [img][1024]
//          BF16 in (pooled position, channel) order
//   fc1:   -> ReLU -> h [img][256] BF16;  fc2: -> z, z / ||z|| -> output
// One kernel template serves the four GEMMs.  A CTA owns 128-row tiles of
// D in turn: 4 producer warps (one row per thread) gather 64-byte K chunks
// (32 BF16) into K-major 8x16-byte core-matrix stages; the matching chunk
// of the weights, laid out beforehand in the same core-matrix order,
// arrives by bulk copy (TMA engine); one thread issues 128 x N x 16 MMAs
// into one of two TMEM accumulators; 4 epilogue warps drain the other one.
// Every wait is bounded; on expiry the roles leave together and a flag is
// raised that dt_sync_status reports.
#include <algorithm>
#include <mutex>

#include "dt_internal.cuh"
#include "encoder_layout.cuh"
#include "tc_util.cuh"

namespace dtk {
namespace {

using namespace enc;

constexpr int TM = 128;                    // rows per tile (MMA M)
constexpr int KE = 32;                     // K elements (BF16) per chunk
constexpr int KB = KE * 2;                 // 64 bytes per row per chunk
constexpr uint32_t LBO = 128;              // next core matrix along K
constexpr uint32_t SBO = (KB / 16) * 128;  // next 8-row group (512 B)
constexpr int STAGES = 6;
constexpr int A_STAGE = TM * KB;           // 8 KB
constexpr int EPI_WARPS = 4, PROD_WARPS = 4;
constexpr int MMA_WARP = EPI_WARPS + PROD_WARPS;
constexpr int THREADS = (MMA_WARP + 1) * 32;

enum Mode { CONV2 = 0, CONV3 = 1, FC1 = 2, FC2 = 3 };

template <int MODE> struct Shape;
template <> struct Shape<CONV2> { static constexpr int N = C2, NCH = 9; };            // K = 9 x 32
template <> struct Shape<CONV3> { static constexpr int N = C3, NCH = 18; };           // K = 9 x 64
template <> struct Shape<FC1> { static constexpr int N = F1, NCH = F0 / KE; };        // K = 1024
template <> struct Shape<FC2> { static constexpr int N = F2, NCH = F1 / KE; };        // K = 256

// Instruction descriptor, kind::f16: FP32 D [4,6) = 1, BF16 A [7,10) = 1 and
// B [10,13) = 1, both K-major, N >> 3 at [17,23), M >> 4 at [24,29).
constexpr uint32_t idesc_bf16_f32(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__host__ __device__ constexpr uint32_t core_off(int row, int j)
{
    return (uint32_t)(row >> 3) * SBO + (uint32_t)j * LBO + (uint32_t)(row & 7) * 16u;
}

struct Ctl {
    uint64_t full[STAGES];
    uint64_t empty[STAGES];
    uint64_t acc_full[2];
    uint64_t acc_empty[2];
    uint64_t final_bar;
    uint32_t tmem_base;
    volatile uint32_t abort;
};

__device__ uint32_t g_enc_tc_error;

__device__ __forceinline__ bool wait_or_abort(uint64_t *bar, uint32_t parity, Ctl *ctl)
{
    for (uint32_t i = 0; i < (kSpinLimit >> 4); ++i) {
        if (mbar_try_wait_sleep(bar, parity, 200u)) return true;
        if (ctl->abort) return false;
    }
    ctl->abort = 1u;
    atomicOr(&g_enc_tc_error, 1u);
    return false;
}

__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, Ctl *ctl, int lane)
{
    bool ok = true;
    if (lane == 0) ok = wait_or_abort(bar, parity, ctl);
    return __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
}

struct GemmArgs {
    const __nv_bfloat16 *src;           // activations read by the A gather
    int64_t rows;                       // rows of D
    const unsigned char *wimg;          // weight chunks [NCH][N rows x 64 B], core-matrix order
    const float *bias;                  // [N]
    __nv_bfloat16 *dst;                 // conv2: a2, conv3: feat, fc1: h, fc2: BF16 output (nullable)
    float *dst_f32;                     // fc2: FP32 output (nullable)
};

// 64 bytes of A row gm, chunk c (zeros where the row or the tap falls outside).
template <int MODE>
__device__ __forceinline__ void gather(const GemmArgs &a, int64_t gm, int c, uint4 (&v)[4])
{
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = make_uint4(0, 0, 0, 0);
    if (gm >= a.rows) return;
    const __nv_bfloat16 *p = nullptr;
    if (MODE == CONV2) {                 // row = (img, y, x) of the 16x16 output; chunk = tap
        const int64_t img = gm / (H2 * H2);
        const int pos = (int)(gm % (H2 * H2)), y = pos / H2, x = pos % H2;
        const int iy = 2 * y + c / 3 - 1, ix = 2 * x + c % 3 - 1;
        if (iy < 0 || ix < 0 || iy >= H1 || ix >= H1) return;
        p = a.src + ((img * H1 * H1) + iy * H1 + ix) * C1;
    } else if (MODE == CONV3) {          // row = (img, pooled position, window member); chunk = (tap, half of ci)
        const int64_t img = gm / (H3 * H3);
        const int r = (int)(gm % (H3 * H3)), pp = r >> 2, sub = r & 3;
        const int y = 2 * (pp / HP) + (sub >> 1), x = 2 * (pp % HP) + (sub & 1);
        const int tap = c >> 1;
        const int iy = 2 * y + tap / 3 - 1, ix = 2 * x + tap % 3 - 1;
        if (iy < 0 || ix < 0 || iy >= H2 || ix >= H2) return;
        p = a.src + ((img * H2 * H2) + iy * H2 + ix) * C2 + (c & 1) * KE;
    } else if (MODE == FC1) {
        p = a.src + gm * F0 + c * KE;
    } else {
        p = a.src + gm * F1 + c * KE;
    }
    const uint4 *q = reinterpret_cast<const uint4 *>(p);
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = __ldg(q + j);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&h);
}

template <int MODE>
__global__ void __launch_bounds__(THREADS, 1) enc_gemm_kernel(const GemmArgs args)
{
    constexpr int N = Shape<MODE>::N, NCH = Shape<MODE>::NCH;
    constexpr int B_STAGE = N * KB;
    constexpr int STAGE = A_STAGE + B_STAGE;
    constexpr uint32_t TMEM_COLS = 2 * N < 32 ? 32 : 2 * N;
    constexpr uint32_t IDESC = idesc_bf16_f32(TM, N);
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        ((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    Ctl *ctl = reinterpret_cast<Ctl *>(smem + (size_t)STAGES * STAGE);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&ctl->full[s], 1 + PROD_WARPS);
            mbar_init(&ctl->empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&ctl->acc_full[b], 1);
            mbar_init(&ctl->acc_empty[b], EPI_WARPS);
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
    const int64_t n_tiles = (args.rows + TM - 1) / TM;

    if (warp >= EPI_WARPS && warp < MMA_WARP) {
        // ------------------------------------------------ producers: A rows
        const int row = (warp - EPI_WARPS) * 32 + lane;
        uint32_t g = 0;
        for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
            const int64_t gm = tile * TM + row;
            uint4 nx[4];
            gather<MODE>(args, gm, 0, nx);
            for (int c = 0; c < NCH; ++c, ++g) {
                uint4 cu[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) cu[j] = nx[j];
                if (c + 1 < NCH) gather<MODE>(args, gm, c + 1, nx);   // one chunk ahead
                const int s = (int)(g % STAGES);
                const uint32_t r = g / STAGES;
                if (!warp_wait(&ctl->empty[s], (r & 1u) ^ 1u, ctl, lane)) goto done;
                unsigned char *stage = smem + (size_t)s * STAGE;
                if (warp == EPI_WARPS && lane == 0) {
                    mbar_arrive_expect_tx(&ctl->full[s], (uint32_t)B_STAGE);
                    bulk_g2s(stage + A_STAGE, args.wimg + (size_t)c * B_STAGE, (uint32_t)B_STAGE,
                             &ctl->full[s]);
                }
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    *reinterpret_cast<uint4 *>(stage + core_off(row, j)) = cu[j];
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(&ctl->full[s]);
            }
        }
    } else if (warp == MMA_WARP) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            uint32_t g = 0, t = 0;
            for (int64_t tile = blockIdx.x; tile < n_tiles && !ctl->abort; tile += gridDim.x, ++t) {
                const uint32_t acc = t & 1u, ra = t >> 1;
                if (!wait_or_abort(&ctl->acc_empty[acc], (ra & 1u) ^ 1u, ctl)) goto mma_done;
                tc_fence_after();
                const uint32_t d_tmem = tmem + acc * (uint32_t)N;
                for (int c = 0; c < NCH; ++c, ++g) {
                    const int s = (int)(g % STAGES);
                    const uint32_t r = g / STAGES;
                    if (!wait_or_abort(&ctl->full[s], r & 1u, ctl)) goto mma_done;
                    tc_fence_after();
                    const uint32_t a_base = smem_u32(smem + (size_t)s * STAGE);
                    const uint32_t b_base = a_base + A_STAGE;
#pragma unroll
                    for (int kk = 0; kk < KE / 16; ++kk) {
                        const uint64_t ad = smem_desc_kmajor(a_base + kk * 2 * LBO, LBO, SBO);
                        const uint64_t bd = smem_desc_kmajor(b_base + kk * 2 * LBO, LBO, SBO);
                        mma_bf16(d_tmem, ad, bd, IDESC, (c | kk) != 0 ? 1u : 0u);
                    }
                    mma_commit(&ctl->empty[s]);
                }
                mma_commit(&ctl->acc_full[acc]);
            }
        mma_done:
            mma_commit(&ctl->final_bar);
            wait_or_abort(&ctl->final_bar, 0u, ctl);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------ epilogue: TMEM lane = row
        const int row = warp * 32 + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        uint32_t t = 0;
        for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++t) {
            const uint32_t acc = t & 1u, ra = t >> 1;
            if (!warp_wait(&ctl->acc_full[acc], ra & 1u, ctl, lane)) goto done;
            tc_fence_after();
            const int64_t gm = tile * TM + row;
            const bool valid = gm < args.rows;
            const uint32_t base = lane_base + acc * (uint32_t)N;
            float ss = 0.f;                         // fc2: squared norm of the row
            for (int pass = 0; pass < (MODE == FC2 ? 2 : 1); ++pass) {
                const float inv = pass == 1 ? 1.f / fmaxf(sqrtf(ss), 1e-12f) : 1.f;
                for (int c0 = 0; c0 < N; c0 += 32) {
                    uint32_t v[32];
                    tmem_ld_32x32b_x32(base + c0, v);
                    tmem_ld_wait();
                    float x[32];
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        x[j] = __uint_as_float(v[j]) + __ldg(args.bias + c0 + j);
                        if (MODE != FC2) x[j] = fmaxf(x[j], 0.f);
                    }
                    if (MODE == CONV3) {            // 2x2 average over four adjacent lanes
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            float sum = x[j] + __shfl_xor_sync(0xffffffffu, x[j], 1);
                            sum += __shfl_xor_sync(0xffffffffu, sum, 2);
                            x[j] = 0.25f * sum;
                        }
                    }
                    if (MODE == FC2 && pass == 0) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) ss += x[j] * x[j];
                        continue;
                    }
                    if (!valid) continue;
                    if (MODE == CONV3 && (lane & 3) != 0) continue;
                    if (MODE == FC2) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) x[j] *= inv;
                        if (args.dst_f32) {
                            float4 *o = reinterpret_cast<float4 *>(args.dst_f32 + gm * N + c0);
#pragma unroll
                            for (int j = 0; j < 8; ++j)
                                o[j] = make_float4(x[4 * j], x[4 * j + 1], x[4 * j + 2], x[4 * j + 3]);
                        }
                        if (!args.dst) continue;
                    }
                    __nv_bfloat16 *dst;
                    if (MODE == CONV3) {
                        const int64_t img = gm / (H3 * H3);
                        const int pp = (int)(gm % (H3 * H3)) >> 2;
                        dst = args.dst + img * F0 + pp * C3 + c0;
                    } else {
                        dst = args.dst + gm * N + c0;
                    }
                    uint4 *o = reinterpret_cast<uint4 *>(dst);
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        o[j] = make_uint4(pack_bf16x2(x[8 * j], x[8 * j + 1]),
                                          pack_bf16x2(x[8 * j + 2], x[8 * j + 3]),
                                          pack_bf16x2(x[8 * j + 4], x[8 * j + 5]),
                                          pack_bf16x2(x[8 * j + 6], x[8 * j + 7]));
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&ctl->acc_empty[acc]);
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

template <int MODE> constexpr size_t gemm_smem()
{
    return (size_t)STAGES * (A_STAGE + Shape<MODE>::N * KB) + sizeof(Ctl) + 1024;
}

// conv1 on CUDA cores: a block per image in turn, 4 positions per thread,
// 32 channels in registers, ReLU, BF16 out in [pos][ch] order.
__global__ void __launch_bounds__(256)
conv1_nhwc_kernel(const uint64_t *__restrict__ bits, int64_t n, const float *__restrict__ P,
                  __nv_bfloat16 *__restrict__ a1)
{
    __shared__ uint64_t img[kWords];
    __shared__ float w[9][C1];                       // [tap][co]
    __shared__ float b[C1];
    for (int i = threadIdx.x; i < 9 * C1; i += blockDim.x)
        w[i % 9][i / 9] = P[OW1 + i];                 // P[OW1 + co * 9 + tap]
    if (threadIdx.x < C1) b[threadIdx.x] = P[OB1 + threadIdx.x];
    for (int64_t m = blockIdx.x; m < n; m += gridDim.x) {
        __syncthreads();
        if (threadIdx.x < kWords) img[threadIdx.x] = bits[m * kWords + threadIdx.x];
        __syncthreads();
        for (int p = threadIdx.x; p < H1 * H1; p += blockDim.x) {
            const int y = p / H1, x = p % H1;
            float acc[C1];
#pragma unroll
            for (int co = 0; co < C1; ++co) acc[co] = b[co];
#pragma unroll
            for (int tap = 0; tap < 9; ++tap) {
                const int r = 2 * y + tap / 3 - 1, c = 2 * x + tap % 3 - 1;
                if (r >= 0 && c >= 0 && r < 64 && c < 64 && ((img[r] >> c) & 1ull)) {
#pragma unroll
                    for (int co = 0; co < C1; ++co) acc[co] += w[tap][co];
                }
            }
            uint4 *o = reinterpret_cast<uint4 *>(a1 + ((m * H1 * H1) + p) * C1);
#pragma unroll
            for (int j = 0; j < 4; ++j)
                o[j] = make_uint4(pack_bf16x2(fmaxf(acc[8 * j], 0.f), fmaxf(acc[8 * j + 1], 0.f)),
                                  pack_bf16x2(fmaxf(acc[8 * j + 2], 0.f), fmaxf(acc[8 * j + 3], 0.f)),
                                  pack_bf16x2(fmaxf(acc[8 * j + 4], 0.f), fmaxf(acc[8 * j + 5], 0.f)),
                                  pack_bf16x2(fmaxf(acc[8 * j + 6], 0.f), fmaxf(acc[8 * j + 7], 0.f)));
        }
    }
}

// Weight chunks for the four GEMMs, BF16 in core-matrix order: chunk c of
// a GEMM with N outputs is N rows x 32 K elements; element (n, e) of chunk
// c sits at core_off(n, e / 8) + 2 (e % 8).  K orders: conv2 (tap, ci),
// conv3 (tap, ci), fc1 (pooled position, channel), fc2 (input).
constexpr int64_t WI2 = 0, WI3 = WI2 + (int64_t)9 * C2 * KB, WIF1 = WI3 + (int64_t)18 * C3 * KB,
                  WIF2 = WIF1 + (int64_t)(F0 / KE) * F1 * KB,
                  WTOT = WIF2 + (int64_t)(F1 / KE) * F2 * KB;   // bytes

__global__ void weight_image_kernel(const float *__restrict__ P, unsigned char *__restrict__ wimg)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // one BF16 element
    if (i >= WTOT / 2) return;
    int64_t off = i * 2, base;
    int N;
    if (off < WI3) { base = WI2; N = C2; }
    else if (off < WIF1) { base = WI3; N = C3; }
    else if (off < WIF2) { base = WIF1; N = F1; }
    else { base = WIF2; N = F2; }
    const int64_t rel = off - base;
    const int c = (int)(rel / ((int64_t)N * KB));
    const int within = (int)(rel % ((int64_t)N * KB));
    // invert core_off: within = (n >> 3) * SBO + j * LBO + (n & 7) * 16 + 2 * e8
    const int n = (within / SBO) * 8 + (within % LBO) / 16;
    const int e = ((within % SBO) / LBO) * 8 + (within % 16) / 2;
    float v;
    if (base == WI2) {
        v = P[OW2 + ((int64_t)n * C1 + e) * 9 + c];                    // tap c, ci e
    } else if (base == WI3) {
        v = P[OW3 + ((int64_t)n * C2 + (c & 1) * KE + e) * 9 + (c >> 1)];
    } else if (base == WIF1) {
        const int k = c * KE + e, pp = k / C3, ch = k % C3;            // feat order (pp, ch)
        v = P[OWF1 + (int64_t)n * F0 + ch * (HP * HP) + pp];
    } else {
        v = P[OWF2 + (int64_t)n * F1 + c * KE + e];
    }
    reinterpret_cast<__nv_bfloat16 *>(wimg)[i] = __float2bfloat16_rn(v);
}

template <int MODE>
int launch_gemm(const GemmArgs &a, cudaStream_t s)
{
    DT_CUDA_TRY(allow_smem((const void *)enc_gemm_kernel<MODE>, (int)gemm_smem<MODE>()));
    const int64_t tiles = (a.rows + TM - 1) / TM;
    const int grid = (int)std::min<int64_t>(tiles, sm_count());
    enc_gemm_kernel<MODE><<<grid, THREADS, gemm_smem<MODE>(), s>>>(a);
    DT_CUDA_TRY(cudaGetLastError());
    return DT_OK;
}

constexpr int64_t BATCH = 8192;            // images per pass (a1: 512 MB)

}  // namespace

int take_enc_tc_error(bool *raised)
{
    uint32_t v = 0, zero = 0;
    DT_CUDA_TRY(cudaMemcpyFromSymbol(&v, g_enc_tc_error, sizeof(v)));
    if (v) DT_CUDA_TRY(cudaMemcpyToSymbol(g_enc_tc_error, &zero, sizeof(zero)));
    *raised = v != 0;
    return DT_OK;
}

int launch_embed_tc(const float *P, const uint64_t *bits, int64_t n, __nv_bfloat16 *out_bf16,
                    float *out_f32, cudaStream_t s)
{
    if (n <= 0) return DT_OK;
    const int64_t nb = std::min<int64_t>(n, BATCH);
    Scratch scratch(s);
    unsigned char *wimg = nullptr;
    __nv_bfloat16 *a1 = nullptr, *a2 = nullptr, *feat = nullptr, *h = nullptr;
    DT_CUDA_TRY(scratch.alloc(&wimg, (size_t)WTOT));
    DT_CUDA_TRY(scratch.alloc(&a1, (size_t)nb * A1 * 2));
    DT_CUDA_TRY(scratch.alloc(&a2, (size_t)nb * A2 * 2));
    DT_CUDA_TRY(scratch.alloc(&feat, (size_t)nb * F0 * 2));
    DT_CUDA_TRY(scratch.alloc(&h, (size_t)nb * F1 * 2));
    weight_image_kernel<<<(unsigned)((WTOT / 2 + 255) / 256), 256, 0, s>>>(P, wimg);
    DT_CUDA_TRY(cudaGetLastError());
    int rc = DT_OK;
    for (int64_t i0 = 0; i0 < n && rc == DT_OK; i0 += nb) {
        const int64_t m = std::min<int64_t>(nb, n - i0);
        conv1_nhwc_kernel<<<(unsigned)std::min<int64_t>(m, (int64_t)sm_count() * 8), 256, 0, s>>>(
            bits + i0 * kWords, m, P, a1);
        DT_CUDA_TRY(cudaGetLastError());
        GemmArgs g2{a1, m * H2 * H2, wimg + WI2, P + OB2, a2, nullptr};
        GemmArgs g3{a2, m * H3 * H3, wimg + WI3, P + OB3, feat, nullptr};
        GemmArgs g4{feat, m, wimg + WIF1, P + OBF1, h, nullptr};
        GemmArgs g5{h, m, wimg + WIF2, P + OBF2, out_bf16 ? out_bf16 + i0 * F2 : nullptr,
                    out_f32 ? out_f32 + i0 * F2 : nullptr};
        rc = launch_gemm<CONV2>(g2, s);
        if (rc == DT_OK) rc = launch_gemm<CONV3>(g3, s);
        if (rc == DT_OK) rc = launch_gemm<FC1>(g4, s);
        if (rc == DT_OK) rc = launch_gemm<FC2>(g5, s);
    }
    return rc;
}

}  // namespace dtk
