// encoder.cu — the learned proposal's encoder, trained and run by
// hand-written kernels (the paper has no learned component).
//
// Network (one 64x64 bit image in, a unit-length 128-d embedding out):
//   conv1 1->32, 3x3, stride 2, pad 1, ReLU   64x64 -> 32x32
//   conv2 32->64, 3x3, stride 2, pad 1, ReLU  32x32 -> 16x16
//   conv3 64->64, 3x3, stride 2, pad 1, ReLU  16x16 -> 8x8
//   2x2 average pooling                        8x8 -> 4x4 (1024 features)
//   fc1 1024->256, ReLU;  fc2 256->128;  z / ||z||
// Pixel (r, c) is bit c of word r of the descriptor.  351,040 FP32
// parameters, one flat buffer in the order w1 b1 w2 b2 w3 b3 wf1 bf1 wf2 bf2
// (conv weights [out][in][ky][kx], fc weights [out][in]).
//
// Training step (enc_train_step): both towers of a batch of (query, target)
// pairs go through the forward kernels with activations kept; the InfoNCE
// loss with in-batch negatives, L = mean_i( log sum_j exp(s_ij) - s_ii ),
// s_ij = <e_q[i], e_t[j]> / tau, is differentiated by hand back through
// every layer; Adam updates the parameters.  Kernels are plain FP32 on CUDA
// cores, one thread per output element (weight gradients split over the
// batch, the splits' partial sums added in a fixed order, so a step is the
// same on every run).  Inference (enc_embed) runs on the tensor cores for
// large batches (enc_tc.cu, BF16 operands); the FP32 inference path here is
// one fused kernel over
// weights re-laid out output-channel-contiguous: each thread keeps all
// output channels of its position in registers (conv2: 64, conv3: 16), a
// CTA keeps an image's conv activations in shared memory and runs the two
// dense layers on 4 pooled feature vectors at once.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include <cuda_bf16.h>

#include "dt_internal.cuh"
#include "encoder_layout.cuh"

namespace dtk {
namespace {

using namespace enc;

__device__ __forceinline__ float bit_px(const uint64_t *img, int r, int c)
{
    if (r < 0 || r >= 64 || c < 0 || c >= 64) return 0.f;
    return (float)((img[r] >> c) & 1ull);
}

// ---------------------------------------------------------------- forward
__global__ void conv1_fwd(const uint64_t *__restrict__ bits, const float *__restrict__ P, int M,
                          float *__restrict__ a1)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)M * A1) return;
    const int x = (int)(i % H1), y = (int)((i / H1) % H1), co = (int)((i / (H1 * H1)) % C1);
    const int64_t m = i / A1;
    const uint64_t *img = bits + m * kWords;
    const float *w = P + OW1 + co * 9;
    float s = P[OB1 + co];
#pragma unroll
    for (int ky = 0; ky < 3; ++ky)
#pragma unroll
        for (int kx = 0; kx < 3; ++kx) s += w[ky * 3 + kx] * bit_px(img, 2 * y + ky - 1, 2 * x + kx - 1);
    a1[i] = fmaxf(s, 0.f);
}

__global__ void conv_fwd(const float *__restrict__ in, const float *__restrict__ w,
                         const float *__restrict__ b, int M, int Ci, int Hi, int Co, int Ho,
                         float *__restrict__ out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t per = (int64_t)Co * Ho * Ho;
    if (i >= (int64_t)M * per) return;
    const int x = (int)(i % Ho), y = (int)((i / Ho) % Ho), co = (int)((i / (Ho * Ho)) % Co);
    const int64_t m = i / per;
    const float *src = in + m * (int64_t)Ci * Hi * Hi;
    float s = b[co];
    for (int ci = 0; ci < Ci; ++ci) {
        const float *wc = w + ((int64_t)co * Ci + ci) * 9;
        const float *sc = src + (int64_t)ci * Hi * Hi;
#pragma unroll
        for (int ky = 0; ky < 3; ++ky) {
            const int iy = 2 * y + ky - 1;
            if (iy < 0 || iy >= Hi) continue;
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) {
                const int ix = 2 * x + kx - 1;
                if (ix < 0 || ix >= Hi) continue;
                s += wc[ky * 3 + kx] * sc[iy * Hi + ix];
            }
        }
    }
    out[i] = fmaxf(s, 0.f);
}

__global__ void pool_fwd(const float *__restrict__ a3, int M, float *__restrict__ p)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)M * F0) return;
    const int x = (int)(i % HP), y = (int)((i / HP) % HP), c = (int)((i / (HP * HP)) % C3);
    const int64_t m = i / F0;
    const float *s = a3 + m * A3 + (int64_t)c * H3 * H3;
    p[i] = 0.25f * (s[(2 * y) * H3 + 2 * x] + s[(2 * y) * H3 + 2 * x + 1] +
                    s[(2 * y + 1) * H3 + 2 * x] + s[(2 * y + 1) * H3 + 2 * x + 1]);
}

// out[m][n] = b[n] + sum_k W[n][k] in[m][k], optional ReLU.
__global__ void fc_fwd(const float *__restrict__ in, const float *__restrict__ W,
                       const float *__restrict__ b, int M, int K, int N, int relu,
                       float *__restrict__ out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)M * N) return;
    const int n = (int)(i % N);
    const int64_t m = i / N;
    const float *x = in + m * K, *w = W + (int64_t)n * K;
    float s = b[n];
    for (int k = 0; k < K; ++k) s += w[k] * x[k];
    out[i] = relu ? fmaxf(s, 0.f) : s;
}

// e = z / ||z|| (one warp per row of 128).
__global__ void l2norm_fwd(const float *__restrict__ z, int M, float *__restrict__ e)
{
    const int lane = threadIdx.x & 31;
    const int64_t m = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (m >= M) return;
    float v[4], ss = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        v[j] = z[m * F2 + lane + 32 * j];
        ss += v[j] * v[j];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    const float inv = 1.f / fmaxf(sqrtf(ss), 1e-12f);
#pragma unroll
    for (int j = 0; j < 4; ++j) e[m * F2 + lane + 32 * j] = v[j] * inv;
}

// ---------------------------------------------------------------- loss
// S[i][j] = <eq_i, et_j> / tau
__global__ void sim_kernel(const float *__restrict__ eq, const float *__restrict__ et, int B,
                           float inv_tau, float *__restrict__ S)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * B) return;
    const int r = i / B, c = i % B;
    float s = 0.f;
    for (int k = 0; k < F2; ++k) s += eq[(int64_t)r * F2 + k] * et[(int64_t)c * F2 + k];
    S[i] = s * inv_tau;
}

// Row-wise softmax: loss_i = lse_i - S_ii; G = (softmax - I) / B in place.
__global__ void infonce_rows(float *__restrict__ S, int B, float *__restrict__ loss_rows)
{
    const int r = blockIdx.x;
    __shared__ float red[32];
    float mx = -INFINITY;
    for (int c = threadIdx.x; c < B; c += blockDim.x) mx = fmaxf(mx, S[(int64_t)r * B + c]);
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < (blockDim.x + 31) / 32 ? red[threadIdx.x] : -INFINITY;
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (threadIdx.x == 0) red[0] = v;
    }
    __syncthreads();
    mx = red[0];
    __syncthreads();
    float se = 0.f;
    for (int c = threadIdx.x; c < B; c += blockDim.x) se += expf(S[(int64_t)r * B + c] - mx);
    for (int o = 16; o > 0; o >>= 1) se += __shfl_xor_sync(0xffffffffu, se, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = se;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) t += red[w];
        red[0] = t;
    }
    __syncthreads();
    const float sum = red[0], lse = mx + logf(sum);
    if (threadIdx.x == 0) loss_rows[r] = lse - S[(int64_t)r * B + r];
    __syncthreads();
    for (int c = threadIdx.x; c < B; c += blockDim.x) {
        const float pr = expf(S[(int64_t)r * B + c] - mx) / sum;
        S[(int64_t)r * B + c] = (pr - (c == r ? 1.f : 0.f)) / (float)B;
    }
}

// de_q = G et / tau ; de_t = G^T eq / tau   (de laid out [2B][128], queries first)
__global__ void infonce_grad(const float *__restrict__ G, const float *__restrict__ eq,
                             const float *__restrict__ et, int B, float inv_tau,
                             float *__restrict__ de)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * B * F2) return;
    const int k = i % F2, row = i / F2;
    float s = 0.f;
    if (row < B) {
        for (int j = 0; j < B; ++j) s += G[(int64_t)row * B + j] * et[(int64_t)j * F2 + k];
    } else {
        const int c = row - B;
        for (int j = 0; j < B; ++j) s += G[(int64_t)j * B + c] * eq[(int64_t)j * F2 + k];
    }
    de[i] = s * inv_tau;
}

// ---------------------------------------------------------------- backward
// dz = (de - e <e, de>) / ||z||
__global__ void l2norm_bwd(const float *__restrict__ z, const float *__restrict__ e,
                           const float *__restrict__ de, int M, float *__restrict__ dz)
{
    const int lane = threadIdx.x & 31;
    const int64_t m = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (m >= M) return;
    float ss = 0.f, ed = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int64_t o = m * F2 + lane + 32 * j;
        ss += z[o] * z[o];
        ed += e[o] * de[o];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ss += __shfl_xor_sync(0xffffffffu, ss, o);
        ed += __shfl_xor_sync(0xffffffffu, ed, o);
    }
    const float inv = 1.f / fmaxf(sqrtf(ss), 1e-12f);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int64_t o = m * F2 + lane + 32 * j;
        dz[o] = (de[o] - e[o] * ed) * inv;
    }
}

// din[m][k] = sum_n W[n][k] dout[m][n], times (act[m][k] > 0) when act given.
__global__ void fc_bwd_data(const float *__restrict__ dout, const float *__restrict__ W, int M,
                            int K, int N, const float *__restrict__ act, float *__restrict__ din)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)M * K) return;
    const int k = (int)(i % K);
    const int64_t m = i / K;
    float s = 0.f;
    for (int n = 0; n < N; ++n) s += W[(int64_t)n * K + k] * dout[m * N + n];
    if (act && act[i] <= 0.f) s = 0.f;
    din[i] = s;
}

// The weight gradients sum over the batch, which is split over blockIdx.y
// for parallelism.  Each split writes its partial sums to part[split][i]
// and sum_partials adds them in split order, so that a training step gives
// the same gradient on every run (atomic float additions would not).

// part[y][n * (K + 1) + k] = sum over split y's rows m of dout[m][n] in[m][k]
// (k < K), or of dout[m][n] (k = K, the bias)
__global__ void fc_bwd_weight(const float *__restrict__ dout, const float *__restrict__ in, int M,
                              int K, int N, int m_chunk, float *__restrict__ part)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t count = (int64_t)N * (K + 1);
    if (i >= count) return;
    const int n = (int)(i / (K + 1)), k = (int)(i % (K + 1));
    const int m0 = blockIdx.y * m_chunk, m1 = min(M, m0 + m_chunk);
    float s = 0.f;
    for (int m = m0; m < m1; ++m) s += dout[(int64_t)m * N + n] * (k < K ? in[(int64_t)m * K + k] : 1.f);
    part[blockIdx.y * count + i] = s;
}

// g = sum over the ny splits of part[y][i], in split order, written to the
// weight gradient (i < n_w: dw[i]) or the bias gradient (db[i - n_w]); for
// a dense layer (fc_k > 0) i = n * (fc_k + 1) + k, the bias at k = fc_k.
__global__ void sum_partials(const float *__restrict__ part, int ny, int64_t count, int fc_k,
                             int64_t n_w, float *__restrict__ dw, float *__restrict__ db)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    float s = 0.f;
    for (int y = 0; y < ny; ++y) s += part[(int64_t)y * count + i];
    if (fc_k > 0) {
        const int64_t n = i / (fc_k + 1), k = i % (fc_k + 1);
        if (k < fc_k) dw[n * fc_k + k] = s;
        else db[n] = s;
    } else if (i < n_w) {
        dw[i] = s;
    } else {
        db[i - n_w] = s;
    }
}

// da3 = pool^T(dp) * (a3 > 0)
__global__ void pool_bwd(const float *__restrict__ dp, const float *__restrict__ a3, int M,
                         float *__restrict__ da3)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)M * A3) return;
    const int x = (int)(i % H3), y = (int)((i / H3) % H3), c = (int)((i / (H3 * H3)) % C3);
    const int64_t m = i / A3;
    const float g = 0.25f * dp[m * F0 + (int64_t)c * HP * HP + (y / 2) * HP + x / 2];
    da3[i] = a3[i] > 0.f ? g : 0.f;
}

// din[m][ci][iy][ix] = sum over (co, ky, kx) with iy = 2y+ky-1, ix = 2x+kx-1 of
// w[co][ci][ky][kx] dout[m][co][y][x], times (in > 0) (the ReLU of the layer below).
__global__ void conv_bwd_data(const float *__restrict__ dout, const float *__restrict__ w, int M,
                              int Ci, int Hi, int Co, int Ho, const float *__restrict__ act,
                              float *__restrict__ din)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t per = (int64_t)Ci * Hi * Hi;
    if (i >= (int64_t)M * per) return;
    if (act[i] <= 0.f) {
        din[i] = 0.f;
        return;
    }
    const int ix = (int)(i % Hi), iy = (int)((i / Hi) % Hi), ci = (int)((i / (Hi * Hi)) % Ci);
    const int64_t m = i / per;
    const float *g = dout + m * (int64_t)Co * Ho * Ho;
    float s = 0.f;
    for (int ky = 0; ky < 3; ++ky) {
        const int ty = iy + 1 - ky;
        if (ty < 0 || (ty & 1) || (ty >> 1) >= Ho) continue;
        for (int kx = 0; kx < 3; ++kx) {
            const int tx = ix + 1 - kx;
            if (tx < 0 || (tx & 1) || (tx >> 1) >= Ho) continue;
            const int y = ty >> 1, x = tx >> 1;
            for (int co = 0; co < Co; ++co)
                s += w[((int64_t)co * Ci + ci) * 9 + ky * 3 + kx] * g[((int64_t)co * Ho + y) * Ho + x];
        }
    }
    din[i] = s;
}

// part[y][i], for split y's rows m: i < Co Ci 9 the weight (co, ci, ky, kx),
// sum over (m, y, x) of dout[m][co][y][x] in[m][ci][2y+ky-1][2x+kx-1]; above,
// the bias co = i - Co Ci 9, sum of dout[m][co].  `in` is FP32 activations,
// or bits when `bits` is non-null (first layer).
__global__ void conv_bwd_weight(const float *__restrict__ dout, const float *__restrict__ in,
                                const uint64_t *__restrict__ bits, int M, int Ci, int Hi, int Co,
                                int Ho, int m_chunk, float *__restrict__ part)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nw = (int64_t)Co * Ci * 9;
    if (i >= nw + Co) return;
    const int m0 = blockIdx.y * m_chunk, m1 = min(M, m0 + m_chunk);
    float s = 0.f;
    if (i < nw) {
        const int kk = (int)(i % 9), ci = (int)((i / 9) % Ci), co = (int)(i / (9 * Ci));
        const int ky = kk / 3, kx = kk % 3;
        for (int m = m0; m < m1; ++m) {
            const float *g = dout + ((int64_t)m * Co + co) * Ho * Ho;
            for (int y = 0; y < Ho; ++y) {
                const int iy = 2 * y + ky - 1;
                if (iy < 0 || iy >= Hi) continue;
                for (int x = 0; x < Ho; ++x) {
                    const int ix = 2 * x + kx - 1;
                    if (ix < 0 || ix >= Hi) continue;
                    const float v = bits ? (float)((bits[(int64_t)m * kWords + iy] >> ix) & 1ull)
                                         : in[(((int64_t)m * Ci + ci) * Hi + iy) * Hi + ix];
                    s += g[y * Ho + x] * v;
                }
            }
        }
    } else {
        const int co = (int)(i - nw);
        for (int m = m0; m < m1; ++m) {
            const float *g = dout + ((int64_t)m * Co + co) * Ho * Ho;
            for (int j = 0; j < Ho * Ho; ++j) s += g[j];
        }
    }
    part[blockIdx.y * (nw + Co) + i] = s;
}

__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m1,
                            float *__restrict__ m2, int64_t n, float lr, float b1, float b2,
                            float eps, float c1, float c2)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi;
    const float b = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    p[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
}

// ---------------------------------------------------------------- fused inference
// Weights re-laid out for inference: conv weights [ci][tap][co] and dense
// weights [in][out], so that a thread's loop over output channels reads
// contiguous, warp-uniform (conv) or coalesced (dense) addresses.
constexpr int64_t TW1 = 0, TW2 = TW1 + 9 * C1, TW3 = TW2 + (int64_t)C1 * 9 * C2,
                  TWF1 = TW3 + (int64_t)C2 * 9 * C3, TWF2 = TWF1 + (int64_t)F0 * F1,
                  TTOT = TWF2 + (int64_t)F1 * F2;

__global__ void relayout_kernel(const float *__restrict__ P, float *__restrict__ T)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= TTOT) return;
    float v;
    if (i < TW2) {                                   // [tap][co] <- [co][0][tap]
        const int64_t tap = i / C1, co = i % C1;
        v = P[OW1 + co * 9 + tap];
    } else if (i < TW3) {                            // [ci][tap][co] <- [co][ci][tap]
        const int64_t r = i - TW2, co = r % C2, tap = (r / C2) % 9, ci = r / (C2 * 9);
        v = P[OW2 + (co * C1 + ci) * 9 + tap];
    } else if (i < TWF1) {
        const int64_t r = i - TW3, co = r % C3, tap = (r / C3) % 9, ci = r / (C3 * 9);
        v = P[OW3 + (co * C2 + ci) * 9 + tap];
    } else if (i < TWF2) {                           // [k][o] <- [o][k]
        const int64_t r = i - TWF1, o = r % F1, k = r / F1;
        v = P[OWF1 + o * F0 + k];
    } else {
        const int64_t r = i - TWF2, o = r % F2, k = r / F2;
        v = P[OWF2 + o * F1 + k];
    }
    T[i] = v;
}

constexpr int EG = 4;           // images per CTA pass (dense layers share weight reads)
constexpr int ET = 256;         // threads

__global__ void __launch_bounds__(ET, 1)
embed_kernel(const uint64_t *__restrict__ bits, int64_t n, const float *__restrict__ P,
             const float *__restrict__ T, __nv_bfloat16 *__restrict__ out_bf16,
             float *__restrict__ out_f32)
{
    extern __shared__ float sm[];
    float *a1 = sm;                       // [C1][H1][H1]
    float *a2 = a1 + A1;                  // [C2][H2][H2]
    float *a3 = a1;                       // [C3][H3][H3], a1 is dead once conv2 is done
    float *feat = a2 + A2;                // [EG][F0]
    float *hid = feat + EG * F0;          // [EG][F1]
    float *zz = hid + EG * F1;            // [EG][F2]
    __shared__ uint64_t img[kWords];
    const int tid = threadIdx.x;
    for (int64_t g0 = (int64_t)blockIdx.x * EG; g0 < n; g0 += (int64_t)gridDim.x * EG) {
        const int gcount = (int)(n - g0 < EG ? n - g0 : EG);
        for (int gi = 0; gi < gcount; ++gi) {
            const int64_t m = g0 + gi;
            if (tid < kWords) img[tid] = bits[m * kWords + tid];
            __syncthreads();
            // conv1: four positions per thread, all 32 channels in registers
            for (int p = tid; p < H1 * H1; p += ET) {
                const int y = p / H1, x = p % H1;
                float acc[C1];
#pragma unroll
                for (int co = 0; co < C1; ++co) acc[co] = P[OB1 + co];
#pragma unroll
                for (int tap = 0; tap < 9; ++tap) {
                    if (bit_px(img, 2 * y + tap / 3 - 1, 2 * x + tap % 3 - 1) != 0.f) {
                        const float4 *w = reinterpret_cast<const float4 *>(T + TW1 + tap * C1);
#pragma unroll
                        for (int c4 = 0; c4 < C1 / 4; ++c4) {
                            const float4 wv = __ldg(w + c4);
                            acc[4 * c4] += wv.x; acc[4 * c4 + 1] += wv.y;
                            acc[4 * c4 + 2] += wv.z; acc[4 * c4 + 3] += wv.w;
                        }
                    }
                }
#pragma unroll
                for (int co = 0; co < C1; ++co) a1[co * H1 * H1 + p] = fmaxf(acc[co], 0.f);
            }
            __syncthreads();
            // conv2: one position per thread, all 64 channels in registers
            {
                const int p = tid, y = p / H2, x = p % H2;
                float acc[C2];
#pragma unroll
                for (int co = 0; co < C2; ++co) acc[co] = P[OB2 + co];
                for (int ci = 0; ci < C1; ++ci) {
#pragma unroll
                    for (int tap = 0; tap < 9; ++tap) {
                        const int iy = 2 * y + tap / 3 - 1, ix = 2 * x + tap % 3 - 1;
                        const float v = (iy >= 0 && ix >= 0) ? a1[(ci * H1 + iy) * H1 + ix] : 0.f;
                        const float4 *w = reinterpret_cast<const float4 *>(T + TW2 + (ci * 9 + tap) * C2);
#pragma unroll
                        for (int c4 = 0; c4 < C2 / 4; ++c4) {
                            const float4 wv = __ldg(w + c4);
                            acc[4 * c4] += v * wv.x; acc[4 * c4 + 1] += v * wv.y;
                            acc[4 * c4 + 2] += v * wv.z; acc[4 * c4 + 3] += v * wv.w;
                        }
                    }
                }
#pragma unroll
                for (int co = 0; co < C2; ++co) a2[co * H2 * H2 + p] = fmaxf(acc[co], 0.f);
            }
            __syncthreads();
            // conv3: 64 positions x 4 blocks of 16 channels
            {
                const int p = tid & 63, cb = tid >> 6, y = p / H3, x = p % H3;
                float acc[16];
#pragma unroll
                for (int c = 0; c < 16; ++c) acc[c] = P[OB3 + cb * 16 + c];
                for (int ci = 0; ci < C2; ++ci) {
#pragma unroll
                    for (int tap = 0; tap < 9; ++tap) {
                        const int iy = 2 * y + tap / 3 - 1, ix = 2 * x + tap % 3 - 1;
                        const float v = (iy >= 0 && ix >= 0) ? a2[(ci * H2 + iy) * H2 + ix] : 0.f;
                        const float4 *w =
                            reinterpret_cast<const float4 *>(T + TW3 + (ci * 9 + tap) * C3 + cb * 16);
#pragma unroll
                        for (int c4 = 0; c4 < 4; ++c4) {
                            const float4 wv = __ldg(w + c4);
                            acc[4 * c4] += v * wv.x; acc[4 * c4 + 1] += v * wv.y;
                            acc[4 * c4 + 2] += v * wv.z; acc[4 * c4 + 3] += v * wv.w;
                        }
                    }
                }
                // a3 overwrites a1, whose last reads (conv2) ended at the barrier above
#pragma unroll
                for (int c = 0; c < 16; ++c) a3[(cb * 16 + c) * H3 * H3 + p] = fmaxf(acc[c], 0.f);
            }
            __syncthreads();
            for (int i = tid; i < F0; i += ET) {
                const int x = i % HP, y = (i / HP) % HP, c = i / (HP * HP);
                const float *s = a3 + c * H3 * H3;
                feat[gi * F0 + i] = 0.25f * (s[(2 * y) * H3 + 2 * x] + s[(2 * y) * H3 + 2 * x + 1] +
                                             s[(2 * y + 1) * H3 + 2 * x] + s[(2 * y + 1) * H3 + 2 * x + 1]);
            }
            __syncthreads();
        }
        // fc1: thread = output unit, EG images at once, coalesced weight rows
        for (int o = tid; o < F1; o += ET) {
            float acc[EG];
#pragma unroll
            for (int gi = 0; gi < EG; ++gi) acc[gi] = P[OBF1 + o];
            for (int k = 0; k < F0; ++k) {
                const float wk = __ldg(T + TWF1 + (int64_t)k * F1 + o);
#pragma unroll
                for (int gi = 0; gi < EG; ++gi) acc[gi] += wk * feat[gi * F0 + k];
            }
#pragma unroll
            for (int gi = 0; gi < EG; ++gi) hid[gi * F1 + o] = fmaxf(acc[gi], 0.f);
        }
        __syncthreads();
        for (int o = tid; o < F2; o += ET) {
            float acc[EG];
#pragma unroll
            for (int gi = 0; gi < EG; ++gi) acc[gi] = P[OBF2 + o];
            for (int k = 0; k < F1; ++k) {
                const float wk = __ldg(T + TWF2 + (int64_t)k * F2 + o);
#pragma unroll
                for (int gi = 0; gi < EG; ++gi) acc[gi] += wk * hid[gi * F1 + k];
            }
#pragma unroll
            for (int gi = 0; gi < EG; ++gi) zz[gi * F2 + o] = acc[gi];
        }
        __syncthreads();
        // normalise: warp per image
        const int lane = tid & 31, wid = tid >> 5;
        for (int gi = wid; gi < gcount; gi += ET / 32) {
            float v[4], ss = 0.f;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                v[j] = zz[gi * F2 + lane + 32 * j];
                ss += v[j] * v[j];
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
            const float inv = 1.f / fmaxf(sqrtf(ss), 1e-12f);
            const int64_t m = g0 + gi;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float e = v[j] * inv;
                if (out_bf16) out_bf16[m * F2 + lane + 32 * j] = __float2bfloat16_rn(e);
                if (out_f32) out_f32[m * F2 + lane + 32 * j] = e;
            }
        }
        __syncthreads();
    }
}

constexpr size_t EMBED_SMEM = (size_t)(A1 + A2 + EG * F0 + EG * F1 + EG * F2) * 4;

unsigned blocks_for(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace
}  // namespace dtk

// ---------------------------------------------------------------- the encoder object
struct dt_encoder {
    int device = 0;
    float *P = nullptr, *G = nullptr, *m1 = nullptr, *m2 = nullptr;   // [NPARAM]
    int64_t step = 0;
    int cap = 0;                  // batch pairs the workspace holds
    float *ws = nullptr;          // activations and gradients for 2*cap images
};

using namespace dtk;

namespace {

struct Ws {
    float *a1, *a2, *a3, *p, *h, *z, *e, *da2, *da3, *dp, *dh, *dz, *de, *S, *loss;
};

size_t ws_floats(int cap)
{
    const size_t M = 2 * (size_t)cap;
    return M * (A1 + A2 + A3 + F0 + F1 + F2 + F2) + M * (A2 + A3 + F0 + F1 + F2 + F2) +
           (size_t)cap * cap + (size_t)cap;
}

Ws carve(float *w, int cap)
{
    const size_t M = 2 * (size_t)cap;
    Ws s;
    s.a1 = w; w += M * A1;
    s.a2 = w; w += M * A2;
    s.a3 = w; w += M * A3;
    s.p = w; w += M * F0;
    s.h = w; w += M * F1;
    s.z = w; w += M * F2;
    s.e = w; w += M * F2;
    s.da2 = w; w += M * A2;
    s.da3 = w; w += M * A3;
    s.dp = w; w += M * F0;
    s.dh = w; w += M * F1;
    s.dz = w; w += M * F2;
    s.de = w; w += M * F2;
    s.S = w; w += (size_t)cap * cap;
    s.loss = w;
    return s;
}

// He-uniform initial weights from SplitMix64 (host), biases zero.
void init_params(std::vector<float> &p, uint64_t seed)
{
    auto fill = [&](int64_t off, int64_t count, int fan_in) {
        const double lim = std::sqrt(6.0 / fan_in);
        uint64_t s = seed + 0x9e3779b97f4a7c15ull * (uint64_t)(off + 1);
        for (int64_t i = 0; i < count; ++i) {
            uint64_t z = (s += 0x9e3779b97f4a7c15ull);
            z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
            z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
            z ^= z >> 31;
            const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
            p[(size_t)(off + i)] = (float)((2.0 * u - 1.0) * lim);
        }
    };
    std::fill(p.begin(), p.end(), 0.f);
    fill(OW1, C1 * 9, 9);
    fill(OW2, C2 * C1 * 9, C1 * 9);
    fill(OW3, C3 * C2 * 9, C2 * 9);
    fill(OWF1, (int64_t)F1 * F0, F0);
    fill(OWF2, (int64_t)F2 * F1, F1);
}

int ensure_ws(dt_encoder *e, int B)
{
    if (B <= e->cap) return DT_OK;
    if (e->ws) cudaFree(e->ws);
    e->ws = nullptr;
    e->cap = 0;
    DT_CUDA_TRY(cudaMalloc((void **)&e->ws, ws_floats(B) * sizeof(float)));
    e->cap = B;
    return DT_OK;
}

// Forward of M images with activations kept in the workspace (rows offset `row0`).
void forward_train(const dt_encoder *enc, const uint64_t *bits, int M, const Ws &w, int row0,
                   cudaStream_t s)
{
    float *a1 = w.a1 + (size_t)row0 * A1, *a2 = w.a2 + (size_t)row0 * A2, *a3 = w.a3 + (size_t)row0 * A3;
    float *p = w.p + (size_t)row0 * F0, *h = w.h + (size_t)row0 * F1, *z = w.z + (size_t)row0 * F2,
          *e = w.e + (size_t)row0 * F2;
    const float *P = enc->P;
    conv1_fwd<<<blocks_for((int64_t)M * A1), 256, 0, s>>>(bits, P, M, a1);
    conv_fwd<<<blocks_for((int64_t)M * A2), 256, 0, s>>>(a1, P + OW2, P + OB2, M, C1, H1, C2, H2, a2);
    conv_fwd<<<blocks_for((int64_t)M * A3), 256, 0, s>>>(a2, P + OW3, P + OB3, M, C2, H2, C3, H3, a3);
    pool_fwd<<<blocks_for((int64_t)M * F0), 256, 0, s>>>(a3, M, p);
    fc_fwd<<<blocks_for((int64_t)M * F1), 256, 0, s>>>(p, P + OWF1, P + OBF1, M, F0, F1, 1, h);
    fc_fwd<<<blocks_for((int64_t)M * F2), 256, 0, s>>>(h, P + OWF2, P + OBF2, M, F1, F2, 0, z);
    l2norm_fwd<<<blocks_for((int64_t)M * 32), 256, 0, s>>>(z, M, e);
}

}  // namespace

extern "C" {

int enc_create(uint64_t seed, dt_encoder **out)
{
    DT_CHECK_ARG(out != nullptr, "out must not be NULL");
    *out = nullptr;
    dt_encoder *e = new dt_encoder();
    DT_CUDA_TRY(cudaGetDevice(&e->device));
    std::vector<float> h((size_t)NPARAM);
    init_params(h, seed);
    const size_t bytes = (size_t)NPARAM * 4;
    if (cudaMalloc((void **)&e->P, bytes) != cudaSuccess || cudaMalloc((void **)&e->G, bytes) != cudaSuccess ||
        cudaMalloc((void **)&e->m1, bytes) != cudaSuccess || cudaMalloc((void **)&e->m2, bytes) != cudaSuccess) {
        set_error("enc_create: allocation failed");
        cudaFree(e->P); cudaFree(e->G); cudaFree(e->m1); cudaFree(e->m2);
        delete e;
        return DT_ENOMEM;
    }
    cudaMemcpy(e->P, h.data(), bytes, cudaMemcpyHostToDevice);
    cudaMemset(e->G, 0, bytes);
    cudaMemset(e->m1, 0, bytes);
    cudaMemset(e->m2, 0, bytes);
    *out = e;
    return DT_OK;
}

void enc_free(dt_encoder *e)
{
    if (!e) return;
    cudaDeviceSynchronize();
    cudaFree(e->P); cudaFree(e->G); cudaFree(e->m1); cudaFree(e->m2); cudaFree(e->ws);
    delete e;
}

int64_t enc_param_count(void) { return NPARAM; }

int enc_get_params(const dt_encoder *e, float *h_params)
{
    DT_CHECK_ARG(e && h_params, "encoder and buffer required");
    DT_CUDA_TRY(cudaMemcpy(h_params, e->P, (size_t)NPARAM * 4, cudaMemcpyDeviceToHost));
    return DT_OK;
}

int enc_set_params(dt_encoder *e, const float *h_params)
{
    DT_CHECK_ARG(e && h_params, "encoder and buffer required");
    DT_CUDA_TRY(cudaMemcpy(e->P, h_params, (size_t)NPARAM * 4, cudaMemcpyHostToDevice));
    return DT_OK;
}

int enc_get_grads(const dt_encoder *e, float *h_grads)
{
    DT_CHECK_ARG(e && h_grads, "encoder and buffer required");
    DT_CUDA_TRY(cudaMemcpy(h_grads, e->G, (size_t)NPARAM * 4, cudaMemcpyDeviceToHost));
    return DT_OK;
}

int enc_embed(const dt_encoder *e, const uint64_t *d_bits, int64_t n, uint16_t *d_out_bf16,
              float *d_out_f32, int32_t path, void *stream)
{
    DT_CHECK_ARG(e && d_bits && n >= 0 && (d_out_bf16 || d_out_f32), "bad arguments");
    DT_CHECK_ARG(path >= 0 && path <= 2, "path must be 0, 1 or 2");
    if (n == 0) return DT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (path == 2 || (path == 0 && n >= 4096))
        return launch_embed_tc(e->P, d_bits, n, reinterpret_cast<__nv_bfloat16 *>(d_out_bf16),
                               d_out_f32, s);
    DT_CUDA_TRY(allow_smem((const void *)embed_kernel, (int)EMBED_SMEM));
    Scratch scratch(s);
    float *T = nullptr;
    DT_CUDA_TRY(scratch.alloc(&T, (size_t)TTOT * 4));
    relayout_kernel<<<blocks_for(TTOT), 256, 0, s>>>(e->P, T);
    const int64_t groups = (n + EG - 1) / EG;
    const unsigned grid = (unsigned)std::min<int64_t>(groups, (int64_t)sm_count());   // one CTA per SM fits
    embed_kernel<<<grid, ET, EMBED_SMEM, s>>>(d_bits, n, e->P, T,
                                              reinterpret_cast<__nv_bfloat16 *>(d_out_bf16), d_out_f32);
    DT_CUDA_TRY(cudaGetLastError());
    return DT_OK;
}

// One InfoNCE step on B (query, target) pairs.  update = 0 leaves the
// parameters unchanged (the gradient stays readable with enc_get_grads).
// h_loss (nullable, host) receives the batch loss (synchronises).
int enc_train_step(dt_encoder *e, const uint64_t *d_q, const uint64_t *d_t, int32_t B, float lr,
                   float tau, int32_t update, float *h_loss, void *stream)
{
    DT_CHECK_ARG(e && d_q && d_t && B >= 2 && B <= 4096 && tau > 0.f, "bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    if (int r = ensure_ws(e, B)) return r;
    const Ws w = carve(e->ws, e->cap);
    const int M = 2 * B;
    float *P = e->P, *G = e->G;
    forward_train(e, d_q, B, w, 0, s);
    forward_train(e, d_t, B, w, B, s);
    const float inv_tau = 1.f / tau;
    const float *eq = w.e, *et = w.e + (size_t)B * F2;
    sim_kernel<<<blocks_for((int64_t)B * B), 256, 0, s>>>(eq, et, B, inv_tau, w.S);
    infonce_rows<<<B, 256, 0, s>>>(w.S, B, w.loss);
    infonce_grad<<<blocks_for((int64_t)2 * B * F2), 256, 0, s>>>(w.S, eq, et, B, inv_tau, w.de);
    DT_CUDA_TRY(cudaMemsetAsync(G, 0, (size_t)NPARAM * 4, s));
    l2norm_bwd<<<blocks_for((int64_t)M * 32), 256, 0, s>>>(w.z, w.e, w.de, M, w.dz);
    const int mc = 64, gy = (M + mc - 1) / mc;
    const int cc = 8, gyc = (M + cc - 1) / cc;
    // per-split partial sums of the weight gradients, reused layer by layer
    Scratch gscratch(s);
    float *part = nullptr;
    const int64_t part_n = std::max({(int64_t)gy * F2 * (F1 + 1), (int64_t)gy * F1 * (F0 + 1),
                                     (int64_t)gyc * (C3 * C2 * 9 + C3), (int64_t)gyc * (C2 * C1 * 9 + C2),
                                     (int64_t)gyc * (C1 * 9 + C1)});
    DT_CUDA_TRY(gscratch.alloc(&part, (size_t)part_n * 4));
    auto fc_grad = [&](const float *dout, const float *in, int K, int N, float *dw, float *db) {
        const int64_t count = (int64_t)N * (K + 1);
        fc_bwd_weight<<<dim3(blocks_for(count), gy), 256, 0, s>>>(dout, in, M, K, N, mc, part);
        sum_partials<<<blocks_for(count), 256, 0, s>>>(part, gy, count, K, 0, dw, db);
    };
    auto conv_grad = [&](const float *dout, const float *in, const uint64_t *bits, int Ci, int Hi, int Co,
                         int Ho, float *dw, float *db) {
        const int64_t nw = (int64_t)Co * Ci * 9, count = nw + Co;
        conv_bwd_weight<<<dim3(blocks_for(count), gyc), 256, 0, s>>>(dout, in, bits, M, Ci, Hi, Co, Ho,
                                                                     cc, part);
        sum_partials<<<blocks_for(count), 256, 0, s>>>(part, gyc, count, 0, nw, dw, db);
    };
    fc_grad(w.dz, w.h, F1, F2, G + OWF2, G + OBF2);
    fc_bwd_data<<<blocks_for((int64_t)M * F1), 256, 0, s>>>(w.dz, P + OWF2, M, F1, F2, w.h, w.dh);
    fc_grad(w.dh, w.p, F0, F1, G + OWF1, G + OBF1);
    fc_bwd_data<<<blocks_for((int64_t)M * F0), 256, 0, s>>>(w.dh, P + OWF1, M, F0, F1, nullptr, w.dp);
    pool_bwd<<<blocks_for((int64_t)M * A3), 256, 0, s>>>(w.dp, w.a3, M, w.da3);
    conv_grad(w.da3, w.a2, nullptr, C2, H2, C3, H3, G + OW3, G + OB3);
    conv_bwd_data<<<blocks_for((int64_t)M * A2), 256, 0, s>>>(w.da3, P + OW3, M, C2, H2, C3, H3, w.a2, w.da2);
    conv_grad(w.da2, w.a1, nullptr, C1, H1, C2, H2, G + OW2, G + OB2);
    // conv1's input gradient is not needed; its output gradient da1 is:
    {
        // da1 = conv2^T(da2) * (a1 > 0), kept in a scratch region sized M * A1
        Scratch scratch(s);
        float *buf = nullptr;
        DT_CUDA_TRY(scratch.alloc(&buf, (size_t)M * A1 * 4));
        conv_bwd_data<<<blocks_for((int64_t)M * A1), 256, 0, s>>>(w.da2, P + OW2, M, C1, H1, C2, H2, w.a1, buf);
        // bits of both towers, contiguous in the order of the activations
        uint64_t *bits = nullptr;
        DT_CUDA_TRY(scratch.alloc(&bits, (size_t)M * kWords * 8));
        DT_CUDA_TRY(cudaMemcpyAsync(bits, d_q, (size_t)B * kWords * 8, cudaMemcpyDeviceToDevice, s));
        DT_CUDA_TRY(cudaMemcpyAsync(bits + (size_t)B * kWords, d_t, (size_t)B * kWords * 8,
                                    cudaMemcpyDeviceToDevice, s));
        conv_grad(buf, nullptr, bits, 1, 64, C1, H1, G + OW1, G + OB1);
    }
    DT_CUDA_TRY(cudaGetLastError());
    if (update) {
        e->step += 1;
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.f - std::pow(b1, (float)e->step), c2 = 1.f - std::pow(b2, (float)e->step);
        adam_kernel<<<blocks_for(NPARAM), 256, 0, s>>>(P, G, e->m1, e->m2, NPARAM, lr, b1, b2, 1e-8f, c1, c2);
        DT_CUDA_TRY(cudaGetLastError());
    }
    if (h_loss) {
        std::vector<float> l((size_t)B);
        DT_CUDA_TRY(cudaMemcpyAsync(l.data(), w.loss, (size_t)B * 4, cudaMemcpyDeviceToHost, s));
        DT_CUDA_TRY(cudaStreamSynchronize(s));
        double t = 0;
        for (float v : l) t += v;
        *h_loss = (float)(t / B);
    }
    return DT_OK;
}

}  // extern "C"
