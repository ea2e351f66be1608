// encoder_layout.cuh — shapes of the learned proposal's encoder and the
// order of its flat FP32 parameter buffer (w1 b1 w2 b2 w3 b3 wf1 bf1 wf2
// bf2; conv weights [out][in][ky][kx], fc weights [out][in]), shared by the
// FP32 kernels (encoder.cu) and the tensor-core inference path (enc_tc.cu).
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace dtk {
namespace enc {

constexpr int C1 = 32, C2 = 64, C3 = 64, H1 = 32, H2 = 16, H3 = 8, HP = 4;
constexpr int F0 = C3 * HP * HP, F1 = 256, F2 = 128;
constexpr int64_t OW1 = 0, OB1 = OW1 + C1 * 9, OW2 = OB1 + C1, OB2 = OW2 + C2 * C1 * 9,
                  OW3 = OB2 + C2, OB3 = OW3 + C3 * C2 * 9, OWF1 = OB3 + C3, OBF1 = OWF1 + F1 * F0,
                  OWF2 = OBF1 + F1, OBF2 = OWF2 + F2 * F1, NPARAM = OBF2 + F2;
static_assert(NPARAM == 351040, "parameter count");
constexpr int A1 = C1 * H1 * H1, A2 = C2 * H2 * H2, A3 = C3 * H3 * H3;

}  // namespace enc

// Encoder inference on the tensor cores (enc_tc.cu): embeddings of n
// descriptors from the FP32 parameters P, BF16 operands with FP32
// accumulation; out_bf16 and/or out_f32 [n][128].  Stream-ordered.
int launch_embed_tc(const float *P, const uint64_t *bits, int64_t n, __nv_bfloat16 *out_bf16,
                    float *out_f32, cudaStream_t s);
int take_enc_tc_error(bool *raised);

}  // namespace dtk
