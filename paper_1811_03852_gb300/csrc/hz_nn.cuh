// hz_nn.cuh -- definitions shared by the conv-net kernels (hz_nn.cu) and their
// tcgen05 versions (hz_nn_tc.cu).
#pragma once

#include <cuda_bf16.h>

#include "hz_internal.cuh"

namespace hz {

constexpr int kC = 16;    // hidden channels
constexpr int kTaps = 27;

struct NnGrid {
  int nx, ny, nz, seg;   // seg: rows per stacked crop (= ny for one field)
  int periodic;          // 1: wrap in i
  int64_t n;
};

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// kernel-side weights (bf16-rounded values; FP32 copies for the CUDA-core layers)
struct NnW {
  const float* w1;                // [27][16]     layer 1, (tap, co)
  const float* b1;                // [16]
  const __nv_bfloat16* w2b;       // [27][16][16] layer 2, (tap, co, ci) for the MMA
  const float* w2f;               // [27][16][16] same values in FP32 (backward)
  const float* b2;
  const __nv_bfloat16* w3b;
  const float* w3f;
  const float* b3;
  const float* w4;                // [27][16]     layer 4, (tap, ci)
  const float* b4;                // [1]
};

// ---- tcgen05 plane kernels (hz_nn_tc.cu) ----
// Tiles of 128 consecutive points of a row (one M = 128 MMA per row and tap),
// two rows per CTA.  Usable when nx >= 128 and no tile straddles a crop seam.
bool nn_tc_ok(const NnGrid& g);
// 16 -> 16 conv + bias (z: pre-activation, optional) + GELU -> hout (BF16)
cudaError_t nn_tc_mid(const NnGrid& g, const __nv_bfloat16* hin, const __nv_bfloat16* wb, const float* bias, float* z,
                      __nv_bfloat16* hout, int* err, int sms, cudaStream_t s);
// 16 -> 1 conv + bias -> out, or out = base + sigma * y (sigma = sqrt(*nrm2 / n))
cudaError_t nn_tc_l4(const NnGrid& g, const __nv_bfloat16* hin, const float* w4, const float* b4, const float* base,
                     const double* nrm2, float* out, int* err, int sms, cudaStream_t s);

}  // namespace hz
