// Host entry points of the camera G-buffer pass (gbuffer.cu).
#pragma once

#include <math.h>

#include "vct_internal.cuh"

namespace vct {

constexpr float kFrameUnits = 131072.0f;  // 2^17 fixed-point units per frame size
constexpr float kFrameLimit = 262144.0f;  // |snapped coordinate| < 2^18
constexpr int kGbTile = 16;               // pixels per tile edge

// Fixed-point snap of one coordinate (float32 without contraction, round
// half to even); false if beyond the frame.  Host and device alike.
__host__ __device__ inline bool frame_snap(float v, float origin, float s, long long *out) {
#ifdef __CUDA_ARCH__
  const float b = __fmul_rn(__fsub_rn(v, origin), s);
  if (!(fabsf(b) < kFrameLimit)) return false;
  *out = __float2ll_rn(b);
#else
  volatile float rel = v - origin;  // two roundings, never one fused operation
  const float b = rel * s;
  if (!(fabsf(b) < kFrameLimit)) return false;
  *out = (long long)nearbyintf(b);
#endif
  return true;
}

size_t gbuffer_fixed_bytes(int width, int height, int n_triangles);
cudaError_t launch_gbuffer(const vct_mesh &m, const vct_camera &cam, float *position,
                           float *normal, float *albedo, uint8_t *mask, int32_t *triangle,
                           void *ws, size_t ws_bytes, int sms, cudaStream_t s);

}  // namespace vct
