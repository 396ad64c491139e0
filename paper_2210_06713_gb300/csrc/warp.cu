// Tilt warp: the Noll 2/3 part of the phase (a linear phase in Eq. 2) only
// moves the PSF, by -(4/pi) a_2 columns and -(4/pi) a_3 rows on a Nyquist-
// sampled PSF grid (64-sample pupil grid, aperture 32 samples across).  So
// the image is resampled at (x + (4/pi) a_2, y + (4/pi) a_3), bilinearly,
// clamping at the borders.
//
// HBM-bound: per pixel it reads a_2, a_3 (8 B) and writes C floats, and the
// gathers of the C source values mostly hit L1/L2 (displacements are a few
// pixels).  One thread handles 4 consecutive pixels of a row (float4 I/O).
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"
#include "tilt.cuh"

namespace {

__global__ void __launch_bounds__(256) k_tilt_warp(const float* __restrict__ img, int C, int H, int W,
                                                   const float* __restrict__ a2, const float* __restrict__ a3,
                                                   float* __restrict__ out, int aligned) {
  const int x4 = (blockIdx.x * blockDim.x + threadIdx.x) * 4;
  const int y = blockIdx.y;
  if (x4 >= W) return;
  const size_t row = (size_t)y * W;
  float dx[4], dy[4];
  const bool vec = aligned && (x4 + 4 <= W);
  if (vec) {
    const float4 u = __ldg(reinterpret_cast<const float4*>(a2 + row + x4));
    const float4 v = __ldg(reinterpret_cast<const float4*>(a3 + row + x4));
    dx[0] = u.x; dx[1] = u.y; dx[2] = u.z; dx[3] = u.w;
    dy[0] = v.x; dy[1] = v.y; dy[2] = v.z; dy[3] = v.w;
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      dx[i] = x4 + i < W ? a2[row + x4 + i] : 0.f;
      dy[i] = x4 + i < W ? a3[row + x4 + i] : 0.f;
    }
  }
  const size_t plane = (size_t)H * W;
  for (int c = 0; c < C; ++c) {
    const float* I = img + c * plane;
    float r[4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
      r[i] = tilt_sample(I, H, W, x4 + i, y, dx[i], dy[i]);
    float* o = out + c * plane + row + x4;
    if (vec) {
      *reinterpret_cast<float4*>(o) = make_float4(r[0], r[1], r[2], r[3]);
    } else {
      for (int i = 0; i < 4 && x4 + i < W; ++i) o[i] = r[i];
    }
  }
}

}  // namespace

int dfp2s_launch_tilt_warp(const float* img, int C, int H, int W, const float* a2, const float* a3, float* out,
                           cudaStream_t st) {
  const int per_row = (W + 3) / 4;
  dim3 grid((per_row + 255) / 256, H);
  const int aligned = ((W & 3) == 0) && (((uintptr_t)a2 | (uintptr_t)a3 | (uintptr_t)out) & 15) == 0;
  k_tilt_warp<<<grid, 256, 0, st>>>(img, C, H, W, a2, a3, out, aligned);
  return dfp2s_launch_status();
}
