// The tilt warp's sampler (the Noll 2/3 part of Eq. 2's phase moves the PSF by
// -(4/pi) (a_2, a_3) pixels on the Nyquist-sampled grid): the image value at
// (x + (4/pi) a_2, y + (4/pi) a_3), bilinear, clamped at the borders.  Shared by
// the warp kernel and the fused warp + blur-operand kernel so that both give the
// same floats.
#pragma once

#include "common.cuh"

constexpr float kTiltPix = 1.27323954473516268615f;  // 4 / pi

DFP2S_DEV float bilinear_clamp(const float* __restrict__ I, int H, int W, float sx, float sy) {
  const float fx = floorf(sx), fy = floorf(sy);
  const float tx = sx - fx, ty = sy - fy;
  const int x0 = (int)fx, y0 = (int)fy;
  const int xa = min(max(x0, 0), W - 1), xb = min(max(x0 + 1, 0), W - 1);
  const int ya = min(max(y0, 0), H - 1), yb = min(max(y0 + 1, 0), H - 1);
  const float v00 = __ldg(I + (size_t)ya * W + xa), v01 = __ldg(I + (size_t)ya * W + xb);
  const float v10 = __ldg(I + (size_t)yb * W + xa), v11 = __ldg(I + (size_t)yb * W + xb);
  const float top = fmaf(tx, v01 - v00, v00);
  const float bot = fmaf(tx, v11 - v10, v10);
  return fmaf(ty, bot - top, top);
}

// warped value of pixel (x, y) given its tilts a_2 = dx, a_3 = dy
DFP2S_DEV float tilt_sample(const float* __restrict__ I, int H, int W, int x, int y, float dx, float dy) {
  return bilinear_clamp(I, H, W, fmaf(kTiltPix, dx, (float)x), fmaf(kTiltPix, dy, (float)y));
}
