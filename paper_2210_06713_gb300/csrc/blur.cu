// Basis blur, Eq. (varying blur): out_c(x) = sum_k w_k(x) (phi_k (*) I_c)(x),
// true convolution over u in [-16, 16]^2, clamp-to-edge borders.
//
// FP32 form (used with FP32 weights, i.e. the exact-P2S frame): per pixel the
// PSF h_x(u) = sum_k w_k(x) phi_k(u) is formed one row of taps at a time in
// registers, then contracted with the image halo in shared memory:
//   out_c(x) = sum_u h_x(u) I_c(x - u).
// That costs 2*1089*(K + C) FLOP per pixel instead of 2*1089*K*C for the
// per-basis convolutions, with identical value in exact arithmetic.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int KS = 33;
constexpr int R = 16;
constexpr int TH = 4;       // tile rows
constexpr int TW = 32;      // tile columns
constexpr int NTH = TH * TW;  // one thread per pixel
constexpr int HR = TH + 2 * R;  // 36 halo rows
constexpr int HC = TW + 2 * R;  // 64 halo columns
constexpr int CG = 4;       // channels per pass
constexpr int PR = 36;      // padded tap-row length

template <typename WT>
DFP2S_DEV float load_w(const WT* w, size_t i);
template <>
DFP2S_DEV float load_w<float>(const float* w, size_t i) { return __ldg(w + i); }
template <>
DFP2S_DEV float load_w<__nv_bfloat16>(const __nv_bfloat16* w, size_t i) { return __bfloat162float(w[i]); }

template <typename WT>
__global__ void __launch_bounds__(NTH) k_blur_psf(const float* __restrict__ img, int C, int H, int W,
                                                  const float* __restrict__ basis, int K, const WT* __restrict__ w,
                                                  float* __restrict__ out) {
  extern __shared__ float4 smem_f4[];
  float* halo = reinterpret_cast<float*>(smem_f4);      // CG x HR x HC
  float* wsm = halo + CG * HR * HC;                      // K x NTH
  float* phis = wsm + K * NTH;                           // K x PR
  const int t = threadIdx.x;
  const int ty = t / TW, tx = t - ty * TW;
  const int x0 = blockIdx.x * TW, y0 = blockIdx.y * TH;
  const int y = y0 + ty, x = x0 + tx;
  const bool live = (y < H) && (x < W);
  const int yc = min(y, H - 1), xc = min(x, W - 1);
  for (int k = 0; k < K; ++k) wsm[k * NTH + t] = load_w<WT>(w, ((size_t)yc * W + xc) * K + k);
  const size_t plane = (size_t)H * W;
  for (int c0 = 0; c0 < C; c0 += CG) {
    const int nc = min(CG, C - c0);
    __syncthreads();
    for (int i = t; i < nc * HR * HC; i += NTH) {
      const int c = i / (HR * HC);
      const int rr = (i / HC) % HR, cc = i % HC;
      const int sy = min(max(y0 - R + rr, 0), H - 1), sx = min(max(x0 - R + cc, 0), W - 1);
      halo[i] = __ldg(img + (c0 + c) * plane + (size_t)sy * W + sx);
    }
    float acc[CG] = {0.f, 0.f, 0.f, 0.f};
    for (int iy = 0; iy < KS; ++iy) {
      __syncthreads();
      for (int i = t; i < K * PR; i += NTH) {
        const int k = i / PR, ix = i - k * PR;
        phis[i] = ix < KS ? __ldg(basis + ((size_t)k * KS + iy) * KS + ix) : 0.f;
      }
      __syncthreads();
      float h[PR];
#pragma unroll
      for (int ix = 0; ix < PR; ++ix) h[ix] = 0.f;
      for (int k = 0; k < K; ++k) {
        const float wv = wsm[k * NTH + t];
        const float4* pr = reinterpret_cast<const float4*>(phis + k * PR);
#pragma unroll
        for (int q = 0; q < PR / 4; ++q) {
          const float4 f = pr[q];
          h[4 * q + 0] = fmaf(wv, f.x, h[4 * q + 0]);
          h[4 * q + 1] = fmaf(wv, f.y, h[4 * q + 1]);
          h[4 * q + 2] = fmaf(wv, f.z, h[4 * q + 2]);
          h[4 * q + 3] = fmaf(wv, f.w, h[4 * q + 3]);
        }
      }
      const int hr = ty + 2 * R - iy;
#pragma unroll
      for (int c = 0; c < CG; ++c) {
        if (c < nc) {
          const float* hrow = halo + (c * HR + hr) * HC + tx + 2 * R;
          float a = acc[c];
#pragma unroll
          for (int ix = 0; ix < KS; ++ix) a = fmaf(h[ix], hrow[-ix], a);
          acc[c] = a;
        }
      }
    }
    if (live)
      for (int c = 0; c < nc; ++c) out[(c0 + c) * plane + (size_t)y * W + x] = acc[c];
  }
}

}  // namespace

int dfp2s_launch_blur(const dfp2s_p2s_dev* p, const float* img, int C, int H, int W, const void* w, int w_dtype,
                      float* out, cudaStream_t st) {
  const int K = p->K;
  const size_t sm = (size_t)(CG * HR * HC + K * NTH + K * PR) * sizeof(float);
  dim3 grid((W + TW - 1) / TW, (H + TH - 1) / TH);
  if (w_dtype == DFP2S_W_BF16) {
    cudaFuncSetAttribute(k_blur_psf<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_blur_psf<__nv_bfloat16><<<grid, NTH, sm, st>>>(img, C, H, W, p->basis, K, (const __nv_bfloat16*)w, out);
  } else {
    cudaFuncSetAttribute(k_blur_psf<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_blur_psf<float><<<grid, NTH, sm, st>>>(img, C, H, W, p->basis, K, (const float*)w, out);
  }
  return dfp2s_launch_status();
}
