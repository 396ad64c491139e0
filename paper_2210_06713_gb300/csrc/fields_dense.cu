// The dense-root form of the field sampler (Sec. III-A's eigen-root form applied per frequency; reading R6):
// E(k) = F(k) xi(k) with F(k) the symmetric root of S~(k) = L diag(lambda(k)) L^T (factor.cu builds it in FP64,
// stores FP32), xi the Fourier-domain white noise of the factored sampler (the same Philox streams, R27), then the
// inverse 2-D FFT per mode.  The fields come out mixed: no mixing pass follows.
//   k_dense_mix   32 pairs of bins ky = 2i, 2i + 1 per CTA: the J modes' Gaussians (one Philox block each; the
//                 corners' real Gaussians scaled by sqrt 2) into shared memory, then E_j = sum_i F_ji xi_i (F read
//                 once per frame: J^2 floats per bin, coalesced across the bins);
//   k_colspec     one frequency column of one mode per thread group: E, the Hermitian completion of columns
//                 0 and N/2, the scale (N/sqrt2)(D/r0)^{5/6}/N^2, the inverse FFT over ky, rows y < H;
//   k_rowifft     (fields.cu) the row transforms and the crop.
#include <cuda_runtime.h>

#include "common.cuh"
#include "fft_reg.cuh"
#include "field_groups.cuh"
#include "kernels.h"

namespace {

using fftr::OutIndex;
using fftr::pad32;
using fftr::Plan;

// 32 bin pairs per CTA: the CTA draws the pairs' J-mode noise into shared memory once (one Philox block per pair
// and mode), then warp q forms E_j for j = q, q + 4, ... of all 32 pairs (lane = pair: the F loads of a warp are
// 256 contiguous bytes, the noise reads 512 contiguous bytes of shared memory).
constexpr int kPairs = 32;

__global__ void __launch_bounds__(128) k_dense_mix(const float* __restrict__ F, int J, int N, int log2N, uint64_t seed,
                                                   uint32_t frame, float2* __restrict__ E) {
  __shared__ float4 xs[48][kPairs];  // (Re, Im) of bins 2i, 2i + 1 per mode and pair
  const int HALF = N / 2 + 1;
  const long long npairs = (long long)HALF * (N / 2);
  const long long p0 = (long long)blockIdx.x * kPairs;
  const size_t nbins = (size_t)HALF * N;
  for (int e = threadIdx.x; e < kPairs * J; e += blockDim.x) {
    const int p = e % kPairs, j = e / kPairs;
    const long long idx = p0 + p;
    float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    if (idx < npairs) {
      const int kx = (int)(idx >> (log2N - 1)), i = (int)(idx & (N / 2 - 1));
      z = dfp2s_gauss4(seed, dfp2s_subsequence(0u, frame, (uint32_t)j), (uint64_t)kx * (N / 2) + i);
      const bool col = kx == 0 || kx == N / 2;
      if (col && (i == 0 || 2 * i == N / 2)) z = make_float4(z.x * 1.41421356237309505f, 0.f, z.z, z.w);  // corner
    }
    xs[j][p] = z;
  }
  __syncthreads();
  const int p = threadIdx.x & 31, q = threadIdx.x >> 5;
  const long long idx = p0 + p;
  if (idx >= npairs) return;
  const int kx = (int)(idx >> (log2N - 1)), i = (int)(idx & (N / 2 - 1));
  const size_t bin0 = (size_t)kx * N + 2 * i;
  for (int j = q; j < J; j += 4) {
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    const float* Fj = F + (size_t)j * J * nbins + bin0;
#pragma unroll 12
    for (int k = 0; k < J; ++k) {
      const float2 f = __ldg(reinterpret_cast<const float2*>(Fj + (size_t)k * nbins));
      const float4 x = xs[k][p];
      acc.x = fmaf(f.x, x.x, acc.x);
      acc.y = fmaf(f.x, x.y, acc.y);
      acc.z = fmaf(f.y, x.z, acc.z);
      acc.w = fmaf(f.y, x.w, acc.w);
    }
    *reinterpret_cast<float4*>(E + (size_t)j * nbins + bin0) = acc;
  }
}

template <int N>
__global__ void __launch_bounds__(Groups<N>::THREADS) k_colspec(float2* __restrict__ S, const float2* __restrict__ E,
                                                                const float2* __restrict__ tw, int H, float scale) {
  using P = Plan<N>;
  using GR = Groups<N>;
  constexpr int V = P::V, T = P::T, G = GR::G, HALF = N / 2 + 1;
  extern __shared__ __align__(16) float2 smem[];
  const int g = threadIdx.x / T;
  const int t = threadIdx.x - g * T;
  const int j = blockIdx.y;
  const int kx = blockIdx.x * G + g;
  const bool live = kx < HALF;
  float2* buf = smem + g * GR::BUFE;
  const float2* col = E + ((size_t)j * HALF + (live ? kx : 0)) * N;
#pragma unroll
  for (int m = 0; m < V; ++m) buf[pad32(t + T * m)] = live ? __ldg(col + t + T * m) : make_float2(0.f, 0.f);
  fftr::group_sync<T>();
  if (live && (kx == 0 || kx == N / 2)) {
    for (int ky = N / 2 + 1 + t; ky < N; ky += T) {
      const float2 e = buf[pad32(N - ky)];
      buf[pad32(ky)] = make_float2(e.x, -e.y);
    }
  }
  fftr::group_sync<T>();
  float2 v[V];
#pragma unroll
  for (int m = 0; m < V; ++m) {
    const float2 e = buf[pad32(t + T * m)];
    v[m] = make_float2(e.x * scale, e.y * scale);
  }
  fftr::group_sync<T>();  // the FFT reuses the buffer
  fftr::fft<N, true>(v, buf, t, tw);
  if (live) {
    float2* out = S + ((size_t)j * HALF + kx) * N;
#pragma unroll
    for (int m = 0; m < V; ++m) {
      const int y = t + T * m;
      if (y < H) out[y] = v[OutIndex<N>::reg(m)];
    }
  }
}

template <int N>
void launch_dense(const dfp2s_factor_dev* f, int H, int W, uint64_t seed, uint32_t frame, float scale, float* fields,
                  cudaStream_t st) {
  using GR = Groups<N>;
  constexpr int G = GR::G, HALF = N / 2 + 1;
  int log2N = 0;
  while ((1 << log2N) < N) ++log2N;
  const unsigned blocks = (unsigned)(((long long)HALF * (N / 2) + kPairs - 1) / kPairs);
  k_dense_mix<<<blocks, 128, 0, st>>>(f->dense, f->J, N, log2N, seed, frame, f->espec);
  if (GR::smem_fft > 48 * 1024)
    cudaFuncSetAttribute(k_colspec<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GR::smem_fft);
  // E carries unit-variance Gaussians: times N / sqrt2 (the noise scale), 1 / N^2 (the inverse FFT), (D/r0)^{5/6}
  const float s = scale * 0.70710678118654752440f / (float)N;
  k_colspec<N><<<dim3((HALF + G - 1) / G, f->J), GR::THREADS, GR::smem_fft, st>>>(f->scratch, f->espec, f->tw, H, s);
  dfp2s_launch_rowifft(f->scratch, fields, f->tw, N, f->J, H, W, st);
}

}  // namespace

int dfp2s_launch_sample_fields_dense(const dfp2s_factor_dev* f, int H, int W, uint64_t seed, uint32_t frame,
                                     float scale, float* fields, cudaStream_t st) {
  if (!f->dense || !f->espec || f->J > 48) return DFP2S_EINVAL;
  switch (f->N) {
    case 16: launch_dense<16>(f, H, W, seed, frame, scale, fields, st); break;
    case 32: launch_dense<32>(f, H, W, seed, frame, scale, fields, st); break;
    case 64: launch_dense<64>(f, H, W, seed, frame, scale, fields, st); break;
    case 128: launch_dense<128>(f, H, W, seed, frame, scale, fields, st); break;
    case 256: launch_dense<256>(f, H, W, seed, frame, scale, fields, st); break;
    case 512: launch_dense<512>(f, H, W, seed, frame, scale, fields, st); break;
    case 1024: launch_dense<1024>(f, H, W, seed, frame, scale, fields, st); break;
    case 2048: launch_dense<2048>(f, H, W, seed, frame, scale, fields, st); break;
    case 4096: launch_dense<4096>(f, H, W, seed, frame, scale, fields, st); break;
    default: return DFP2S_EINVAL;
  }
  return dfp2s_launch_status();
}
