// Zernike field sampler (Sec. III-A and III-C of the paper): white noise ->
// 2-D FFT per mode -> multiply by the per-mode spectral factor -> inverse FFT
// -> crop -> pixel-wise mixing by L.
//
// Three passes over a per-factor scratch spectrum S[j][kx][y] (complex FP32,
// kx in [0, N/2], y in [0, N); column-major in the sense that a frequency
// column is contiguous):
//   k_rowfft_noise  Philox noise made in registers, two real rows packed as one
//                   complex FFT, split into the two half spectra, written
//                   transposed so the column pass reads contiguous columns;
//   k_colfilter     column FFT, multiply by sqrt(lambda_j)/N^2, inverse column
//                   FFT, keep rows y < H (written in place);
//   k_rowifft       rows y < H: Hermitian completion of two rows packed as one
//                   complex spectrum, inverse FFT, crop to W, write fields;
// and k_mix applies a(x) = L a~(x) in place.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace {

struct BlockSync {
  DFP2S_DEV void operator()() const { __syncthreads(); }
};

// FFTs per CTA so that one CTA holds 8192 complex values (1024 threads at N/8
// threads per FFT).
inline int ffts_per_cta(int N) {
  int f = 8192 / N;
  return f > 8 ? 8 : (f < 1 ? 1 : f);
}

// -------------------------------------------------------------- pass 1
__global__ void __launch_bounds__(1024) k_rowfft_noise(float2* __restrict__ S, const float2* __restrict__ tw, int N,
                                                       int nfft, uint64_t seed, uint32_t frame) {
  extern __shared__ float2 smem[];
  const int nb = N >> 3;
  const int g = threadIdx.x / nb;  // which FFT of this CTA
  const int t = threadIdx.x - g * nb;
  const int j = blockIdx.y;
  const int rows = 2 * nfft;
  const int y0 = blockIdx.x * rows;
  float2* buf = smem + g * fpad_size(N);
  const uint64_t sub = dfp2s_subsequence(0u, frame, (uint32_t)j);
  {
    // this thread makes positions 8t .. 8t+7 of rows ya = y0 + 2g and yb = ya + 1
    const int ya = y0 + 2 * g, yb = ya + 1;
    const uint64_t qa = ((uint64_t)ya * N + 8 * t) >> 2;
    const uint64_t qb = ((uint64_t)yb * N + 8 * t) >> 2;
    const float4 a0 = dfp2s_gauss4(seed, sub, qa), a1 = dfp2s_gauss4(seed, sub, qa + 1);
    const float4 b0 = dfp2s_gauss4(seed, sub, qb), b1 = dfp2s_gauss4(seed, sub, qb + 1);
    const int x = 8 * t;
    buf[fpad(x + 0)] = make_float2(a0.x, b0.x);
    buf[fpad(x + 1)] = make_float2(a0.y, b0.y);
    buf[fpad(x + 2)] = make_float2(a0.z, b0.z);
    buf[fpad(x + 3)] = make_float2(a0.w, b0.w);
    buf[fpad(x + 4)] = make_float2(a1.x, b1.x);
    buf[fpad(x + 5)] = make_float2(a1.y, b1.y);
    buf[fpad(x + 6)] = make_float2(a1.z, b1.z);
    buf[fpad(x + 7)] = make_float2(a1.w, b1.w);
  }
  __syncthreads();
  fft_smem<false>(buf, N, t, tw, BlockSync());
  // split Z = X_a + i X_b:  X_a[k] = (Z[k] + conj Z[N-k]) / 2,  X_b[k] = (Z[k] - conj Z[N-k]) / (2i)
  const int half = N / 2 + 1;
  const int total = half * rows;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int k = idx / rows;
    const int r = idx - k * rows;
    const float2* zb = smem + (r >> 1) * fpad_size(N);
    const float2 zk = zb[fpad(k)];
    const float2 zn = zb[fpad((N - k) & (N - 1))];
    float2 x;
    if ((r & 1) == 0) {
      x = make_float2(0.5f * (zk.x + zn.x), 0.5f * (zk.y - zn.y));
    } else {
      x = make_float2(0.5f * (zk.y + zn.y), -0.5f * (zk.x - zn.x));
    }
    S[((size_t)j * half + k) * N + y0 + r] = x;
  }
}

// -------------------------------------------------------------- pass 2
__global__ void __launch_bounds__(1024) k_colfilter(float2* __restrict__ S, const float* __restrict__ mult,
                                                    const float2* __restrict__ tw, int N, int ncol, int H) {
  extern __shared__ float2 smem[];
  const int nb = N >> 3;
  const int g = threadIdx.x / nb;
  const int t = threadIdx.x - g * nb;
  const int j = blockIdx.y;
  const int half = N / 2 + 1;
  const int kx = blockIdx.x * ncol + g;
  const bool live = kx < half;
  float2* buf = smem + g * fpad_size(N);
  float2* col = S + ((size_t)j * half + (live ? kx : 0)) * N;
  const float* m = mult + ((size_t)j * half + (live ? kx : 0)) * N;
  for (int i = t; i < N; i += nb) buf[fpad(i)] = live ? col[i] : make_float2(0.f, 0.f);
  __syncthreads();
  fft_smem<false>(buf, N, t, tw, BlockSync());
  for (int i = t; i < N; i += nb) {
    const float s = live ? m[i] : 0.f;
    buf[fpad(i)] = cscale(buf[fpad(i)], s);
  }
  __syncthreads();
  fft_smem<true>(buf, N, t, tw, BlockSync());
  if (live)
    for (int i = t; i < H; i += nb) col[i] = buf[fpad(i)];
}

// -------------------------------------------------------------- pass 3
__global__ void __launch_bounds__(1024) k_rowifft(const float2* __restrict__ S, float* __restrict__ out,
                                                  const float2* __restrict__ tw, int N, int nfft, int H, int W) {
  extern __shared__ float2 smem[];
  const int nb = N >> 3;
  const int g = threadIdx.x / nb;
  const int t = threadIdx.x - g * nb;
  const int j = blockIdx.y;
  const int half = N / 2 + 1;
  const int rows = 2 * nfft;
  const int y0 = blockIdx.x * rows;
  // gather: (k, pair) with the pair index fastest; each thread reads rows ya, yb of column k (16 bytes)
  const int total = half * nfft;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int k = idx / nfft;
    const int p = idx - k * nfft;
    const int ya = y0 + 2 * p;
    const float2* colp = S + ((size_t)j * half + k) * N;
    float2 ga = make_float2(0.f, 0.f), gb = make_float2(0.f, 0.f);
    if (ya + 1 < H) {
      const float4 v = *reinterpret_cast<const float4*>(colp + ya);
      ga = make_float2(v.x, v.y);
      gb = make_float2(v.z, v.w);
    } else if (ya < H) {
      ga = colp[ya];
    }
    if (k == 0 || k == N / 2) {  // C2R convention: DC and Nyquist bins are real
      ga.y = 0.f;
      gb.y = 0.f;
    }
    float2* zb = smem + p * fpad_size(N);
    zb[fpad(k)] = make_float2(ga.x - gb.y, ga.y + gb.x);  // Z[k] = Ga + i Gb
    if (k > 0 && k < N / 2) zb[fpad(N - k)] = make_float2(ga.x + gb.y, gb.x - ga.y);  // conj Ga + i conj Gb
  }
  __syncthreads();
  fft_smem<true>(smem + g * fpad_size(N), N, t, tw, BlockSync());
  const int outs = rows * W;
  for (int idx = threadIdx.x; idx < outs; idx += blockDim.x) {
    const int r = idx / W;
    const int x = idx - r * W;
    const int y = y0 + r;
    if (y >= H) continue;
    const float2 z = smem[(r >> 1) * fpad_size(N) + fpad(x)];
    out[((size_t)j * H + y) * W + x] = (r & 1) ? z.y : z.x;
  }
}

// ------------------------------------------------------------------- mix
// a_i = sum_{j <= i} L_ij a~_j at every pixel, in place; JB >= J is the
// register bucket.
template <int JB>
__global__ void __launch_bounds__(256) k_mix(float* __restrict__ fields, const float* __restrict__ L, float scale,
                                             int J, size_t npix) {
  __shared__ float Ls[JB * JB];
  for (int i = threadIdx.x; i < JB * JB; i += blockDim.x) {
    const int r = i / JB, c = i - r * JB;
    Ls[i] = (r < J && c < J && c <= r) ? L[r * J + c] * scale : 0.f;
  }
  __syncthreads();
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npix) return;
  float v[JB];
#pragma unroll
  for (int j = 0; j < JB; ++j) v[j] = j < J ? fields[(size_t)j * npix + p] : 0.f;
#pragma unroll
  for (int i = JB - 1; i >= 0; --i) {
    if (i < J) {
      float acc = 0.f;
#pragma unroll
      for (int j = 0; j <= i; ++j) acc = fmaf(Ls[i * JB + j], v[j], acc);
      fields[(size_t)i * npix + p] = acc;
    }
  }
}

__global__ void k_philox_words(uint64_t seed, uint64_t sub, uint64_t q0, int nq, uint32_t* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nq) return;
  const uint4 w = philox_at(seed, sub, q0 + i);
  reinterpret_cast<uint4*>(out)[i] = w;
}

__global__ void k_gaussian(uint64_t seed, uint64_t sub, size_t nq, float* __restrict__ out) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nq) return;
  reinterpret_cast<float4*>(out)[i] = dfp2s_gauss4(seed, sub, i);
}

}  // namespace

// ----------------------------------------------------------------- launchers
int dfp2s_launch_sample_fields(float2* S, const float* mult, const float2* tw, int N, int J, int H, int W,
                               uint64_t seed, uint32_t frame, const float* L, float scale, float* fields,
                               cudaStream_t st) {
  const int nfft = ffts_per_cta(N);
  const int threads = nfft * (N / 8);
  const size_t sm = (size_t)nfft * fpad_size(N) * sizeof(float2);
  if (sm > 48 * 1024) {
    cudaFuncSetAttribute(k_rowfft_noise, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaFuncSetAttribute(k_colfilter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaFuncSetAttribute(k_rowifft, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  }
  const int half = N / 2 + 1;
  k_rowfft_noise<<<dim3(N / (2 * nfft), J), threads, sm, st>>>(S, tw, N, nfft, seed, frame);
  k_colfilter<<<dim3((half + nfft - 1) / nfft, J), threads, sm, st>>>(S, mult, tw, N, nfft, H);
  k_rowifft<<<dim3((H + 2 * nfft - 1) / (2 * nfft), J), threads, sm, st>>>(S, fields, tw, N, nfft, H, W);
  const size_t npix = (size_t)H * W;
  const int blocks = (int)((npix + 255) / 256);
  if (J <= 16) k_mix<16><<<blocks, 256, 0, st>>>(fields, L, scale, J, npix);
  else if (J <= 40) k_mix<40><<<blocks, 256, 0, st>>>(fields, L, scale, J, npix);
  else k_mix<64><<<blocks, 256, 0, st>>>(fields, L, scale, J, npix);
  return cudaGetLastError() == cudaSuccess ? DFP2S_OK : DFP2S_ECUDA;
}

int dfp2s_launch_philox_words(uint64_t seed, uint64_t sub, uint64_t q0, int nq, uint32_t* out, cudaStream_t st) {
  k_philox_words<<<(nq + 255) / 256, 256, 0, st>>>(seed, sub, q0, nq, out);
  return cudaGetLastError() == cudaSuccess ? DFP2S_OK : DFP2S_ECUDA;
}

int dfp2s_launch_gaussian(uint64_t seed, uint64_t sub, size_t nq, float* out, cudaStream_t st) {
  k_gaussian<<<(unsigned)((nq + 255) / 256), 256, 0, st>>>(seed, sub, nq, out);
  return cudaGetLastError() == cudaSuccess ? DFP2S_OK : DFP2S_ECUDA;
}
