// Phase-to-space weights (Sec. II-C of the paper).
//
// Exact form (the fallback and the judge of the surrogate): for each pixel the
// PSF of Eq. (2), h = |DFT{P exp(-j phi)}|^2 with phi = sum_{j >= 4} a_j Z_j,
// on a 64 x 64 pupil grid whose aperture (radius 16 samples) fills the central
// 33 x 33 window, so the DFT is pruned to that window on input and to the 33 x 33
// PSF window on output: X = F U F^T with F[k][i] = exp(-2 pi i (k-16)(i-16)/64).
// h is normalised to unit sum and projected on the orthonormal basis under the
// constraint that the projected PSF keeps that unit sum (reading R28 of the
// least-squares projection of Eq. p2s PSF): with s_k = sum_u phi_k(u),
// w = Phi^T h + s (1 - s^T Phi^T h) / (s^T s).  FP32 throughout (tables built
// in FP64).
//
// Learned form: the surrogate network J -> 256 -> 256 -> K with GELU (erf), its
// output moved onto s^T w = 1 the same way.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>

#include "common.cuh"
#include "kernels.h"
#include "zernike.cuh"

namespace {

constexpr int KS = 33;
constexpr int KS2 = KS * KS;
constexpr int PB = 8;       // pixels per batch of the exact kernel
constexpr int NT = 256;     // threads of the exact kernel

__global__ void k_p2s_tables(int J, int K, const float* __restrict__ basis, float* __restrict__ zt,
                             float* __restrict__ mask, float2* __restrict__ dft, float* __restrict__ phiT) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= KS2) return;
  const int i = q / KS, l = q - i * KS;  // window row (y) and column (x)
  const int iy = i - 16, ix = l - 16;
  const double x = ix / 16.0, y = iy / 16.0;
  const double rho = sqrt(x * x + y * y), th = atan2(y, x);
  const bool inside = ix * ix + iy * iy <= 256;
  mask[q] = inside ? 1.f : 0.f;
  for (int jj = 0; jj < J - 2; ++jj) {
    const double z = dfp2s_zernike(jj + 4, rho, th);
    zt[(size_t)jj * KS2 + q] = inside ? (float)z : 0.f;
  }
  // DFT matrix entry (k = i, index = l): exp(-2 pi i (k-16)(i-16)/64)
  {
    const double pi = 3.14159265358979323846;
    const double a = -2.0 * pi * (double)(iy * ix) / 64.0;
    dft[q] = make_float2((float)cos(a), (float)sin(a));
  }
  for (int kk = 0; kk < K; ++kk) phiT[(size_t)q * K + kk] = basis[(size_t)kk * KS2 + q];
}

// s_k = sum_u phi_k(u) and s_k / (s^T s), FP64 sums (one block)
__global__ void k_flux_tables(const float* __restrict__ basis, int K, float* __restrict__ flux) {
  __shared__ double sk[DFP2S_MAX_K];
  __shared__ double ss;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    double t = 0.0;
    for (int q = 0; q < KS2; ++q) t += (double)basis[(size_t)k * KS2 + q];
    sk[k] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < K; ++k) t += sk[k] * sk[k];
    ss = t;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    flux[k] = (float)sk[k];
    flux[K + k] = (float)(sk[k] / ss);
  }
}

DFP2S_DEV float warp_sum(float v) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

template <typename WT>
DFP2S_DEV void store_w(WT* w, size_t idx, float v);
template <>
DFP2S_DEV void store_w<float>(float* w, size_t idx, float v) { w[idx] = v; }
template <>
DFP2S_DEV void store_w<__nv_bfloat16>(__nv_bfloat16* w, size_t idx, float v) { w[idx] = __float2bfloat16_rn(v); }

template <typename WT, bool PSF_OUT>
__global__ void __launch_bounds__(NT) k_p2s_exact(const float* __restrict__ fields, int J, int npix, int K,
                                                  const float* __restrict__ zt, const float* __restrict__ mask,
                                                  const float2* __restrict__ dft, const float* __restrict__ phiT,
                                                  const float* __restrict__ flux, WT* __restrict__ w) {
  extern __shared__ float4 smem_f4[];
  float2* F = reinterpret_cast<float2*>(smem_f4);
  float2* U = F + KS2;
  float2* T = U + KS2;
  float (*ph)[KS2] = reinterpret_cast<float (*)[KS2]>(T + KS2);
  float (*a_s)[DFP2S_MAX_J] = reinterpret_cast<float (*)[DFP2S_MAX_J]>(&ph[PB][0]);
  float* hsum = &a_s[PB][0];
  float* red = hsum + PB;
  float* fred = red + NT / 32;  // per-warp parts of each pixel's flux s^T w (PB x 4 per pixel group)
  const int tid = threadIdx.x;
  for (int q = tid; q < KS2; q += NT) F[q] = dft[q];
  const int nbatch = (npix + PB - 1) / PB;
  for (int batch = blockIdx.x; batch < nbatch; batch += gridDim.x) {
    const int p0 = batch * PB;
    __syncthreads();
    for (int idx = tid; idx < PB * J; idx += NT) {
      const int p = idx / J, j = idx - p * J;
      a_s[p][j] = (p0 + p < npix) ? fields[(size_t)j * npix + p0 + p] : 0.f;
    }
    __syncthreads();
    // phase on the pupil window for the PB pixels (modes Noll 4..J+1 = fields 2..J-1)
    for (int q = tid; q < KS2; q += NT) {
      float acc[PB];
#pragma unroll
      for (int p = 0; p < PB; ++p) acc[p] = 0.f;
      for (int jj = 0; jj < J - 2; ++jj) {
        const float z = __ldg(zt + (size_t)jj * KS2 + q);
#pragma unroll
        for (int p = 0; p < PB; ++p) acc[p] = fmaf(a_s[p][jj + 2], z, acc[p]);
      }
#pragma unroll
      for (int p = 0; p < PB; ++p) ph[p][q] = acc[p];
    }
    __syncthreads();
    for (int p = 0; p < PB; ++p) {
      // U = P exp(-j phi)
      for (int q = tid; q < KS2; q += NT) {
        float s, c;
        sincosf(ph[p][q], &s, &c);
        const float m = __ldg(mask + q);
        U[q] = make_float2(m * c, -m * s);
      }
      __syncthreads();
      // T[ky][l] = sum_i F[ky][i] U[i][l]
      for (int o = tid; o < KS2; o += NT) {
        const int ky = o / KS, l = o - ky * KS;
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll 11
        for (int i = 0; i < KS; ++i) {
          const float2 f = F[ky * KS + i], u = U[i * KS + l];
          acc.x = fmaf(f.x, u.x, fmaf(-f.y, u.y, acc.x));
          acc.y = fmaf(f.x, u.y, fmaf(f.y, u.x, acc.y));
        }
        T[o] = acc;
      }
      __syncthreads();
      // X[ky][kx] = sum_l T[ky][l] F[kx][l];  h = |X|^2
      float part = 0.f;
      for (int o = tid; o < KS2; o += NT) {
        const int ky = o / KS, kx = o - ky * KS;
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll 11
        for (int l = 0; l < KS; ++l) {
          const float2 t = T[ky * KS + l], f = F[kx * KS + l];
          acc.x = fmaf(t.x, f.x, fmaf(-t.y, f.y, acc.x));
          acc.y = fmaf(t.x, f.y, fmaf(t.y, f.x, acc.y));
        }
        const float h = fmaf(acc.x, acc.x, acc.y * acc.y);
        ph[p][o] = h;
        part += h;
      }
      for (int off = 16; off > 0; off >>= 1) part += __shfl_down_sync(0xffffffffu, part, off);
      if ((tid & 31) == 0) red[tid >> 5] = part;
      __syncthreads();
      if (tid == 0) {
        float s = 0.f;
        for (int i = 0; i < NT / 32; ++i) s += red[i];
        hsum[p] = s;
      }
    }
    __syncthreads();
    if (PSF_OUT) {  // the normalised PSFs themselves, npix x 1089 FP32
      float* hout = reinterpret_cast<float*>(w);
      for (int idx = tid; idx < PB * KS2; idx += NT) {
        const int p = idx / KS2, q = idx - p * KS2;
        if (p0 + p < npix) hout[(size_t)(p0 + p) * KS2 + q] = ph[p][q] / hsum[p];
      }
      continue;
    }
    // w[p][k] = sum_q Phi[k][q] h[p][q] / sum h[p], then w += (1 - s^T w) s / (s^T s)
    {
      const int kk = tid % 128;
      const int pg = tid / 128;  // pixels pg*4 .. pg*4+3
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      if (kk < K) {
        for (int q = 0; q < KS2; ++q) {
          const float ph_ = __ldg(phiT + (size_t)q * K + kk);
#pragma unroll
          for (int i = 0; i < 4; ++i) acc[i] = fmaf(ph_, ph[pg * 4 + i][q], acc[i]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[i] = acc[i] / hsum[pg * 4 + i];
      }
      const float sk = kk < K ? __ldg(flux + kk) : 0.f;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float m = warp_sum(sk * acc[i]);
        if ((tid & 31) == 0) fred[(pg * 4 + i) * 4 + ((tid >> 5) & 3)] = m;
      }
      __syncthreads();
      if (kk < K) {
        const float gk = __ldg(flux + K + kk);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float* fr = fred + (pg * 4 + i) * 4;
          const float m = (fr[0] + fr[1]) + (fr[2] + fr[3]);
          const int p = p0 + pg * 4 + i;
          if (p < npix) store_w<WT>(w, (size_t)p * K + kk, fmaf(1.f - m, gk, acc[i]));
        }
      }
    }
  }
}

// ----------------------------------------------------------- surrogate (SIMT)
constexpr int MP = 32;  // pixels per CTA
constexpr int HID = 256;

DFP2S_DEV float gelu_erf(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }

// W1t: J x 256, W2t: 256 x 256, W3t: 256 x K (transposed so threads read consecutive outputs)
template <typename WT>
__global__ void __launch_bounds__(HID) k_p2s_mlp(const float* __restrict__ fields, int J, int npix, int K,
                                                 const float* __restrict__ W1t, const float* __restrict__ b1,
                                                 const float* __restrict__ W2t, const float* __restrict__ b2,
                                                 const float* __restrict__ W3t, const float* __restrict__ b3,
                                                 const float* __restrict__ in_scale, const float* __restrict__ out_scale,
                                                 const float* __restrict__ out_shift, const float* __restrict__ flux,
                                                 WT* __restrict__ w) {
  extern __shared__ float4 smem_f4[];
  float (*h1)[HID] = reinterpret_cast<float (*)[HID]>(smem_f4);
  float (*h2)[HID] = h1 + MP;
  float (*xin)[DFP2S_MAX_J] = reinterpret_cast<float (*)[DFP2S_MAX_J]>(h2 + MP);
  const int tid = threadIdx.x;
  const int p0 = blockIdx.x * MP;
  for (int idx = tid; idx < MP * J; idx += HID) {
    const int p = idx % MP, j = idx / MP;
    xin[p][j] = (p0 + p < npix) ? fields[(size_t)j * npix + p0 + p] * in_scale[j] : 0.f;
  }
  __syncthreads();
  {
    float acc[MP];
    const float bb = b1[tid];
#pragma unroll
    for (int p = 0; p < MP; ++p) acc[p] = bb;
    for (int i = 0; i < J; ++i) {
      const float wv = __ldg(W1t + (size_t)i * HID + tid);
#pragma unroll
      for (int p = 0; p < MP; ++p) acc[p] = fmaf(wv, xin[p][i], acc[p]);
    }
#pragma unroll
    for (int p = 0; p < MP; ++p) h1[p][tid] = gelu_erf(acc[p]);
  }
  __syncthreads();
  {
    float acc[MP];
    const float bb = b2[tid];
#pragma unroll
    for (int p = 0; p < MP; ++p) acc[p] = bb;
    for (int i = 0; i < HID; ++i) {
      const float wv = __ldg(W2t + (size_t)i * HID + tid);
#pragma unroll
      for (int p = 0; p < MP; ++p) acc[p] = fmaf(wv, h1[p][i], acc[p]);
    }
#pragma unroll
    for (int p = 0; p < MP; ++p) h2[p][tid] = gelu_erf(acc[p]);
  }
  __syncthreads();
  if (tid < K) {
    float acc[MP];
    const float bb = b3[tid];
#pragma unroll
    for (int p = 0; p < MP; ++p) acc[p] = bb;
    for (int i = 0; i < HID; ++i) {
      const float wv = __ldg(W3t + (size_t)i * K + tid);
#pragma unroll
      for (int p = 0; p < MP; ++p) acc[p] = fmaf(wv, h2[p][i], acc[p]);
    }
    const float sc = out_scale[tid], sh = out_shift[tid];
#pragma unroll
    for (int p = 0; p < MP; ++p) h1[p][tid] = fmaf(acc[p], sc, sh);  // h1 is free after layer 2
  }
  __syncthreads();
  // the flux s^T w of each pixel's weights (warp w: pixels w, w + 8, ...), then w += (1 - s^T w) s / (s^T s)
  float* mass = &xin[0][0];
  {
    const int warp = tid >> 5, lane = tid & 31;
    for (int p = warp; p < MP; p += HID / 32) {
      float m = 0.f;
      for (int k = lane; k < K; k += 32) m = fmaf(h1[p][k], __ldg(flux + k), m);
      m = warp_sum(m);
      if (lane == 0) mass[p] = m;
    }
  }
  __syncthreads();
  if (tid < K) {
    const float gk = __ldg(flux + K + tid);
    for (int p = 0; p < MP; ++p)
      if (p0 + p < npix) store_w<WT>(w, (size_t)(p0 + p) * K + tid, fmaf(1.f - mass[p], gk, h1[p][tid]));
  }
}

}  // namespace

int dfp2s_p2s_build_tables(dfp2s_p2s_dev* p, cudaStream_t st) {
  k_p2s_tables<<<(KS2 + 127) / 128, 128, 0, st>>>(p->J, p->K, p->basis, p->zt, p->mask, p->dft, p->phiT);
  if (p->flux) k_flux_tables<<<1, 128, 0, st>>>(p->basis, p->K, p->flux);  // absent in PSF-only tables
  return dfp2s_launch_status();
}

int dfp2s_launch_p2s_exact(const dfp2s_p2s_dev* p, const float* fields, int H, int W, void* w, int w_dtype,
                           cudaStream_t st) {
  const int npix = H * W;
  const int nbatch = (npix + PB - 1) / PB;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = nbatch < sms * 3 ? nbatch : sms * 3;
  const size_t sm = 3 * KS2 * sizeof(float2) + (PB * KS2 + PB * DFP2S_MAX_J + PB + NT / 32 + 4 * PB) * sizeof(float);
  cudaFuncSetAttribute(k_p2s_exact<__nv_bfloat16, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  cudaFuncSetAttribute(k_p2s_exact<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  cudaFuncSetAttribute(k_p2s_exact<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (w_dtype == DFP2S_W_PSF)
    k_p2s_exact<float, true><<<grid, NT, sm, st>>>(fields, p->J, npix, p->K, p->zt, p->mask, p->dft, p->phiT,
                                                   p->flux, (float*)w);
  else if (w_dtype == DFP2S_W_BF16)
    k_p2s_exact<__nv_bfloat16, false><<<grid, NT, sm, st>>>(fields, p->J, npix, p->K, p->zt, p->mask, p->dft,
                                                          p->phiT, p->flux, (__nv_bfloat16*)w);
  else
    k_p2s_exact<float, false><<<grid, NT, sm, st>>>(fields, p->J, npix, p->K, p->zt, p->mask, p->dft, p->phiT,
                                                    p->flux, (float*)w);
  return dfp2s_launch_status();
}

int dfp2s_launch_p2s_mlp(const dfp2s_p2s_dev* p, const float* fields, int H, int W, void* w, int w_dtype,
                         cudaStream_t st) {
  const int npix = H * W;
  const int grid = (npix + MP - 1) / MP;
  const size_t sm = (2 * MP * HID + MP * DFP2S_MAX_J) * sizeof(float);
  cudaFuncSetAttribute(k_p2s_mlp<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  cudaFuncSetAttribute(k_p2s_mlp<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (w_dtype == DFP2S_W_BF16)
    k_p2s_mlp<__nv_bfloat16><<<grid, HID, sm, st>>>(fields, p->J, npix, p->K, p->W1, p->b1, p->W2, p->b2, p->W3,
                                                  p->b3, p->in_scale, p->out_scale, p->out_shift, p->flux, (__nv_bfloat16*)w);
  else
    k_p2s_mlp<float><<<grid, HID, sm, st>>>(fields, p->J, npix, p->K, p->W1, p->b1, p->W2, p->b2, p->W3, p->b3,
                                          p->in_scale, p->out_scale, p->out_shift, p->flux, (float*)w);
  return dfp2s_launch_status();
}
