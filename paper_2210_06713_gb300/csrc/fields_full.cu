// The exact FFT sampler of the full cross-spectral density of the Zernike fields (Sec. III-B; no approximation).
//
// Under the path-integrated model the J x J cross spectrum is S(k) = D(k) P Gamma(|f_k|) P^T D(k)^H (D the
// per-mode angular factors c_j sqrt(n_j+1) Theta_j(phi_k), P the J x R indicator of each mode's radial order,
// Gamma the R x R matrix of the radial spectra G_{n n'}), so chol(Gamma) gives a rank-R root and R complex
// Gaussians per frequency: the factor build (factor.cu) stores chol(Gamma) per octant bin in FP32; per frame
//   k_fullnoise  R Philox streams per bin -> the order fields eta_o = sum_r C_or z_r (R x (N/2+1) x N, plus the
//                second half of the root on the Nyquist lines kx = N/2 and ky = N/2);
//   k_colfull    one frequency column per thread group and mode: kappa_j conj(Theta_j) eta_{o_j} (the Nyquist
//                lines and corners by their own rules), Hermitian completion of columns 0 and N/2, inverse FFT
//                over ky, rows y < H, the same spectrum layout k_colgen leaves;
//   k_rowifft    (fields.cu) the row transforms and the crop.
// No mixing pass follows: the cross-correlations are in S.
#include <cuda_runtime.h>

#include "common.cuh"
#include "fft_reg.cuh"
#include "field_groups.cuh"
#include "kernels.h"

namespace {

using fftr::OutIndex;
using fftr::pad32;
using fftr::Plan;

constexpr int kMaxR = 10;  // radial orders of Noll 2..65

// Pass 0, k_fullnoise<R> (grid side N at run time): per half-plane bin (kx, ky) the R complex Gaussians z_r
// (Philox tag 5, stream r, the element layout of the factored sampler's noise) and the order fields
// eta_o = sum_{r <= o} C_or(|k|) z_r, C the Cholesky factor of the radial-order matrix Gamma(|k|).  On the lines
// kx = N/2 (0 < ky < N/2) and ky = N/2 (0 < kx < N/2) also eta'_o from streams R + r.  One thread per pair of bins
// ky = 2i, 2i + 1 (one Philox block).
template <int R>
__global__ void __launch_bounds__(256) k_fullnoise(const float* __restrict__ C, float2* __restrict__ eta, int N,
                                                   int log2N, uint64_t seed, uint32_t frame) {
  constexpr int TRI = R * (R + 1) / 2, TRIP = (TRI + 3) / 4 * 4;  // table rows padded to whole float4
  const int HALF = N / 2 + 1;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= HALF * (N / 2)) return;
  const int kx = idx >> (log2N - 1), i = idx & (N / 2 - 1);
  const uint64_t q = (uint64_t)kx * (N / 2) + i;
  float4 z[R];
#pragma unroll
  for (int r = 0; r < R; ++r) z[r] = dfp2s_gauss4(seed, dfp2s_subsequence(5u, frame, (uint32_t)r), q);
  // both bins' Cholesky rows first (all loads in flight), then eta for both bins, stored as one float4 per order
  float c[2][TRIP];
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    const int ky = 2 * i + b;
    const int ay = ky < N / 2 ? ky : N - ky;
    const int oa = kx > ay ? kx : ay, ob = kx > ay ? ay : kx;
    const float4* row = reinterpret_cast<const float4*>(C + (size_t)(oa * (oa + 1) / 2 + ob) * TRIP);
#pragma unroll
    for (int e = 0; e < TRIP / 4; ++e) {
      const float4 v = __ldg(row + e);
      c[b][4 * e] = v.x;
      c[b][4 * e + 1] = v.y;
      c[b][4 * e + 2] = v.z;
      c[b][4 * e + 3] = v.w;
    }
  }
#pragma unroll
  for (int o = 0; o < R; ++o) {
    float4 e = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int r = 0; r <= o; ++r) {
      const float c0 = c[0][o * (o + 1) / 2 + r], c1 = c[1][o * (o + 1) / 2 + r];
      e.x = fmaf(c0, z[r].x, e.x);
      e.y = fmaf(c0, z[r].y, e.y);
      e.z = fmaf(c1, z[r].z, e.z);
      e.w = fmaf(c1, z[r].w, e.w);
    }
    *reinterpret_cast<float4*>(eta + ((size_t)o * HALF + kx) * N + 2 * i) = e;
  }
  // the lines kx = N/2 (0 < ky < N/2) and ky = N/2 (0 < kx < N/2): eta' from streams R + r
  const bool colline = kx == N / 2 && i < N / 4;  // bins 2i, 2i + 1 < N/2 (bin 0 is a corner)
  const bool rowline = kx > 0 && kx < N / 2 && i == N / 4;  // bin 2i = N/2
  if (colline || rowline) {
    float4 w[R];
#pragma unroll
    for (int r = 0; r < R; ++r) w[r] = dfp2s_gauss4(seed, dfp2s_subsequence(5u, frame, (uint32_t)(R + r)), q);
    float2* nyq = eta + (size_t)R * HALF * N;
#pragma unroll
    for (int o = 0; o < R; ++o) {
      float4 e = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int r = 0; r <= o; ++r) {
        const float c0 = c[0][o * (o + 1) / 2 + r], c1 = c[1][o * (o + 1) / 2 + r];
        e.x = fmaf(c0, w[r].x, e.x);
        e.y = fmaf(c0, w[r].y, e.y);
        e.z = fmaf(c1, w[r].z, e.z);
        e.w = fmaf(c1, w[r].w, e.w);
      }
      float2* base = nyq + (size_t)o * (N + HALF);
      if (colline) {
        if (i > 0) base[2 * i] = make_float2(e.x, e.y);
        base[2 * i + 1] = make_float2(e.z, e.w);
      } else {
        base[N + kx] = make_float2(e.x, e.y);
      }
    }
  }
}

// cos(m phi), sin(m phi) of the direction of the signed frequency (x, y) != 0, by powers of the unit vector.
DFP2S_DEV float2 unit_power(float x, float y, int m) {
  const float inv = rsqrtf(x * x + y * y);
  const float2 u = make_float2(x * inv, y * inv);
  float2 p = make_float2(1.f, 0.f);
  for (int k = 0; k < m; ++k) p = make_float2(p.x * u.x - p.y * u.y, p.x * u.y + p.y * u.x);
  return p;
}

// Noll's Theta_j at the signed frequency (x, y): prefactor times cos(m phi) (even j) or sin(m phi) (odd j).
DFP2S_DEV float2 theta_at(const dfp2s_full_mode& md, float x, float y) {
  float a = 1.f;
  if (md.m != 0) {
    const float2 p = unit_power(x, y, md.m);
    a = md.odd ? p.y : p.x;
  }
  return make_float2(md.pre_re * a, md.pre_im * a);
}

// Pass 1, k_colfull: one frequency column kx of mode j per group.  E_j(kx, ky) from eta_{o_j}: kappa/sqrt2
// conj(Theta(k)) eta on generic bins, kappa/2 (conj(Theta(k)) eta + Theta(-k) eta') on the Nyquist lines, kappa
// Re(conj(Theta) eta) on the three Nyquist corners, 0 at DC (kappa = kappa0_j (D/r0)^{5/6}, the 1/N^2 of the
// inverse transform included); columns kx = 0 and N/2 completed by E(kx, N - ky) = conj E(kx, ky); then the
// inverse FFT over ky and the rows y < H to S[j][kx][y], as k_colgen leaves them for k_rowifft.
template <int N>
__global__ void __launch_bounds__(Groups<N>::THREADS) k_colfull(float2* __restrict__ S, const float2* __restrict__ eta,
                                                                const dfp2s_full_mode* __restrict__ modes, int R,
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
  const dfp2s_full_mode md = modes[j];
  const float kappa = md.kappa0 * scale;
  const float2* col = eta + ((size_t)md.o * HALF + (live ? kx : 0)) * N;
  const float2* nyq = eta + (size_t)R * HALF * N + (size_t)md.o * (N + HALF);
  const float xs = kx == N / 2 ? -(float)(N / 2) : (float)kx;  // signed frequency of the column
  if (kx != N / 2) {
    // the generic rule on every bin (the column's eta loads all in flight first); the bin ky = N/2 (a Nyquist
    // line, or a corner in column 0) and DC are rewritten by the thread that holds them
    float2 hv[V];
#pragma unroll
    for (int m = 0; m < V; ++m) hv[m] = live ? __ldg(col + t + T * m) : make_float2(0.f, 0.f);
    const float s = kappa * 0.70710678118654752440f;
#pragma unroll
    for (int m = 0; m < V; ++m) {
      const int ky = t + T * m;
      const float ys = ky < N / 2 ? (float)ky : (float)(ky - N);
      const float2 th = theta_at(md, xs, ys);
      const float2 h = hv[m];
      buf[pad32(ky)] = make_float2(s * (th.x * h.x + th.y * h.y), s * (th.x * h.y - th.y * h.x));  // conj(Theta) eta
    }
    constexpr int MH = (N / 2) / T, TH = (N / 2) % T;
    if (live && t == TH) {
      const float ys = -(float)(N / 2);
      const float2 th = theta_at(md, xs, ys);
      const float2 h = hv[MH];
      const float re = th.x * h.x + th.y * h.y, im = th.x * h.y - th.y * h.x;
      float2 e;
      if (kx == 0) {
        e = make_float2(kappa * re, 0.f);
      } else {  // -k negates x and keeps y = -N/2
        const float2 tm = theta_at(md, -xs, ys);
        const float2 h2 = __ldg(nyq + N + kx);
        e = make_float2(0.5f * kappa * (re + tm.x * h2.x - tm.y * h2.y), 0.5f * kappa * (im + tm.x * h2.y + tm.y * h2.x));
      }
      buf[pad32(N / 2)] = e;
    }
    if (live && kx == 0 && t == 0) buf[pad32(0)] = make_float2(0.f, 0.f);
  } else {
    // the column kx = N/2: corners at ky = 0 and N/2, the Nyquist line between (-k keeps x = -N/2, negates y);
    // the upper half follows from the completion
    for (int ky = t; ky <= N / 2; ky += T) {
      const float ys = ky < N / 2 ? (float)ky : -(float)(N / 2);
      const float2 th = theta_at(md, xs, ys);
      const float2 h = __ldg(col + ky);
      const float re = th.x * h.x + th.y * h.y, im = th.x * h.y - th.y * h.x;
      float2 e;
      if (ky == 0 || ky == N / 2) {
        e = make_float2(kappa * re, 0.f);
      } else {
        const float2 tm = theta_at(md, xs, -ys);
        const float2 h2 = __ldg(nyq + ky);
        e = make_float2(0.5f * kappa * (re + tm.x * h2.x - tm.y * h2.y), 0.5f * kappa * (im + tm.x * h2.y + tm.y * h2.x));
      }
      buf[pad32(ky)] = e;
    }
  }
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
  for (int m = 0; m < V; ++m) v[m] = buf[pad32(t + T * m)];
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

}  // namespace

namespace {

template <int N>
void launch_full(const dfp2s_factor_dev* f, int H, int W, uint64_t seed, uint32_t frame, float scale, float* fields,
                 cudaStream_t st) {
  using GR = Groups<N>;
  constexpr int G = GR::G, HALF = N / 2 + 1;
  const size_t sm = GR::smem;
  if (sm > 48 * 1024) cudaFuncSetAttribute(k_colfull<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GR::smem_fft);
  const unsigned blocks = (unsigned)((HALF * (N / 2) + 255) / 256);
  int log2N = 0;
  while ((1 << log2N) < N) ++log2N;
  switch (f->R) {
#define DFP2S_FULLNOISE(RR) \
  case RR: k_fullnoise<RR><<<blocks, 256, 0, st>>>(f->fchol, f->eta, N, log2N, seed, frame); break;
    DFP2S_FULLNOISE(2) DFP2S_FULLNOISE(3) DFP2S_FULLNOISE(4) DFP2S_FULLNOISE(5)
    DFP2S_FULLNOISE(6) DFP2S_FULLNOISE(7) DFP2S_FULLNOISE(8) DFP2S_FULLNOISE(9) DFP2S_FULLNOISE(10)
#undef DFP2S_FULLNOISE
    default: break;
  }
  k_colfull<N><<<dim3((HALF + G - 1) / G, f->J), GR::THREADS, GR::smem_fft, st>>>(f->scratch, f->eta, f->fmode, f->R,
                                                                                  f->tw, H, scale);
  dfp2s_launch_rowifft(f->scratch, fields, f->tw, N, f->J, H, W, st);
}

}  // namespace

int dfp2s_launch_sample_fields_full(const dfp2s_factor_dev* f, int H, int W, uint64_t seed, uint32_t frame,
                                    float scale, float* fields, cudaStream_t st) {
  if (!f->fchol || f->R < 2 || f->R > kMaxR) return DFP2S_EINVAL;
  switch (f->N) {
    case 16: launch_full<16>(f, H, W, seed, frame, scale, fields, st); break;
    case 32: launch_full<32>(f, H, W, seed, frame, scale, fields, st); break;
    case 64: launch_full<64>(f, H, W, seed, frame, scale, fields, st); break;
    case 128: launch_full<128>(f, H, W, seed, frame, scale, fields, st); break;
    case 256: launch_full<256>(f, H, W, seed, frame, scale, fields, st); break;
    case 512: launch_full<512>(f, H, W, seed, frame, scale, fields, st); break;
    case 1024: launch_full<1024>(f, H, W, seed, frame, scale, fields, st); break;
    case 2048: launch_full<2048>(f, H, W, seed, frame, scale, fields, st); break;
    case 4096: launch_full<4096>(f, H, W, seed, frame, scale, fields, st); break;
    default: return DFP2S_EINVAL;
  }
  return dfp2s_launch_status();
}
