// Zernike field sampler (Sec. III-A and III-C of the paper): white noise ->
// 2-D FFT per mode -> multiply by the per-mode spectral factor -> inverse FFT
// -> crop -> pixel-wise mixing by L.
//
// The white noise is drawn in the Fourier domain: E = FFT2(e) of real white
// noise e is Hermitian white noise (variance N^2 per bin, N^2/2 per real and
// imaginary part off the four self-conjugate bins), so the sampler draws E from
// Philox directly (same distribution, no forward transform).  Two passes over a
// per-factor scratch spectrum S[j][kx][y] (complex FP32, kx in [0, N/2], rows
// y < H; a frequency column is contiguous), each FFT done in registers by a
// group of threads (fft_reg.cuh):
//   k_colgen   one column kx per group: Philox noise E(kx, .), Hermitian in ky
//              for kx = 0 and N/2, times sqrt(lambda_j)/N^2, inverse FFT over ky,
//              rows y < H;
//   k_rowifft  2G rows per block read through a tile; per row pair the
//              Hermitian completion of Ga + i Gb over kx, inverse FFT, rows to
//              the fields, cropped to W;
// and k_mix applies a(x) = L a~(x) in place.
#include <cuda_runtime.h>

#include "common.cuh"
#include "fft_reg.cuh"
#include "field_groups.cuh"
#include "kernels.h"

namespace {

using fftr::OutIndex;
using fftr::pad32;
using fftr::Plan;


// -------------------------------------------------------------- pass 1
// One frequency column kx of mode j per group.  The column's Fourier-domain white noise E(kx, ky)
// (Re, Im = Gaussians 2 (kx N + ky) + {0, 1}; one Philox block covers ky = 2i, 2i + 1) is staged in
// shared memory in natural order; columns kx = 0 and N/2 are made Hermitian in ky (E(kx, N - ky) =
// conj E(kx, ky), real at ky = 0 and N/2 with variance N^2).  Then E (N / sqrt 2) sqrt(lambda_j) / N^2,
// the inverse FFT over ky, and the rows y < H to S[j][kx][y].
template <int N>
DFP2S_DEV void colgen_body(float2* __restrict__ S, const float* __restrict__ mult, const float2* __restrict__ tw, int H,
                           uint64_t seed, uint32_t frame, float cN) {
  using P = Plan<N>;
  using GR = Groups<N>;
  constexpr int V = P::V, T = P::T, G = GR::G, HALF = N / 2 + 1;
  extern __shared__ __align__(16) float2 smem[];
  const int g = threadIdx.x / T;
  const int t = threadIdx.x - g * T;
  const int j = blockIdx.y;
  const int kx = blockIdx.x * G + g;
  const bool live = kx < HALF;  // dead groups still join the block-wide exchanges when T > 32
  float2* buf = smem + g * GR::BUFE;
  {
    const uint64_t sub = dfp2s_subsequence(0u, frame, (uint32_t)j);
    const uint64_t q0 = (uint64_t)(live ? kx : 0) * (N / 2);
#pragma unroll
    for (int c = 0; c < V / 2; ++c) {
      const int i = t + T * c;
      const float4 z = dfp2s_gauss4(seed, sub, q0 + i);
      buf[pad32(2 * i)] = make_float2(z.x, z.y);
      buf[pad32(2 * i + 1)] = make_float2(z.z, z.w);
    }
  }
  fftr::group_sync<T>();
  if (live && (kx == 0 || kx == N / 2)) {
    // the upper half is written from the lower half only, and bins 0 and N/2 by thread 0 alone
    for (int ky = N / 2 + 1 + t; ky < N; ky += T) {
      const float2 e = buf[pad32(N - ky)];
      buf[pad32(ky)] = make_float2(e.x, -e.y);
    }
    if (t == 0) {
      buf[pad32(0)] = make_float2(buf[pad32(0)].x * 1.41421356237309505f, 0.f);
      buf[pad32(N / 2)] = make_float2(buf[pad32(N / 2)].x * 1.41421356237309505f, 0.f);
    }
  }
  fftr::group_sync<T>();
  const float* mc = mult + ((size_t)j * HALF + (live ? kx : 0)) * N;
  float2 v[V];
#pragma unroll
  for (int m = 0; m < V; ++m) {
    const float s = live ? __ldg(mc + t + T * m) * cN : 0.f;
    v[m] = cscale(buf[pad32(t + T * m)], s);
  }
  fftr::group_sync<T>();  // the FFT reuses the buffer
  fftr::fft<N, true>(v, buf, t, tw);
  if (live) {
    float2* col = S + ((size_t)j * HALF + kx) * N;
#pragma unroll
    for (int m = 0; m < V; ++m) {
      const int y = t + T * m;
      if (y < H) col[y] = v[OutIndex<N>::reg(m)];
    }
  }
}

template <int N>
__global__ void __launch_bounds__(Groups<N>::THREADS) k_colgen(float2* __restrict__ S, const float* __restrict__ mult,
                                                               const float2* __restrict__ tw, int H, uint64_t seed,
                                                               uint32_t frame, float cN) {
  colgen_body<N>(S, mult, tw, H, seed, frame, cN);
}
// The same with three blocks per SM (80 registers): the noise phase is issue-bound, and the extra warps hide the
// latencies of its dependent chains
template <int N>
__global__ void __launch_bounds__(Groups<N>::THREADS, 3) k_colgen3(float2* __restrict__ S, const float* __restrict__ mult,
                                                                   const float2* __restrict__ tw, int H, uint64_t seed,
                                                                   uint32_t frame, float cN) {
  colgen_body<N>(S, mult, tw, H, seed, frame, cN);
}

// -------------------------------------------------------------- pass 2
template <int N>
__global__ void __launch_bounds__(Groups<N>::THREADS) k_rowifft(const float2* __restrict__ S, float* __restrict__ out,
                                                                const float2* __restrict__ tw, int H, int W) {
  using P = Plan<N>;
  using GR = Groups<N>;
  constexpr int V = P::V, T = P::T, G = GR::G, HALF = N / 2 + 1;
  extern __shared__ __align__(16) float2 smem[];
  const int g = threadIdx.x / T;
  const int t = threadIdx.x - g * T;
  const int j = blockIdx.y;
  const int y0 = blockIdx.x * 2 * G;
  const float2* Sj = S + (size_t)j * HALF * N;
  // the tile: every element an asynchronous 8-byte copy straight into its padded place, so that all of a
  // thread's loads are in flight at once (no register staging); rows past H are zero
  constexpr int TOT = HALF * 2 * G;
  constexpr int PER = (TOT + GR::THREADS - 1) / GR::THREADS;
  const uint32_t tile = (uint32_t)__cvta_generic_to_shared(smem);
#pragma unroll
  for (int b = 0; b < PER; ++b) {
    const int i = threadIdx.x + b * GR::THREADS;
    if (i < TOT) {
      const int k = i / (2 * G), r = i - k * (2 * G);
      if (y0 + r < H)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(tile + (uint32_t)((k * GR::TS + r) * 8)),
                     "l"(Sj + (size_t)k * N + y0 + r)
                     : "memory");
      else
        smem[k * GR::TS + r] = make_float2(0.f, 0.f);
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  // C2R convention: the DC and Nyquist bins are real
  for (int i = threadIdx.x; i < 4 * G; i += GR::THREADS) smem[(i < 2 * G ? 0 : N / 2) * GR::TS + (i % (2 * G))].y = 0.f;
  __syncthreads();
  // Z[n] = Ga[n] + i Gb[n] for n <= N/2, conj Ga[N-n] + i conj Gb[N-n] above
  float2 v[V];
#pragma unroll
  for (int m = 0; m < V; ++m) {
    const int n = t + T * m;
    if (n <= N / 2) {
      const float2 ga = smem[n * GR::TS + 2 * g], gb = smem[n * GR::TS + 2 * g + 1];
      v[m] = make_float2(ga.x - gb.y, ga.y + gb.x);
    } else {
      const float2 ga = smem[(N - n) * GR::TS + 2 * g], gb = smem[(N - n) * GR::TS + 2 * g + 1];
      v[m] = make_float2(ga.x + gb.y, gb.x - ga.y);
    }
  }
  __syncthreads();  // the groups' FFT buffers overlay the tile
  fftr::fft<N, true>(v, smem + g * GR::BUFE, t, tw);
  const int ya = y0 + 2 * g, yb = ya + 1;
  float* oa = out + ((size_t)j * H + ya) * W;
  float* ob = oa + W;
#pragma unroll
  for (int m = 0; m < V; ++m) {
    const int x = t + T * m;
    if (x < W) {
      const float2 z = v[OutIndex<N>::reg(m)];
      if (ya < H) oa[x] = z.x;
      if (yb < H) ob[x] = z.y;
    }
  }
}

// ------------------------------------------------------------------- mix
// a_i = sum_{j <= i} L_ij a~_j at every pixel, in place; JB >= J (a multiple of
// 4) is the register bucket.  Each thread mixes a pair of adjacent pixels
// (8-byte loads and stores; needs an even pixel count) and reads four
// coefficients of L per shared-memory load.
template <int JB, bool AR>
__global__ void __launch_bounds__(128, 4) k_mix_pairs(float* __restrict__ fields, const float* __restrict__ L,
                                                   float scale, int J, size_t npix, const float* __restrict__ prev,
                                                   float alpha) {
  __shared__ __align__(16) float Ls[JB * JB];
  for (int i = threadIdx.x; i < JB * JB; i += blockDim.x) {
    const int r = i / JB, c = i - r * JB;
    Ls[i] = (r < J && c < J && c <= r) ? L[r * J + c] * scale : 0.f;
  }
  __syncthreads();
  const size_t p = 2 * ((size_t)blockIdx.x * blockDim.x + threadIdx.x);
  if (p >= npix) return;
  float2 v[JB];
#pragma unroll
  for (int j = 0; j < JB; ++j)
    v[j] = j < J ? *reinterpret_cast<const float2*>(fields + (size_t)j * npix + p) : make_float2(0.f, 0.f);
  // rows in a runtime loop (so the compiler does not hoist L into registers), the
  // triangle's columns as uniform branches over an unrolled loop
  for (int i = 0; i < J; ++i) {
    float ax = 0.f, ay = 0.f;
#pragma unroll
    for (int j4 = 0; j4 < JB / 4; ++j4) {
      if (4 * j4 <= i) {
        const float4 l = *reinterpret_cast<const float4*>(Ls + i * JB + 4 * j4);
        ax = fmaf(l.x, v[4 * j4].x, ax);
        ay = fmaf(l.x, v[4 * j4].y, ay);
        ax = fmaf(l.y, v[4 * j4 + 1].x, ax);
        ay = fmaf(l.y, v[4 * j4 + 1].y, ay);
        ax = fmaf(l.z, v[4 * j4 + 2].x, ax);
        ay = fmaf(l.z, v[4 * j4 + 2].y, ay);
        ax = fmaf(l.w, v[4 * j4 + 3].x, ax);
        ay = fmaf(l.w, v[4 * j4 + 3].y, ay);
      }
    }
    if (AR) {  // a_t = alpha a_{t-1} + sqrt(1 - alpha^2) (L a~)_t, the root folded into `scale`
      const float2 q = *reinterpret_cast<const float2*>(prev + (size_t)i * npix + p);
      ax = fmaf(alpha, q.x, ax);
      ay = fmaf(alpha, q.y, ay);
    }
    *reinterpret_cast<float2*>(fields + (size_t)i * npix + p) = make_float2(ax, ay);
  }
}

// One pixel per thread (odd pixel counts).
template <int JB, bool AR>
__global__ void __launch_bounds__(128, 4) k_mix(float* __restrict__ fields, const float* __restrict__ L, float scale,
                                             int J, size_t npix, const float* __restrict__ prev, float alpha) {
  __shared__ __align__(16) float Ls[JB * JB];
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
  for (int i = 0; i < J; ++i) {
    float acc = 0.f;
#pragma unroll
    for (int j4 = 0; j4 < JB / 4; ++j4) {
      if (4 * j4 <= i) {
        const float4 l = *reinterpret_cast<const float4*>(Ls + i * JB + 4 * j4);
        acc = fmaf(l.x, v[4 * j4], acc);
        acc = fmaf(l.y, v[4 * j4 + 1], acc);
        acc = fmaf(l.z, v[4 * j4 + 2], acc);
        acc = fmaf(l.w, v[4 * j4 + 3], acc);
      }
    }
    if (AR) acc = fmaf(alpha, prev[(size_t)i * npix + p], acc);
    fields[(size_t)i * npix + p] = acc;
  }
}

template <int JB, bool AR>
void launch_mix(float* fields, const float* L, float scale, int J, size_t npix, const float* prev, float alpha,
                cudaStream_t st) {
  if constexpr (JB <= 40) {
    if (npix % 2 == 0) {
      const size_t pairs = npix / 2;
      k_mix_pairs<JB, AR><<<(unsigned)((pairs + 127) / 128), 128, 0, st>>>(fields, L, scale, J, npix, prev, alpha);
      return;
    }
  }
  k_mix<JB, AR><<<(unsigned)((npix + 127) / 128), 128, 0, st>>>(fields, L, scale, J, npix, prev, alpha);
}

template <bool AR>
void launch_mix_any(float* fields, const float* L, float scale, int J, size_t npix, const float* prev, float alpha,
                    cudaStream_t st) {
  if (J <= 16) launch_mix<16, AR>(fields, L, scale, J, npix, prev, alpha, st);
  else if (J <= 40) launch_mix<40, AR>(fields, L, scale, J, npix, prev, alpha, st);
  else launch_mix<64, AR>(fields, L, scale, J, npix, prev, alpha, st);
}

// ------------------------------------------------------------ subharmonics (Sec. IV-B; reading R31)
DFP2S_DEV float dfp2s_pow3f(int k) {  // 3^k, exact in FP32 for k <= 15
  float r = 1.f;
  for (int i = 0; i < k; ++i) r *= 3.f;
  return r;
}

// This frame's complex amplitudes c_{j,p,d} = s_{j,p,d} (g_re + i g_im): Philox tag 6, subsequence mode j,
// counter 4 p + k for directions 2k, 2k + 1 (levels counted from 0 here).  One thread per (j, p, k).
__global__ void k_sh_coeffs(const float* __restrict__ amp, int J, int levels, uint64_t seed, uint32_t frame,
                            float2* __restrict__ coef) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= J * levels * 4) return;
  const int j = i / (levels * 4), r = i - j * levels * 4;  // r = 4 p + k
  const float4 g = dfp2s_gauss4(seed, dfp2s_subsequence(6u, frame, (uint32_t)j), (uint64_t)r);
  const size_t e = (size_t)j * levels * 8 + 2 * r;  // direction 2k of level p: 8 p + 2 k = 2 r
  coef[e] = make_float2(amp[e] * g.x, amp[e] * g.y);
  coef[e + 1] = make_float2(amp[e + 1] * g.z, amp[e + 1] * g.w);
}

// Adds sum_{p,d} Re[c_{j,p,d} u^n v^m] to every unit field, u = e^{2 pi i x / (N 3^p)}, v = e^{2 pi i y / (N 3^p)}
// (pixel (y, x)).  Per row the m-sums C_n = sum_m c_{(n,m)} v^m are formed once, so a pixel takes
// Re(C_0) + Re(C_1 u) + Re(C_{-1} conj u) = A + B u.x + D u.y per mode and level.  One CTA per row.
__global__ void __launch_bounds__(256) k_sh_add(float* __restrict__ fields, int J, int H, int W, int N, int levels,
                                             const float2* __restrict__ coef) {
  extern __shared__ float4 shc[];  // [j][p]: A, B, D, 0
  const int y = blockIdx.x;
  const size_t plane = (size_t)H * W;
  for (int e = threadIdx.x; e < J * levels; e += blockDim.x) {
    const int p = e % levels;
    const float2* c = coef + (size_t)e * 8;  // e = j * levels + p
    float sv, cv;
    sincospif(2.f * (float)y / ((float)N * dfp2s_pow3f(p + 1)), &sv, &cv);
    // directions: 0 (-1,-1), 1 (0,-1), 2 (1,-1), 3 (-1,0), 4 (1,0), 5 (-1,1), 6 (0,1), 7 (1,1)
    const float2 vp = make_float2(cv, sv), vm = make_float2(cv, -sv);
    const float2 cm1 = make_float2(c[0].x * vm.x - c[0].y * vm.y + c[3].x + c[5].x * vp.x - c[5].y * vp.y,
                                   c[0].x * vm.y + c[0].y * vm.x + c[3].y + c[5].x * vp.y + c[5].y * vp.x);
    const float c0x = c[1].x * vm.x - c[1].y * vm.y + c[6].x * vp.x - c[6].y * vp.y;
    const float2 c1 = make_float2(c[2].x * vm.x - c[2].y * vm.y + c[4].x + c[7].x * vp.x - c[7].y * vp.y,
                                  c[2].x * vm.y + c[2].y * vm.x + c[4].y + c[7].x * vp.y + c[7].y * vp.x);
    // Re(C_1 u) + Re(C_-1 conj u) = (C1.x + Cm1.x) u.x + (Cm1.y - C1.y) u.y
    shc[e] = make_float4(c0x, c1.x + cm1.x, cm1.y - c1.y, 0.f);
  }
  __syncthreads();
  for (int x = threadIdx.x; x < W; x += blockDim.x) {
    float2 u[12];
#pragma unroll
    for (int p = 0; p < 12; ++p)
      if (p < levels) sincospif(2.f * (float)x / ((float)N * dfp2s_pow3f(p + 1)), &u[p].y, &u[p].x);
    float* f = fields + (size_t)y * W + x;
    for (int j0 = 0; j0 < J; j0 += 4) {  // four modes at a time: their loads in flight together
      float v[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] = j0 + k < J ? f[(size_t)(j0 + k) * plane] : 0.f;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        float add = 0.f;
#pragma unroll
        for (int p = 0; p < 12; ++p) {
          if (p < levels && j0 + k < J) {
            const float4 t = shc[(j0 + k) * levels + p];
            add += t.x + t.y * u[p].x + t.z * u[p].y;
          }
        }
        v[k] += add;
      }
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (j0 + k < J) f[(size_t)(j0 + k) * plane] = v[k];
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
// variant: the column pass's kernel, 0 = k_colgen (the compiler's register budget), 1 = k_colgen3 (three blocks
// per SM, at most 80 registers; N <= 2048), -1 = the default (k_colgen3 at N = 1024 only).  Same results.
template <int N>
void launch_passes(float2* S, const float* mult, const float2* tw, int J, int H, int W, uint64_t seed,
                   uint32_t frame, float* fields, cudaStream_t st, int variant) {
  using GR = Groups<N>;
  constexpr int G = GR::G, HALF = N / 2 + 1;
  const size_t sm = GR::smem;
  if (variant < 0) variant = N == 1024 ? 1 : 0;
  if (N > 2048) variant = 0;
  if (sm > 48 * 1024) {
    if constexpr (N <= 2048) cudaFuncSetAttribute(k_colgen3<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GR::smem_fft);
    cudaFuncSetAttribute(k_colgen<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GR::smem_fft);
    cudaFuncSetAttribute(k_rowifft<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  }
  const float cN = (float)(N * 0.70710678118654752440);  // the noise scale N / sqrt 2
  const dim3 grid((HALF + G - 1) / G, J);
  bool done = false;
  if constexpr (N <= 2048) {
    if (variant == 1) {
      k_colgen3<N><<<grid, GR::THREADS, GR::smem_fft, st>>>(S, mult, tw, H, seed, frame, cN);
      done = true;
    }
  }
  if (!done) k_colgen<N><<<grid, GR::THREADS, GR::smem_fft, st>>>(S, mult, tw, H, seed, frame, cN);
  k_rowifft<N><<<dim3((H + 2 * G - 1) / (2 * G), J), GR::THREADS, sm, st>>>(S, fields, tw, H, W);
}

int dfp2s_launch_sample_fields(float2* S, const float* mult, const float2* tw, int N, int J, int H, int W,
                               uint64_t seed, uint32_t frame, const float* L, float scale, float* fields,
                               cudaStream_t st, const float* prev, float alpha, bool mix, int variant,
                               const dfp2s_factor_dev* sh) {
  switch (N) {
    case 16: launch_passes<16>(S, mult, tw, J, H, W, seed, frame, fields, st, variant); break;
    case 32: launch_passes<32>(S, mult, tw, J, H, W, seed, frame, fields, st, variant); break;
    case 64: launch_passes<64>(S, mult, tw, J, H, W, seed, frame, fields, st, variant); break;
    case 128: launch_passes<128>(S, mult, tw, J, H, W, seed, frame, fields, st, variant); break;
    case 256: launch_passes<256>(S, mult, tw, J, H, W, seed, frame, fields, st, variant); break;
    case 512: launch_passes<512>(S, mult, tw, J, H, W, seed, frame, fields, st, variant); break;
    case 1024: launch_passes<1024>(S, mult, tw, J, H, W, seed, frame, fields, st, variant); break;
    case 2048: launch_passes<2048>(S, mult, tw, J, H, W, seed, frame, fields, st, variant); break;
    case 4096: launch_passes<4096>(S, mult, tw, J, H, W, seed, frame, fields, st, variant); break;
    default: return DFP2S_EINVAL;
  }
  const size_t npix = (size_t)H * W;
  if (sh && sh->sh_levels > 0) {
    const int L = sh->sh_levels;
    k_sh_coeffs<<<(J * L * 4 + 255) / 256, 256, 0, st>>>(sh->sh_amp, J, L, seed, frame, sh->sh_coef);
    k_sh_add<<<H, 256, (size_t)J * L * sizeof(float4), st>>>(fields, J, H, W, N, L, sh->sh_coef);
  }
  if (!mix) return dfp2s_launch_status();
  if (prev) launch_mix_any<true>(fields, L, scale * sqrtf(1.f - alpha * alpha), J, npix, prev, alpha, st);
  else launch_mix_any<false>(fields, L, scale, J, npix, nullptr, 0.f, st);
  return dfp2s_launch_status();
}

int dfp2s_launch_philox_words(uint64_t seed, uint64_t sub, uint64_t q0, int nq, uint32_t* out, cudaStream_t st) {
  k_philox_words<<<(nq + 255) / 256, 256, 0, st>>>(seed, sub, q0, nq, out);
  return dfp2s_launch_status();
}

int dfp2s_launch_gaussian(uint64_t seed, uint64_t sub, size_t nq, float* out, cudaStream_t st) {
  k_gaussian<<<(unsigned)((nq + 255) / 256), 256, 0, st>>>(seed, sub, nq, out);
  return dfp2s_launch_status();
}

template <int N>
static void launch_rowifft(const float2* S, float* out, const float2* tw, int J, int H, int W, cudaStream_t st) {
  using GR = Groups<N>;
  constexpr int G = GR::G;
  if (GR::smem > 48 * 1024) cudaFuncSetAttribute(k_rowifft<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GR::smem);
  k_rowifft<N><<<dim3((H + 2 * G - 1) / (2 * G), J), GR::THREADS, GR::smem, st>>>(S, out, tw, H, W);
}

int dfp2s_launch_rowifft(const float2* S, float* out, const float2* tw, int N, int J, int H, int W, cudaStream_t st) {
  switch (N) {
    case 16: launch_rowifft<16>(S, out, tw, J, H, W, st); break;
    case 32: launch_rowifft<32>(S, out, tw, J, H, W, st); break;
    case 64: launch_rowifft<64>(S, out, tw, J, H, W, st); break;
    case 128: launch_rowifft<128>(S, out, tw, J, H, W, st); break;
    case 256: launch_rowifft<256>(S, out, tw, J, H, W, st); break;
    case 512: launch_rowifft<512>(S, out, tw, J, H, W, st); break;
    case 1024: launch_rowifft<1024>(S, out, tw, J, H, W, st); break;
    case 2048: launch_rowifft<2048>(S, out, tw, J, H, W, st); break;
    case 4096: launch_rowifft<4096>(S, out, tw, J, H, W, st); break;
    default: return DFP2S_EINVAL;
  }
  return dfp2s_launch_status();
}
