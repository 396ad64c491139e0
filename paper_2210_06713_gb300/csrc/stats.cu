// Lagged covariances of Zernike coefficient fields: the statistic against which
// the sampler is judged (Sec. III-D: the covariance of the sampled fields at
// separation s is Eq. (A tilde)'s A~(s), and A_0 at s = 0).
//
//   C_l[i][j] = (1 / n_l) sum over pixels x with x + d_l in the frame of a_i(x) a_j(x + d_l)
//
// Per lag a J x J x n_l contraction.  A CTA takes runs of RUN valid pixels (a
// grid-stride walk over them) and stages a(x) and a(x + d) for the run in shared
// memory ([pixel][field], the fields padded to NBI x TB with zeros); the next
// run's values are loaded into registers meanwhile.  The J x J pairs are cut
// into TB x TB register tiles, one per thread of a group of NBI^2 threads
// (NBI = ceil(J / TB)); the CTA holds floor(256 / NBI^2) groups, and group g
// sums pixels g, g + ng, ... of each run: per pixel 2 TB / 2 eight-byte shared
// loads and TB^2 FMAs.  The sums of FOLD_RUNS runs (plain FP32) enter FP32
// accumulators with Kahan compensation (FP64 arithmetic is a small fraction of
// the FP32 rate on this part); at the end the groups' sums are added in group
// order in shared memory (compensated FP32), and a second kernel sums the CTAs'
// partials in FP64 in a fixed order.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int RUN = 64;
constexpr int THREADS = 256;
constexpr int TB = 6;                                 // register tile side
constexpr int NBI_MAX = (DFP2S_MAX_J + TB - 1) / TB;  // 11
constexpr int JPAD = NBI_MAX * TB;                    // 66 fields per staged pixel (even: 8-byte loads)
constexpr int SPLIT = THREADS / RUN;                  // staging: field groups of a pixel
constexpr int NJ = (DFP2S_MAX_J + SPLIT - 1) / SPLIT; // fields per staging thread
constexpr int FOLD_RUNS = 4;                          // runs summed in plain FP32 before a compensated fold

struct CovSmem {
  float xs[RUN][JPAD], ys[RUN][JPAD];
  float red_s[DFP2S_MAX_J * DFP2S_MAX_J], red_c[DFP2S_MAX_J * DFP2S_MAX_J];  // the groups' sum, compensation
};

__global__ void __launch_bounds__(THREADS, 1) k_cov_partial(const float* __restrict__ a, int J, int H, int W,
                                                         const int2* __restrict__ lags, int nb,
                                                         double* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char cov_raw[];
  CovSmem& s = *reinterpret_cast<CovSmem*>(cov_raw);
  const int l = blockIdx.y;
  const int2 d = lags[l];  // (dy, dx)
  const int y0 = max(0, -d.x), y1 = min(H, H - d.x), x0 = max(0, -d.y), x1 = min(W, W - d.y);
  const int ny = y1 - y0, nx = x1 - x0;
  const long long n = (long long)ny * nx;
  const long long runs = (n + RUN - 1) / RUN;
  const size_t plane = (size_t)H * W;
  const int npairs = J * J;
  const int nbi = (J + TB - 1) / TB, G = nbi * nbi, ng = THREADS / G;
  const int grp = threadIdx.x / G, w = threadIdx.x - grp * G;
  const bool active = grp < ng;
  const int i0 = (w / nbi) * TB, j0 = (w - (w / nbi) * nbi) * TB;
  for (int e = threadIdx.x; e < RUN * JPAD; e += THREADS) {  // the padding fields stay zero
    (&s.xs[0][0])[e] = 0.f;
    (&s.ys[0][0])[e] = 0.f;
  }
  for (int e = threadIdx.x; e < npairs; e += THREADS) s.red_s[e] = s.red_c[e] = 0.f;
  float acc[TB][TB], cmp[TB][TB];  // compensated sums over the runs
#pragma unroll
  for (int m = 0; m < TB; ++m)
#pragma unroll
    for (int k = 0; k < TB; ++k) acc[m][k] = cmp[m][k] = 0.f;
  // staging role: pixel q of a run for fields jg, jg + SPLIT, ...
  const int q = threadIdx.x % RUN, jg = threadIdx.x / RUN;
  float nx_[NJ], ny_[NJ];
  auto load_run = [&](long long r) {
    const long long p = r * RUN + q;
    const bool in = r < runs && p < n;
    const int pi = in ? (int)p : 0;  // n < 2^31
    const int yy = pi / nx, xx = pi - yy * nx;
    const float* p1 = a + jg * plane + (size_t)(y0 + yy) * W + (x0 + xx);
    const float* p2 = a + jg * plane + (size_t)(y0 + yy + d.x) * W + (x0 + xx + d.y);
#pragma unroll
    for (int e = 0; e < NJ; ++e) {
      const bool ld = in && jg + e * SPLIT < J;
      nx_[e] = ld ? __ldg(p1) : 0.f;
      ny_[e] = ld ? __ldg(p2) : 0.f;
      p1 += SPLIT * plane;
      p2 += SPLIT * plane;
    }
  };
  float sm[TB][TB];  // the group's plain FP32 sums since the last fold
#pragma unroll
  for (int m = 0; m < TB; ++m)
#pragma unroll
    for (int k = 0; k < TB; ++k) sm[m][k] = 0.f;
  auto fold = [&]() {
#pragma unroll
    for (int m = 0; m < TB; ++m)
#pragma unroll
      for (int k = 0; k < TB; ++k) {
        const float y = __fsub_rn(sm[m][k], cmp[m][k]);
        const float t = __fadd_rn(acc[m][k], y);
        cmp[m][k] = __fsub_rn(__fsub_rn(t, acc[m][k]), y);
        acc[m][k] = t;
        sm[m][k] = 0.f;
      }
  };
  int since = 0;
  load_run(blockIdx.x);
  for (long long r = blockIdx.x; r < runs; r += nb) {
    __syncthreads();  // the previous run's reads are done (and, the first time, the zero fill)
#pragma unroll
    for (int e = 0; e < NJ; ++e) {
      const int j = jg + e * SPLIT;
      if (j < J) {
        s.xs[q][j] = nx_[e];
        s.ys[q][j] = ny_[e];
      }
    }
    __syncthreads();
    load_run(r + nb);
    if (active) {
      for (int qq = grp; qq < RUN; qq += ng) {
        float xv[TB], yv[TB];
#pragma unroll
        for (int m = 0; m < TB; m += 2) {
          const float2 x2 = *reinterpret_cast<const float2*>(&s.xs[qq][i0 + m]);
          const float2 y2 = *reinterpret_cast<const float2*>(&s.ys[qq][j0 + m]);
          xv[m] = x2.x;
          xv[m + 1] = x2.y;
          yv[m] = y2.x;
          yv[m + 1] = y2.y;
        }
#pragma unroll
        for (int m = 0; m < TB; ++m)
#pragma unroll
          for (int k = 0; k < TB; ++k) sm[m][k] = fmaf(xv[m], yv[k], sm[m][k]);
      }
      if (++since == FOLD_RUNS) {
        fold();
        since = 0;
      }
    }
  }
  if (active) fold();
  // the groups' compensated sums, in group order, by compensated FP32 additions in shared memory (FP64 once per
  // pair at the end: FP64 arithmetic runs at a small fraction of the FP32 rate here)
  auto kahan = [](float& sum, float& c, float v) {
    const float y = __fsub_rn(v, c);
    const float t = __fadd_rn(sum, y);
    c = __fsub_rn(__fsub_rn(t, sum), y);
    sum = t;
  };
  for (int g = 0; g < ng; ++g) {
    __syncthreads();
    if (grp == g) {
#pragma unroll
      for (int m = 0; m < TB; ++m)
#pragma unroll
        for (int k = 0; k < TB; ++k) {
          const int i = i0 + m, j = j0 + k;
          if (i < J && j < J) {
            kahan(s.red_s[i * J + j], s.red_c[i * J + j], acc[m][k]);
            kahan(s.red_s[i * J + j], s.red_c[i * J + j], -cmp[m][k]);
          }
        }
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < npairs; e += THREADS)
    part[((size_t)l * nb + blockIdx.x) * npairs + e] = (double)s.red_s[e] - (double)s.red_c[e];
}

__global__ void k_cov_reduce(const double* __restrict__ part, int nb, int npairs, const int2* __restrict__ lags,
                             int H, int W, double* __restrict__ out) {
  const int l = blockIdx.y;
  const int pr = blockIdx.x * blockDim.x + threadIdx.x;
  if (pr >= npairs) return;
  const int2 d = lags[l];
  const double n = (double)(H - abs(d.x)) * (double)(W - abs(d.y));
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += part[((size_t)l * nb + b) * npairs + pr];
  out[(size_t)l * npairs + pr] = s / n;
}

}  // namespace

int dfp2s_launch_field_covariance(const float* a, int J, int H, int W, const int* lags_host, int n_lags, double* out,
                                  cudaStream_t st) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long npix = (long long)H * W;
  const long long runs = (npix + RUN - 1) / RUN;
  const int nb = (int)(runs < sms ? runs : sms);  // one CTA per SM and lag
  const int npairs = J * J;
  int2* dl = nullptr;
  double* part = nullptr;
  if (dfp2s_device_malloc_async((void**)&dl, n_lags * sizeof(int2), st) != cudaSuccess ||
      dfp2s_device_malloc_async((void**)&part, (size_t)n_lags * nb * npairs * sizeof(double), st) != cudaSuccess) {
    if (dl) cudaFreeAsync(dl, st);
    return DFP2S_ENOMEM;
  }
  // lags_host holds (dy, dx) pairs; int2 (x, y) = (dy, dx)
  if (cudaMemcpyAsync(dl, lags_host, n_lags * sizeof(int2), cudaMemcpyHostToDevice, st) != cudaSuccess) {
    cudaFreeAsync(dl, st);
    cudaFreeAsync(part, st);
    return DFP2S_ECUDA;
  }
  cudaFuncSetAttribute(k_cov_partial, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(CovSmem));
  k_cov_partial<<<dim3(nb, n_lags), THREADS, sizeof(CovSmem), st>>>(a, J, H, W, dl, nb, part);
  k_cov_reduce<<<dim3((npairs + 255) / 256, n_lags), 256, 0, st>>>(part, nb, npairs, dl, H, W, out);
  const bool ok = dfp2s_launch_status() == DFP2S_OK;
  cudaFreeAsync(dl, st);
  cudaFreeAsync(part, st);
  return ok ? DFP2S_OK : DFP2S_ECUDA;
}
