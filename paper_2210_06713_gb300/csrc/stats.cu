// Lagged covariances of Zernike coefficient fields: the statistic against which
// the sampler is judged (Sec. III-D: the covariance of the sampled fields at
// separation s is Eq. (A tilde)'s A~(s), and A_0 at s = 0).
//
//   C_l[i][j] = (1 / n_l) sum over pixels x with x + d_l in the frame of a_i(x) a_j(x + d_l)
//
// One block row per lag: each block takes runs of 32 valid pixels (a grid-stride
// walk over them), stages a(x) and a(x + d) for the run in shared memory, and
// each thread accumulates a 4 x 4 register tile of (i, j) pairs (i = ti + 16 m,
// j = tj + 16 n for thread (ti, tj) of a 16 x 16 arrangement): products and the
// run's sum in FP32, the runs in FP32 with Kahan compensation (FP64 arithmetic
// is a small fraction of the FP32 rate on this part).  A second kernel sums the
// blocks' partials in FP64 in a fixed order.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int RUN = 32;
constexpr int THREADS = 256;
constexpr int T4 = DFP2S_MAX_J / 16;  // register tile side (4)

__global__ void __launch_bounds__(THREADS, 1) k_cov_partial(const float* __restrict__ a, int J, int H, int W,
                                                         const int2* __restrict__ lags, int nb,
                                                         double* __restrict__ part) {
  // [pixel][field], rows padded to an odd stride: the staging writes walk the pixels, the sums walk the fields
  __shared__ float xs[RUN][DFP2S_MAX_J + 1], ys[RUN][DFP2S_MAX_J + 1];
  const int l = blockIdx.y;
  const int2 d = lags[l];  // (dy, dx)
  const int y0 = max(0, -d.x), y1 = min(H, H - d.x), x0 = max(0, -d.y), x1 = min(W, W - d.y);
  const int ny = y1 - y0, nx = x1 - x0;
  const long long n = (long long)ny * nx;
  const long long runs = (n + RUN - 1) / RUN;
  const size_t plane = (size_t)H * W;
  const int npairs = J * J;
  const int ti = threadIdx.x >> 4, tj = threadIdx.x & 15;
  float acc[T4][T4], cmp[T4][T4];  // compensated sums over the runs
#pragma unroll
  for (int m = 0; m < T4; ++m)
#pragma unroll
    for (int k = 0; k < T4; ++k) acc[m][k] = cmp[m][k] = 0.f;
  // staging role of this thread: pixel q of a run for fields jg, jg + 8, ... (up to 8 of them); the next run's
  // values are loaded into registers while the current one is summed
  const int q = threadIdx.x & (RUN - 1), jg = threadIdx.x / RUN;
  constexpr int NJ = DFP2S_MAX_J / (THREADS / RUN);
  float nx_[NJ], ny_[NJ];
  auto load_run = [&](long long r) {
    const long long p = r * RUN + q;
    const bool in = r < runs && p < n;
    const int pi = in ? (int)p : 0;  // n < 2^31
    const int yy = pi / nx, xx = pi - yy * nx;
    const size_t o1 = (size_t)(y0 + yy) * W + (x0 + xx);
    const size_t o2 = (size_t)(y0 + yy + d.x) * W + (x0 + xx + d.y);
#pragma unroll
    for (int e = 0; e < NJ; ++e) {
      const int j = jg + e * (THREADS / RUN);
      nx_[e] = (in && j < J) ? a[j * plane + o1] : 0.f;
      ny_[e] = (in && j < J) ? a[j * plane + o2] : 0.f;
    }
  };
  load_run(blockIdx.x);
  for (long long r = blockIdx.x; r < runs; r += nb) {
    __syncthreads();  // the previous run's reads are done
#pragma unroll
    for (int e = 0; e < NJ; ++e) {
      xs[q][jg + e * (THREADS / RUN)] = nx_[e];
      ys[q][jg + e * (THREADS / RUN)] = ny_[e];
    }
    __syncthreads();
    load_run(r + nb);
    float sm[T4][T4];
#pragma unroll
    for (int m = 0; m < T4; ++m)
#pragma unroll
      for (int k = 0; k < T4; ++k) sm[m][k] = 0.f;
    const int nm = (J - ti + 15) / 16, nk = (J - tj + 15) / 16;  // tile rows / columns inside J
#pragma unroll 4
    for (int qq = 0; qq < RUN; ++qq) {
      float xv[T4], yv[T4];
#pragma unroll
      for (int m = 0; m < T4; ++m) xv[m] = m < nm ? xs[qq][ti + 16 * m] : 0.f;
#pragma unroll
      for (int k = 0; k < T4; ++k) yv[k] = k < nk ? ys[qq][tj + 16 * k] : 0.f;
#pragma unroll
      for (int m = 0; m < T4; ++m)
#pragma unroll
        for (int k = 0; k < T4; ++k) sm[m][k] = fmaf(xv[m], yv[k], sm[m][k]);
    }
#pragma unroll
    for (int m = 0; m < T4; ++m)
#pragma unroll
      for (int k = 0; k < T4; ++k) {
        const float y = __fsub_rn(sm[m][k], cmp[m][k]);
        const float t = __fadd_rn(acc[m][k], y);
        cmp[m][k] = __fsub_rn(__fsub_rn(t, acc[m][k]), y);
        acc[m][k] = t;
      }
  }
#pragma unroll
  for (int m = 0; m < T4; ++m)
#pragma unroll
    for (int k = 0; k < T4; ++k) {
      const int i = ti + 16 * m, j = tj + 16 * k;
      if (i < J && j < J)
        part[((size_t)l * nb + blockIdx.x) * npairs + i * J + j] = (double)acc[m][k] - (double)cmp[m][k];
    }
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
  const int nb = (int)(runs < 2LL * sms ? runs : 2LL * sms);
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
  k_cov_partial<<<dim3(nb, n_lags), THREADS, 0, st>>>(a, J, H, W, dl, nb, part);
  k_cov_reduce<<<dim3((npairs + 255) / 256, n_lags), 256, 0, st>>>(part, nb, npairs, dl, H, W, out);
  const bool ok = dfp2s_launch_status() == DFP2S_OK;
  cudaFreeAsync(dl, st);
  cudaFreeAsync(part, st);
  return ok ? DFP2S_OK : DFP2S_ECUDA;
}
