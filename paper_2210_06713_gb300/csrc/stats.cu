// Lagged covariances of Zernike coefficient fields: the statistic against which
// the sampler is judged (Sec. III-D: the covariance of the sampled fields at
// separation s is Eq. (A tilde)'s A~(s), and A_0 at s = 0).
//
//   C_l[i][j] = (1 / n_l) sum over pixels x with x + d_l in the frame of a_i(x) a_j(x + d_l)
//
// One block row per lag: each block takes runs of 32 valid pixels (a grid-stride
// walk over them), stages a(x) and a(x + d) for the run in shared memory, and
// each thread accumulates its (i, j) pairs: products and the run's sum in FP32,
// the runs in FP64.  A second kernel sums the blocks' partials in a fixed order.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int RUN = 32;
constexpr int THREADS = 256;
constexpr int MAXPAIRS = DFP2S_MAX_J * DFP2S_MAX_J;
constexpr int PPT = MAXPAIRS / THREADS;  // pairs per thread at most (16)

__global__ void __launch_bounds__(THREADS) k_cov_partial(const float* __restrict__ a, int J, int H, int W,
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
  double acc[PPT];
#pragma unroll
  for (int k = 0; k < PPT; ++k) acc[k] = 0.0;
  for (long long r = blockIdx.x; r < runs; r += nb) {
    __syncthreads();  // the previous run's reads are done
    for (int e = threadIdx.x; e < J * RUN; e += THREADS) {
      const int j = e / RUN, q = e - j * RUN;
      const long long p = r * RUN + q;
      float u = 0.f, v = 0.f;
      if (p < n) {
        const int y = y0 + (int)(p / nx), x = x0 + (int)(p % nx);
        u = a[j * plane + (size_t)y * W + x];
        v = a[j * plane + (size_t)(y + d.x) * W + (x + d.y)];
      }
      xs[q][j] = u;
      ys[q][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      const int pr = threadIdx.x + k * THREADS;
      if (pr < npairs) {
        const int i = pr / J, j = pr - i * J;
        float s = 0.f;
#pragma unroll 8
        for (int q = 0; q < RUN; ++q) s = fmaf(xs[q][i], ys[q][j], s);
        acc[k] += (double)s;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    const int pr = threadIdx.x + k * THREADS;
    if (pr < npairs) part[((size_t)l * nb + blockIdx.x) * npairs + pr] = acc[k];
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
  if (cudaMallocAsync((void**)&dl, n_lags * sizeof(int2), st) != cudaSuccess ||
      cudaMallocAsync((void**)&part, (size_t)n_lags * nb * npairs * sizeof(double), st) != cudaSuccess) {
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
  const bool ok = cudaGetLastError() == cudaSuccess;
  cudaFreeAsync(dl, st);
  cudaFreeAsync(part, st);
  return ok ? DFP2S_OK : DFP2S_ECUDA;
}
