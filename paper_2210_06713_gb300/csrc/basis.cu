// PSF basis of the phase-to-space transform (Sec. II-C, Eq. p2s PSF): the paper
// takes the basis from a principal component analysis of a PSF database; here
// (reading R15) it is the top-K right singular vectors of the uncentred
// n_psf x 1089 matrix H of exact PSFs, in FP64 on the device:
//
//   1. Zernike vectors a ~ N(0, A_0(D/r0)) (Philox tag 1, D/r0 pooled evenly,
//      tilts zeroed) -> exact PSFs with the P2S kernel (PSF output mode);
//   2. one-sided Jacobi (Hestenes) on the columns of H: every round of the
//      round-robin tournament rotates 545 disjoint column pairs in parallel so
//      that they become orthogonal, accumulating the same rotations in V; sweeps
//      repeat until every pair of columns with norm^2 > 1e-12 |H|_F^2 has
//      |h_p . h_q| < 1e-12 |h_p| |h_q|.  Then H V = U S and the columns
//      of V are the right singular vectors with singular values |H v_j|;
//   3. the K columns with the largest norms, each signed so that its entry of
//      largest magnitude is positive (first such entry on ties).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int KS2 = 33 * 33;
constexpr int NCOL = KS2 + 1;  // even number of players for the tournament (one dummy)

__global__ void k_to_f64_colmajor(const float* __restrict__ Hf, int m, double* __restrict__ Hd) {
  // Hf: m x KS2 row-major -> Hd: column-major (column j contiguous, length m)
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)m * KS2) return;
  const int r = (int)(i / KS2), c = (int)(i - (size_t)r * KS2);
  Hd[(size_t)c * m + r] = Hf[i];
}

__global__ void k_eye(double* __restrict__ V) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)KS2 * KS2) return;
  const int c = (int)(i / KS2), r = (int)(i - (size_t)c * KS2);
  V[i] = (r == c) ? 1.0 : 0.0;
}

DFP2S_DEV double block_sum(double v, double* red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
  __syncthreads();
  if (threadIdx.x == 0) red[0] = t;
  __syncthreads();
  const double r = red[0];
  __syncthreads();
  return r;
}

// one round of the tournament: pair i = (player at position i, player at position NCOL-1-i),
// position 0 fixed to player 0, positions 1.. hold players rotated by `round`
__global__ void __launch_bounds__(256) k_jacobi_round(double* __restrict__ Hd, int m, double* __restrict__ V,
                                                      int round, double floor2,
                                                      unsigned long long* __restrict__ offmax) {
  __shared__ double red[8];
  __shared__ double cs[2];
  const int i = blockIdx.x;
  auto player = [&](int pos) { return pos == 0 ? 0 : ((pos - 1 + round) % (NCOL - 1)) + 1; };
  int p = player(i), q = player(NCOL - 1 - i);
  if (p > q) {
    const int t = p;
    p = q;
    q = t;
  }
  if (q >= KS2) return;  // the dummy player
  double* hp = Hd + (size_t)p * m;
  double* hq = Hd + (size_t)q * m;
  double a = 0.0, b = 0.0, g = 0.0;
  for (int r = threadIdx.x; r < m; r += blockDim.x) {
    const double x = hp[r], y = hq[r];
    a += x * x;
    b += y * y;
    g += x * y;
  }
  a = block_sum(a, red);
  b = block_sum(b, red);
  g = block_sum(g, red);
  if (threadIdx.x == 0) {
    double c = 1.0, s = 0.0;
    const double ab = sqrt(a * b);
    if (ab > 1e-30 && fabs(g) > 1e-15 * ab) {
      const double zeta = (b - a) / (2.0 * g);
      const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
      c = 1.0 / sqrt(1.0 + t * t);
      s = c * t;
      // convergence is judged on columns whose norm^2 exceeds 1e-12 |H|_F^2 (the
      // rest only carries rounding noise and does not reach the top-K basis)
      if (a > floor2 && b > floor2) {
        const double r = fabs(g) / ab;
        atomicMax(offmax, (unsigned long long)__double_as_longlong(r));
      }
    }
    cs[0] = c;
    cs[1] = s;
  }
  __syncthreads();
  const double c = cs[0], s = cs[1];
  if (s == 0.0) return;
  for (int r = threadIdx.x; r < m; r += blockDim.x) {
    const double x = hp[r], y = hq[r];
    hp[r] = c * x - s * y;
    hq[r] = s * x + c * y;
  }
  double* vp = V + (size_t)p * KS2;
  double* vq = V + (size_t)q * KS2;
  for (int r = threadIdx.x; r < KS2; r += blockDim.x) {
    const double x = vp[r], y = vq[r];
    vp[r] = c * x - s * y;
    vq[r] = s * x + c * y;
  }
}

__global__ void k_col_norms(const double* __restrict__ Hd, int m, double* __restrict__ sig) {
  __shared__ double red[8];
  const int c = blockIdx.x;
  double a = 0.0;
  for (int r = threadIdx.x; r < m; r += blockDim.x) a += Hd[(size_t)c * m + r] * Hd[(size_t)c * m + r];
  a = block_sum(a, red);
  if (threadIdx.x == 0) sig[c] = sqrt(a);
}

// descending order of the 1089 singular values (bitonic sort of 2048 slots), one CTA
__global__ void __launch_bounds__(1024) k_sort_desc(const double* __restrict__ sig, int* __restrict__ order,
                                                    double* __restrict__ sorted) {
  __shared__ double v[2048];
  __shared__ int ix[2048];
  for (int i = threadIdx.x; i < 2048; i += 1024) {
    v[i] = i < KS2 ? sig[i] : -1.0;
    ix[i] = i;
  }
  __syncthreads();
  for (int k = 2; k <= 2048; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < 2048; i += 1024) {
        const int l = i ^ j;
        if (l > i) {
          // descending overall: within blocks with (i & k) == 0 sort descending
          const bool desc = (i & k) == 0;
          const bool before = (v[i] > v[l]) || (v[i] == v[l] && ix[i] < ix[l]);  // true: i belongs first
          if (desc ? !before : before) {
            const double tv = v[i];
            v[i] = v[l];
            v[l] = tv;
            const int ti = ix[i];
            ix[i] = ix[l];
            ix[l] = ti;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < KS2; i += 1024) {
    order[i] = ix[i];
    sorted[i] = v[i];
  }
}

// basis row k = column order[k] of V, signed so that its largest-magnitude entry is positive
__global__ void k_gather_basis(const double* __restrict__ V, const int* __restrict__ order, int K,
                               float* __restrict__ basis) {
  __shared__ double best[256];
  __shared__ int besti[256];
  const int k = blockIdx.x;
  const double* v = V + (size_t)order[k] * KS2;
  double bv = -1.0;
  int bi = KS2;
  for (int r = threadIdx.x; r < KS2; r += blockDim.x) {
    const double a = fabs(v[r]);
    if (a > bv || (a == bv && r < bi)) {
      bv = a;
      bi = r;
    }
  }
  best[threadIdx.x] = bv;
  besti[threadIdx.x] = bi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const double a = best[threadIdx.x + o];
      const int ai = besti[threadIdx.x + o];
      if (a > best[threadIdx.x] || (a == best[threadIdx.x] && ai < besti[threadIdx.x])) {
        best[threadIdx.x] = a;
        besti[threadIdx.x] = ai;
      }
    }
    __syncthreads();
  }
  const double sgn = v[besti[0]] < 0 ? -1.0 : 1.0;
  for (int r = threadIdx.x; r < KS2; r += blockDim.x) basis[(size_t)k * KS2 + r] = (float)(sgn * v[r]);
}

}  // namespace

int dfp2s_basis_build_device(int J, const float* L32, int K, int n_psf, const double* dr_host, int n_dr, uint64_t seed,
                             float* basis_out, double* sigma_host, int* sweeps_out, cudaStream_t st) {
  struct Bufs {
    float *a = nullptr, *h = nullptr, *drs = nullptr, *dummy_basis = nullptr;
    double *Hd = nullptr, *V = nullptr, *sig = nullptr, *sorted = nullptr;
    int* order = nullptr;
    unsigned long long* rotated = nullptr;
    dfp2s_p2s_dev t{};
    ~Bufs() {
      void* all[] = {a, h, drs, dummy_basis, Hd, V, sig, sorted, order, rotated, t.phiT, t.zt, t.mask, t.dft};
      for (void* p : all)
        if (p) cudaFree(p);
    }
  } b;
  const int m = n_psf;
  if (dfp2s_device_malloc((void**)&b.a, (size_t)J * m * sizeof(float)) != cudaSuccess ||
      dfp2s_device_malloc((void**)&b.h, (size_t)m * KS2 * sizeof(float)) != cudaSuccess ||
      dfp2s_device_malloc((void**)&b.drs, 8 * sizeof(float)) != cudaSuccess ||
      dfp2s_device_malloc((void**)&b.dummy_basis, KS2 * sizeof(float)) != cudaSuccess ||
      dfp2s_device_malloc((void**)&b.Hd, (size_t)m * KS2 * sizeof(double)) != cudaSuccess ||
      dfp2s_device_malloc((void**)&b.V, (size_t)KS2 * KS2 * sizeof(double)) != cudaSuccess ||
      dfp2s_device_malloc((void**)&b.sig, KS2 * sizeof(double)) != cudaSuccess ||
      dfp2s_device_malloc((void**)&b.sorted, KS2 * sizeof(double)) != cudaSuccess ||
      dfp2s_device_malloc((void**)&b.order, KS2 * sizeof(int)) != cudaSuccess ||
      dfp2s_device_malloc((void**)&b.rotated, sizeof(unsigned long long)) != cudaSuccess ||
      dfp2s_device_malloc((void**)&b.t.phiT, KS2 * sizeof(float)) != cudaSuccess ||
      dfp2s_device_malloc((void**)&b.t.zt, (size_t)(J - 2) * KS2 * sizeof(float)) != cudaSuccess ||
      dfp2s_device_malloc((void**)&b.t.mask, KS2 * sizeof(float)) != cudaSuccess ||
      dfp2s_device_malloc((void**)&b.t.dft, KS2 * sizeof(float2)) != cudaSuccess)
    return DFP2S_ENOMEM;
  float hdr[8];
  for (int i = 0; i < n_dr; ++i) hdr[i] = (float)dr_host[i];
  cudaMemcpyAsync(b.drs, hdr, n_dr * sizeof(float), cudaMemcpyHostToDevice, st);
  cudaMemsetAsync(b.dummy_basis, 0, KS2 * sizeof(float), st);
  b.t.J = J;
  b.t.K = 1;
  b.t.basis = b.dummy_basis;
  int rc;
  if ((rc = dfp2s_p2s_build_tables(&b.t, st))) return rc;
  if ((rc = dfp2s_launch_draw_vectors(m, J, L32, b.drs, n_dr, seed, 1u, b.a, st))) return rc;
  if ((rc = dfp2s_launch_p2s_exact(&b.t, b.a, 1, m, b.h, DFP2S_W_PSF, st))) return rc;
  k_to_f64_colmajor<<<(unsigned)(((size_t)m * KS2 + 255) / 256), 256, 0, st>>>(b.h, m, b.Hd);
  k_eye<<<(unsigned)(((size_t)KS2 * KS2 + 255) / 256), 256, 0, st>>>(b.V);
  if (dfp2s_launch_status() != DFP2S_OK) return DFP2S_ECUDA;
  // rounding floor for the convergence test: 1e-12 of the squared Frobenius norm
  double floor2 = 0.0;
  {
    std::vector<double> hs(KS2);
    k_col_norms<<<KS2, 256, 0, st>>>(b.Hd, m, b.sig);
    if (cudaMemcpyAsync(hs.data(), b.sig, KS2 * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return DFP2S_ECUDA;
    for (double v : hs) floor2 += v * v;
    floor2 *= 1e-12;
  }
  // sweeps of the tournament, each captured once as a graph
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cs;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return DFP2S_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    cudaStreamDestroy(cs);
    return DFP2S_ECUDA;
  }
  cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  cudaMemsetAsync(b.rotated, 0, sizeof(unsigned long long), cs);
  for (int r = 0; r < NCOL - 1; ++r) k_jacobi_round<<<NCOL / 2, 256, 0, cs>>>(b.Hd, m, b.V, r, floor2, b.rotated);
  cudaError_t ce = cudaStreamEndCapture(cs, &graph);
  if (ce == cudaSuccess) ce = cudaGraphInstantiate(&exec, graph, 0);
  int sweep = 0;
  for (; ce == cudaSuccess && sweep < 40; ++sweep) {
    unsigned long long bits = 0;
    if ((ce = cudaGraphLaunch(exec, cs)) != cudaSuccess) break;
    if ((ce = cudaMemcpyAsync(&bits, b.rotated, sizeof(bits), cudaMemcpyDeviceToHost, cs)) != cudaSuccess) break;
    if ((ce = cudaStreamSynchronize(cs)) != cudaSuccess) break;
    double off;
    memcpy(&off, &bits, sizeof(off));
    if (off < 1e-12) {
      ++sweep;
      break;
    }
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cs);
  if (ce != cudaSuccess) return DFP2S_ECUDA;
  if (sweeps_out) *sweeps_out = sweep;
  k_col_norms<<<KS2, 256, 0, st>>>(b.Hd, m, b.sig);
  k_sort_desc<<<1, 1024, 0, st>>>(b.sig, b.order, b.sorted);
  k_gather_basis<<<K, 256, 0, st>>>(b.V, b.order, K, basis_out);
  if (sigma_host) cudaMemcpyAsync(sigma_host, b.sorted, KS2 * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (dfp2s_launch_status() != DFP2S_OK) return DFP2S_ECUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? DFP2S_OK : DFP2S_ECUDA;
}
