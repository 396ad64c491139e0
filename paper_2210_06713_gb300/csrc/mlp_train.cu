// Training of the P2S surrogate network on the device (Sec. II-C: the paper,
// after Mao et al. 2021, maps each pixel's Zernike vector to the PSF-basis
// coefficients with a small neural network; the shape and the training are this
// project's choice): J -> 256 -> 256 -> K with GELU (erf form), FP32 SIMT
// kernels for forward, backward and Adam, one training step captured in a CUDA
// graph and replayed.
//
// Data: n Zernike vectors a ~ N(0, A_0(D/r0)) (Philox tag 2, D/r0 cycling over a
// list, tilt fields zeroed), targets w = exact P2S weights from the same kernel
// that serves frames.  Inputs are scaled per field by 1/std, targets
// standardised per k.  The loss is either sum_b r_b^T G r_b / (B K), r = y - t,
// with G the expected blurred-image error per weight error under a
// 1 / (|f|^2 + 1) image spectrum (k_prior_*), or sum_k lw_k r_k^2 / (B K) with
// lw_k = 1 (plain MSE on standardised weights) or lw_k = var_k / mean(var) (MSE
// of the PSF, since the basis is orthonormal: G of a flat spectrum).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int HID = 256;
constexpr float kInvSqrt2 = 0.70710678118654752f;
constexpr float kInvSqrt2Pi = 0.39894228040143268f;

DFP2S_DEV float gelu(float z) { return 0.5f * z * (1.f + erff(z * kInvSqrt2)); }
DFP2S_DEV float gelu_grad(float z) {
  return 0.5f * (1.f + erff(z * kInvSqrt2)) + z * kInvSqrt2Pi * __expf(-0.5f * z * z);
}

// ------------------------------------------------------------------ GEMM
// C[M x N] = sum_k A(m, k) B(k, n) with A(m, k) = TA ? A[k lda + m] : A[m lda + k],
// B(k, n) = TB ? B[n ldb + k] : B[k ldb + n].  64 x 64 tiles, 256 threads, 4 x 4 per thread.
enum { EPI_NONE = 0, EPI_BIAS = 1, EPI_BIAS_GELU = 2, EPI_GELU_GRAD = 3 };

template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, const float* __restrict__ A, int lda,
                                              const float* __restrict__ B, int ldb, float* __restrict__ C, int ldc,
                                              const float* __restrict__ bias, float* __restrict__ Zout,
                                              const float* __restrict__ Zin) {
  __shared__ float As[16][64 + 4];
  __shared__ float Bs[16][64 + 4];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += 16) {
    for (int i = threadIdx.x; i < 16 * 64; i += 256) {
      const int kk = i / 64, mm = i % 64;
      const int m = m0 + mm, k = k0 + kk;
      float v = 0.f;
      if (m < M && k < K) v = TA ? A[(size_t)k * lda + m] : A[(size_t)m * lda + k];
      As[kk][mm] = v;
      const int n = n0 + mm;
      float u = 0.f;
      if (n < N && k < K) u = TB ? B[(size_t)n * ldb + k] : B[(size_t)k * ldb + n];
      Bs[kk][mm] = u;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = As[kk][ty * 4 + i];
        b[i] = Bs[kk][tx * 4 + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty * 4 + i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx * 4 + j;
      if (n >= N) continue;
      float v = acc[i][j];
      const size_t o = (size_t)m * ldc + n;
      if (EPI == EPI_BIAS) v += bias[n];
      if (EPI == EPI_BIAS_GELU) {
        v += bias[n];
        Zout[o] = v;
        v = gelu(v);
      }
      if (EPI == EPI_GELU_GRAD) v *= gelu_grad(Zin[o]);
      C[o] = v;
    }
  }
}

template <bool TA, bool TB, int EPI>
void gemm(cudaStream_t st, int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C, int ldc,
          const float* bias = nullptr, float* Zout = nullptr, const float* Zin = nullptr) {
  dim3 grid((N + 63) / 64, (M + 63) / 64);
  k_gemm<TA, TB, EPI><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, Zout, Zin);
}

// column sums: out[n] = sum_m X[m * N + n]
__global__ void k_colsum(const float* __restrict__ X, int M, int N, float* __restrict__ out) {
  const int n = blockIdx.x * 32 + (threadIdx.x & 31);
  const int part = threadIdx.x >> 5;  // 8 partial rows
  __shared__ float red[8][33];
  float s = 0.f;
  if (n < N)
    for (int m = part; m < M; m += 8) s += X[(size_t)m * N + n];
  red[part][threadIdx.x & 31] = s;
  __syncthreads();
  if (part == 0 && n < N) {
    float t = 0.f;
    for (int i = 0; i < 8; ++i) t += red[i][threadIdx.x & 31];
    out[n] = t;
  }
}

// dY = 2 lw (Y - T) / (B K); loss += sum lw (Y - T)^2 / (B K)
__global__ void k_loss_grad(const float* __restrict__ Y, const float* __restrict__ T, const float* __restrict__ lw,
                            int B, int K, float* __restrict__ dY, float* __restrict__ loss) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const float inv = 1.f / ((float)B * (float)K);
  float l = 0.f;
  if (i < (size_t)B * K) {
    const int k = (int)(i % K);
    const float r = Y[i] - T[i];
    dY[i] = 2.f * lw[k] * r * inv;
    l = lw[k] * r * r * inv;
  }
  for (int off = 16; off > 0; off >>= 1) l += __shfl_down_sync(0xffffffffu, l, off);
  if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, l);
}

// dY = R (the residual Y - T), overwritten below by the gradient
__global__ void k_residual(const float* __restrict__ Y, const float* __restrict__ T, size_t n, float* __restrict__ R) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) R[i] = Y[i] - T[i];
}

// with RG = R G (G symmetric): loss += sum RG * R / (B K); dY = 2 RG / (B K), in place over R
__global__ void k_gram_loss_grad(const float* __restrict__ RG, float* __restrict__ RdY, int B, int K,
                                 float* __restrict__ loss) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const float inv = 1.f / ((float)B * (float)K);
  float l = 0.f;
  if (i < (size_t)B * K) {
    const float r = RdY[i], rg = RG[i];
    l = rg * r * inv;
    RdY[i] = 2.f * rg * inv;
  }
  for (int off = 16; off > 0; off >>= 1) l += __shfl_down_sync(0xffffffffu, l, off);
  if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, l);
}

// ------------------------------------------------------- image-prior loss form
// G_kl = sum_f S(f) Re(Phi_k(f) conj Phi_l(f)), Phi_k the DFT of the 33 x 33 basis
// function k at the origin of a 64 x 64 torus, S(f) = 1 / (fx^2 + fy^2 + 1) with
// integer frequencies in [-32, 32): the expected energy that a weight error puts
// into the blurred image (Eq. varying blur) for images with that spectrum.
// FP64 throughout; the twiddles exp(-2 pi i m / 64) come from sincospi of exact
// multiples of 1/32.
constexpr int PM = 64;
constexpr int PS = 33;

__device__ void prior_twiddles(double2* tw) {
  for (int m = threadIdx.x; m < PM; m += blockDim.x) {
    double sn, cs;
    sincospi(-(double)m / (PM / 2), &sn, &cs);
    tw[m] = make_double2(cs, sn);
  }
  __syncthreads();
}

// rows: T[k][u][fx] = sum_v phi_k(u, v) e^{-2 pi i fx v / 64}
__global__ void k_prior_dft_rows(const float* __restrict__ basis, double2* __restrict__ Tm) {
  __shared__ double2 tw[PM];
  prior_twiddles(tw);
  const int k = blockIdx.x;
  for (int i = threadIdx.x; i < PS * PM; i += blockDim.x) {
    const int u = i / PM, fx = i - u * PM;
    double re = 0.0, im = 0.0;
    for (int v = 0; v < PS; ++v) {
      const double b = basis[((size_t)k * PS + u) * PS + v];
      const double2 w = tw[(fx * v) & (PM - 1)];
      re += b * w.x;
      im += b * w.y;
    }
    Tm[((size_t)k * PS + u) * PM + fx] = make_double2(re, im);
  }
}

// columns: Phi[k][fy][fx] = sum_u T[k][u][fx] e^{-2 pi i fy u / 64}
__global__ void k_prior_dft_cols(const double2* __restrict__ Tm, double2* __restrict__ Phi) {
  __shared__ double2 tw[PM];
  prior_twiddles(tw);
  const int k = blockIdx.x;
  for (int i = threadIdx.x; i < PM * PM; i += blockDim.x) {
    const int fy = i / PM, fx = i - fy * PM;
    double re = 0.0, im = 0.0;
    for (int u = 0; u < PS; ++u) {
      const double2 t = Tm[((size_t)k * PS + u) * PM + fx];
      const double2 w = tw[(fy * u) & (PM - 1)];
      re += t.x * w.x - t.y * w.y;
      im += t.x * w.y + t.y * w.x;
    }
    Phi[(size_t)k * PM * PM + i] = make_double2(re, im);
  }
}

__global__ void k_prior_gram(const double2* __restrict__ Phi, int K, double* __restrict__ G) {
  const int k = blockIdx.x, l = blockIdx.y;
  double acc = 0.0;
  for (int i = threadIdx.x; i < PM * PM; i += blockDim.x) {
    int fy = i / PM, fx = i - fy * PM;
    if (fy >= PM / 2) fy -= PM;
    if (fx >= PM / 2) fx -= PM;
    const double S = 1.0 / ((double)(fx * fx + fy * fy) + 1.0);
    const double2 a = Phi[(size_t)k * PM * PM + i], b = Phi[(size_t)l * PM * PM + i];
    acc += S * (a.x * b.x + a.y * b.y);
  }
  __shared__ double red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) G[(size_t)k * K + l] = red[0];
}

// G^ = diag(sd) G diag(sd) / mean_k(sd_k^2 G_kk)
__global__ void k_prior_scale(const double* __restrict__ G, const float* __restrict__ sd, int K, float* __restrict__ Gh) {
  __shared__ double mean;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < K; ++k) t += (double)sd[k] * sd[k] * G[(size_t)k * K + k];
    mean = t / K;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < K * K; i += blockDim.x) {
    const int k = i / K, l = i - k * K;
    Gh[i] = (float)((double)sd[k] * G[i] * sd[l] / mean);
  }
}

struct TrainState {
  int step;
  float lr, bc1, bc2;  // learning rate, 1 - beta1^t, 1 - beta2^t
  float loss;
};

// advances the step counter and the one-cycle schedule (5 % linear warm-up, cosine decay)
__global__ void k_step_begin(TrainState* s, int total, float lr_max) {
  const int t = ++s->step;
  const float warm = fmaxf(1.f, 0.05f * total);
  float lr;
  if (t <= warm) lr = lr_max * t / warm;
  else lr = 0.5f * lr_max * (1.f + cosf(3.14159265358979f * (t - warm) / fmaxf(1.f, total - warm)));
  s->lr = lr;
  s->bc1 = 1.f - powf(0.9f, (float)t);
  s->bc2 = 1.f - powf(0.999f, (float)t);
  s->loss = 0.f;
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       size_t n, const TrainState* __restrict__ s) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = 0.9f * m[i] + 0.1f * gi;
  const float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= s->lr * (mi / s->bc1) / (sqrtf(vi / s->bc2) + 1e-8f);
}

// batch: X[b][j] = a[idx][j] in_scale[j], T[b][k] = (w[idx][k] - mu[k]) / sd[k], idx from Philox (tag 5)
__global__ void k_gather(const float* __restrict__ Af, int n, int ntrain, int J, const float* __restrict__ Wt, int K,
                         const float* __restrict__ in_scale, const float* __restrict__ mu,
                         const float* __restrict__ sd, int B, uint64_t seed, const TrainState* __restrict__ s,
                         float* __restrict__ X, float* __restrict__ T) {
  const int b = blockIdx.x;
  __shared__ int idx;
  if (threadIdx.x == 0) {
    const uint4 w = philox_at(seed, dfp2s_subsequence(5u, (uint32_t)s->step, 0u), (uint64_t)b);
    idx = (int)(((uint64_t)w.x * (uint64_t)ntrain) >> 32);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < J; j += blockDim.x) X[(size_t)b * J + j] = Af[(size_t)j * n + idx] * in_scale[j];
  for (int k = threadIdx.x; k < K; k += blockDim.x)
    T[(size_t)b * K + k] = (Wt[(size_t)idx * K + k] - mu[k]) / sd[k];
}

// uniform(-r, r) initialisation of weights from Philox tag 4, zero biases
__global__ void k_init_params(float* __restrict__ p, size_t n, size_t off, int fan_in, int is_bias, uint64_t seed) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (is_bias) {
    p[i] = 0.f;
    return;
  }
  const uint4 w = philox_at(seed, dfp2s_subsequence(4u, 0u, 0u), off + i);
  const float u = ((float)(w.x >> 8) + 0.5f) * (1.f / 16777216.f);
  p[i] = (2.f * u - 1.f) / sqrtf((float)fan_in);
}

// per-column mean and standard deviation over n rows (FP64 accumulation)
// data(row, col) = colmajor ? X[col * n + row] : X[row * ncol + col]
__global__ void k_col_stats(const float* __restrict__ X, int n, int ncol, int colmajor, float* __restrict__ mean,
                            float* __restrict__ stdv) {
  const int c = blockIdx.x;
  double s = 0.0, s2 = 0.0;
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    const double v = colmajor ? X[(size_t)c * n + r] : X[(size_t)r * ncol + c];
    s += v;
    s2 += v * v;
  }
  __shared__ double rs[256], rs2[256];
  rs[threadIdx.x] = s;
  rs2[threadIdx.x] = s2;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      rs[threadIdx.x] += rs[threadIdx.x + o];
      rs2[threadIdx.x] += rs2[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double m = rs[0] / n;
    const double var = fmax(rs2[0] / n - m * m, 0.0);
    mean[c] = (float)m;
    stdv[c] = (float)sqrt(var);
  }
}

__global__ void k_inscale(const float* __restrict__ sd, int J, float* __restrict__ in_scale) {
  const int j = threadIdx.x;
  if (j < J) in_scale[j] = (j < 2 || !(sd[j] > 0.f)) ? 0.f : 1.f / sd[j];
}

__global__ void k_loss_weights(const float* __restrict__ sd, int K, int psf, float* __restrict__ lw) {
  __shared__ float tot;
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int k = 0; k < K; ++k) t += sd[k] * sd[k];
    tot = t / K;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < K; k += blockDim.x) lw[k] = psf ? sd[k] * sd[k] / tot : 1.f;
}

// ||pred - ref||^2 and ||ref||^2 over n x K
__global__ void k_err(const float* __restrict__ pred, const float* __restrict__ ref, size_t n, double* __restrict__ acc) {
  double d = 0.0, r = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double e = (double)pred[i] - ref[i];
    d += e * e;
    r += (double)ref[i] * ref[i];
  }
  for (int off = 16; off > 0; off >>= 1) {
    d += __shfl_down_sync(0xffffffffu, d, off);
    r += __shfl_down_sync(0xffffffffu, r, off);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&acc[0], d);
    atomicAdd(&acc[1], r);
  }
}

struct Net {
  int J, K;
  float *W1, *b1, *W2, *b2, *W3, *b3;
  size_t n;
};

Net carve(float* base, int J, int K) {
  Net t;
  t.J = J;
  t.K = K;
  t.W1 = base;
  t.b1 = t.W1 + (size_t)HID * J;
  t.W2 = t.b1 + HID;
  t.b2 = t.W2 + (size_t)HID * HID;
  t.W3 = t.b2 + HID;
  t.b3 = t.W3 + (size_t)K * HID;
  t.n = (size_t)HID * J + HID + (size_t)HID * HID + HID + (size_t)K * HID + K;
  return t;
}

struct Act {
  float *Z1, *H1, *Z2, *H2, *Y, *dY, *dH2, *dH1, *RG;
};

// forward and backward of one batch (X: B x J, T: B x K) into the flat gradient buffer g
// (G, K x K symmetric, selects the quadratic-form loss; otherwise the per-k weights lw)
void fwd_bwd(cudaStream_t st, const Net& p, const Net& g, const Act& a, const float* X, const float* T,
             const float* lw, const float* G, int B, float* loss) {
  const int J = p.J, K = p.K;
  gemm<false, true, EPI_BIAS_GELU>(st, B, HID, J, X, J, p.W1, J, a.H1, HID, p.b1, a.Z1);
  gemm<false, true, EPI_BIAS_GELU>(st, B, HID, HID, a.H1, HID, p.W2, HID, a.H2, HID, p.b2, a.Z2);
  gemm<false, true, EPI_BIAS>(st, B, K, HID, a.H2, HID, p.W3, HID, a.Y, K, p.b3);
  const unsigned nb = (unsigned)(((size_t)B * K + 255) / 256);
  if (G) {
    k_residual<<<nb, 256, 0, st>>>(a.Y, T, (size_t)B * K, a.dY);
    gemm<false, false, EPI_NONE>(st, B, K, K, a.dY, K, G, K, a.RG, K);
    k_gram_loss_grad<<<nb, 256, 0, st>>>(a.RG, a.dY, B, K, loss);
  } else {
    k_loss_grad<<<nb, 256, 0, st>>>(a.Y, T, lw, B, K, a.dY, loss);
  }
  gemm<true, false, EPI_NONE>(st, K, HID, B, a.dY, K, a.H2, HID, g.W3, HID);
  k_colsum<<<(K + 31) / 32, 256, 0, st>>>(a.dY, B, K, g.b3);
  gemm<false, false, EPI_GELU_GRAD>(st, B, HID, K, a.dY, K, p.W3, HID, a.dH2, HID, nullptr, nullptr, a.Z2);
  gemm<true, false, EPI_NONE>(st, HID, HID, B, a.dH2, HID, a.H1, HID, g.W2, HID);
  k_colsum<<<(HID + 31) / 32, 256, 0, st>>>(a.dH2, B, HID, g.b2);
  gemm<false, false, EPI_GELU_GRAD>(st, B, HID, HID, a.dH2, HID, p.W2, HID, a.dH1, HID, nullptr, nullptr, a.Z1);
  gemm<true, false, EPI_NONE>(st, HID, J, B, a.dH1, HID, X, J, g.W1, J);
  k_colsum<<<(HID + 31) / 32, 256, 0, st>>>(a.dH1, B, HID, g.b1);
}

struct Pool {
  std::vector<void*> bufs;
  ~Pool() {
    for (void* b : bufs) cudaFree(b);
  }
  template <typename T>
  T* get(size_t n) {
    void* p = nullptr;
    if (dfp2s_device_malloc(&p, n * sizeof(T) + 16) != cudaSuccess) return nullptr;
    bufs.push_back(p);
    return static_cast<T*>(p);
  }
};

Act make_act(Pool& pool, int B, int K) {
  Act a;
  a.Z1 = pool.get<float>((size_t)B * HID);
  a.H1 = pool.get<float>((size_t)B * HID);
  a.Z2 = pool.get<float>((size_t)B * HID);
  a.H2 = pool.get<float>((size_t)B * HID);
  a.Y = pool.get<float>((size_t)B * K);
  a.dY = pool.get<float>((size_t)B * K);
  a.dH2 = pool.get<float>((size_t)B * HID);
  a.dH1 = pool.get<float>((size_t)B * HID);
  a.RG = pool.get<float>((size_t)B * K);
  return a;
}

bool act_ok(const Act& a) { return a.Z1 && a.H1 && a.Z2 && a.H2 && a.Y && a.dY && a.dH2 && a.dH1 && a.RG; }

}  // namespace

size_t dfp2s_mlp_nparams(int J, int K) { return carve(nullptr, J, K).n; }

int dfp2s_prior_gram_device(const float* basis, int K, const float* sd, float* Gh, cudaStream_t st) {
  Pool pool;
  double2* Tm = pool.get<double2>((size_t)K * PS * PM);
  double2* Phi = pool.get<double2>((size_t)K * PM * PM);
  double* G = pool.get<double>((size_t)K * K);
  if (!Tm || !Phi || !G) return DFP2S_ENOMEM;
  k_prior_dft_rows<<<K, 256, 0, st>>>(basis, Tm);
  k_prior_dft_cols<<<K, 256, 0, st>>>(Tm, Phi);
  k_prior_gram<<<dim3(K, K), 256, 0, st>>>(Phi, K, G);
  k_prior_scale<<<1, 256, 0, st>>>(G, sd, K, Gh);
  if (dfp2s_launch_status() != DFP2S_OK) return DFP2S_ECUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? DFP2S_OK : DFP2S_ECUDA;  // before the pool frees
}

int dfp2s_mlp_loss_grad_device(int J, int K, int B, const float* params, const float* X, const float* T,
                               const float* lw, const float* G, float* grads, float* loss, cudaStream_t st) {
  Pool pool;
  Act a = make_act(pool, B, K);
  if (!act_ok(a)) return DFP2S_ENOMEM;
  const Net p = carve(const_cast<float*>(params), J, K);
  const Net g = carve(grads, J, K);
  if (loss) cudaMemsetAsync(loss, 0, sizeof(float), st);
  fwd_bwd(st, p, g, a, X, T, lw, G, B, loss);
  if (dfp2s_launch_status() != DFP2S_OK) return DFP2S_ECUDA;
  return cudaStreamSynchronize(st) == cudaSuccess ? DFP2S_OK : DFP2S_ECUDA;
}

// Zernike vectors for n samples, fields layout [J][n]: z from Philox tag `tag`
// (Gaussian row s, column j of a rows x roundup4(J) block), a = L(D/r0_s) z with
// D/r0_s = dr[s % nd], tilt fields zeroed.
__global__ void k_draw_vectors(int n, int J, const float* __restrict__ L, const float* __restrict__ drs, int nd,
                               uint64_t seed, uint32_t tag, float* __restrict__ out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int cols = (J + 3) / 4 * 4;
  float z[DFP2S_MAX_J];
  const uint64_t sub = dfp2s_subsequence(tag, 0u, 0u);
  for (int q = 0; q < cols / 4; ++q) {
    const float4 g = dfp2s_gauss4(seed, sub, ((uint64_t)s * cols) / 4 + q);
    if (4 * q + 0 < J) z[4 * q + 0] = g.x;
    if (4 * q + 1 < J) z[4 * q + 1] = g.y;
    if (4 * q + 2 < J) z[4 * q + 2] = g.z;
    if (4 * q + 3 < J) z[4 * q + 3] = g.w;
  }
  const float sc = powf(drs[s % nd], 5.f / 6.f);
  for (int i = 0; i < J; ++i) {
    float acc = 0.f;
    for (int j = 0; j <= i; ++j) acc = fmaf(L[i * J + j], z[j], acc);
    out[(size_t)i * n + s] = i < 2 ? 0.f : acc * sc;
  }
}

int dfp2s_launch_draw_vectors(int n, int J, const float* L, const float* drs, int nd, uint64_t seed, uint32_t tag,
                              float* out, cudaStream_t st) {
  k_draw_vectors<<<(n + 127) / 128, 128, 0, st>>>(n, J, L, drs, nd, seed, tag, out);
  return dfp2s_launch_status();
}

int dfp2s_mlp_train_device(dfp2s_p2s_dev* p, const float* L32, const dfp2s_mlp_train_params* tp, float* report,
                           float* params_out_host, cudaStream_t st) {
  const int J = p->J, K = p->K, n = tp->n_pairs, B = tp->batch;
  const int nval = (int)(n * (double)tp->val_fraction);
  const int ntrain = n - nval;
  Pool pool;
  float* Af = pool.get<float>((size_t)J * n);
  float* Wt = pool.get<float>((size_t)n * K);
  float* drs = pool.get<float>(8);
  const size_t np = dfp2s_mlp_nparams(J, K);
  float* params = pool.get<float>(np);
  float* grads = pool.get<float>(np);
  float* m1 = pool.get<float>(np);
  float* m2 = pool.get<float>(np);
  float* in_mu = pool.get<float>(J);
  float* in_sd = pool.get<float>(J);
  float* in_scale = pool.get<float>(J);
  float* mu = pool.get<float>(K);
  float* sd = pool.get<float>(K);
  float* lw = pool.get<float>(K);
  float* Gh = tp->image_prior_loss ? pool.get<float>((size_t)K * K) : nullptr;
  float* X = pool.get<float>((size_t)B * J);
  float* T = pool.get<float>((size_t)B * K);
  TrainState* state = pool.get<TrainState>(1);
  double* eacc = pool.get<double>(2);
  Act a = make_act(pool, B, K);
  if (!Af || !Wt || !drs || !params || !grads || !m1 || !m2 || !in_mu || !in_sd || !in_scale || !mu || !sd || !lw ||
      !X || !T || !state || !eacc || !act_ok(a) || (tp->image_prior_loss && !Gh))
    return DFP2S_ENOMEM;
  float hdr[8];
  for (int i = 0; i < tp->n_dr; ++i) hdr[i] = (float)tp->D_over_r0[i];
  cudaMemcpyAsync(drs, hdr, tp->n_dr * sizeof(float), cudaMemcpyHostToDevice, st);
  // training pairs: vectors (tag 2) -> exact P2S weights
  int rc = dfp2s_launch_draw_vectors(n, J, L32, drs, tp->n_dr, tp->seed, 2u, Af, st);
  if (rc) return rc;
  if ((rc = dfp2s_launch_p2s_exact(p, Af, 1, n, Wt, DFP2S_W_F32, st))) return rc;
  // normalisation statistics over the training part
  k_col_stats<<<J, 256, 0, st>>>(Af, n, J, 1, in_mu, in_sd);
  k_col_stats<<<K, 256, 0, st>>>(Wt, ntrain, K, 0, mu, sd);
  k_inscale<<<1, 64, 0, st>>>(in_sd, J, in_scale);
  k_loss_weights<<<1, 128, 0, st>>>(sd, K, tp->psf_weighted_loss, lw);
  if (tp->image_prior_loss && (rc = dfp2s_prior_gram_device(p->basis, K, sd, Gh, st))) return rc;
  // parameters
  const Net pn = carve(params, J, K);
  const Net gn = carve(grads, J, K);
  struct Seg {
    float* ptr;
    size_t n;
    int fan, bias;
  } segs[6] = {{pn.W1, (size_t)HID * J, J, 0}, {pn.b1, HID, J, 1},        {pn.W2, (size_t)HID * HID, HID, 0},
               {pn.b2, HID, HID, 1},           {pn.W3, (size_t)K * HID, HID, 0}, {pn.b3, (size_t)K, HID, 1}};
  for (auto& sgm : segs) {
    const size_t off = sgm.ptr - params;
    k_init_params<<<(unsigned)((sgm.n + 255) / 256), 256, 0, st>>>(sgm.ptr, sgm.n, off, sgm.fan, sgm.bias, tp->seed);
  }
  cudaMemsetAsync(m1, 0, np * sizeof(float), st);
  cudaMemsetAsync(m2, 0, np * sizeof(float), st);
  cudaMemsetAsync(state, 0, sizeof(TrainState), st);
  if (dfp2s_launch_status() != DFP2S_OK) return DFP2S_ECUDA;
  // one training step, captured once and replayed
  cudaStream_t cs;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return DFP2S_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    cudaStreamDestroy(cs);
    return DFP2S_ECUDA;
  }
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  k_step_begin<<<1, 1, 0, cs>>>(state, tp->steps, tp->lr);
  k_gather<<<B, 128, 0, cs>>>(Af, n, ntrain, J, Wt, K, in_scale, mu, sd, B, tp->seed, state, X, T);
  fwd_bwd(cs, pn, gn, a, X, T, lw, Gh, B, &state->loss);
  k_adam<<<(unsigned)((np + 255) / 256), 256, 0, cs>>>(params, grads, m1, m2, np, state);
  cudaError_t ce = cudaStreamEndCapture(cs, &graph);
  if (ce == cudaSuccess) ce = cudaGraphInstantiate(&exec, graph, 0);
  if (ce != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    return DFP2S_ECUDA;
  }
  for (int s = 0; s < tp->steps; ++s) {
    if ((ce = cudaGraphLaunch(exec, cs)) != cudaSuccess) break;
  }
  TrainState hs;
  memset(&hs, 0, sizeof(hs));
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(&hs, state, sizeof(hs), cudaMemcpyDeviceToHost, cs);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(cs);
  cudaGraphExecDestroy(exec);
  cudaGraphDestroy(graph);
  cudaStreamDestroy(cs);
  if (ce != cudaSuccess) return DFP2S_ECUDA;
  // install the network: fold the standardisation into the handle's scales
  rc = dfp2s_p2s_install_mlp(p, pn.W1, pn.b1, pn.W2, pn.b2, pn.W3, pn.b3, in_scale, sd, mu);
  if (rc) return rc;
  // validation: weight relative L2 on the held-out pairs
  double herr[2] = {0.0, 0.0};
  if (nval > 0) {
    float* pred = pool.get<float>((size_t)nval * K);
    if (!pred) return DFP2S_ENOMEM;
    float* Aval = pool.get<float>((size_t)J * nval);
    if (!Aval) return DFP2S_ENOMEM;
    for (int j = 0; j < J; ++j)
      cudaMemcpyAsync(Aval + (size_t)j * nval, Af + (size_t)j * n + ntrain, nval * sizeof(float),
                      cudaMemcpyDeviceToDevice, st);
    if ((rc = dfp2s_launch_p2s_mlp(p, Aval, 1, nval, pred, DFP2S_W_F32, st))) return rc;
    cudaMemsetAsync(eacc, 0, 2 * sizeof(double), st);
    k_err<<<256, 256, 0, st>>>(pred, Wt + (size_t)ntrain * K, (size_t)nval * K, eacc);
    cudaMemcpyAsync(herr, eacc, 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
  }
  if (params_out_host) cudaMemcpyAsync(params_out_host, params, np * sizeof(float), cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) return DFP2S_ECUDA;
  if (report) {
    report[0] = hs.loss;
    report[1] = herr[1] > 0 ? (float)sqrt(herr[0] / herr[1]) : 0.f;
    report[2] = (float)hs.step;
  }
  return DFP2S_OK;
}
