// C ABI of libdfp2s (declared in include/dfp2s.h): argument checks, handle
// lifetimes, scratch ownership and the per-frame pipeline of Fig. dfp2s.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <vector>

#include "common.cuh"
#include "kernels.h"

// ---------------------------------------------------------------- errors
namespace {
thread_local char g_err[512] = {0};
thread_local int g_err_code = 0;

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }
}  // namespace

int dfp2s_fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  g_err_code = code;
  return code;
}

namespace {
thread_local cudaError_t g_launch_err = cudaSuccess;
}

// simulated allocation failure: the n-th next device allocation (1 = the next one) fails; 0 = none armed
static std::atomic<int> g_fail_alloc{0};

static bool take_simulated_failure() {
  int n = g_fail_alloc.load();
  while (n > 0) {
    if (g_fail_alloc.compare_exchange_weak(n, n - 1)) return n == 1;
  }
  return false;
}

cudaError_t dfp2s_device_malloc(void** p, size_t bytes) {
  if (take_simulated_failure()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

cudaError_t dfp2s_device_malloc_async(void** p, size_t bytes, cudaStream_t st) {
  if (take_simulated_failure()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMallocAsync(p, bytes, st);
}

extern "C" int dfp2s_debug_fail_allocation(int n) {
  if (n < 0 || n > (1 << 20)) return dfp2s_fail(DFP2S_EINVAL, "n = %d out of range", n);
  g_fail_alloc.store(n);
  return DFP2S_OK;
}

int dfp2s_launch_status() {
  const cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) return DFP2S_OK;
  g_launch_err = e;
  return DFP2S_ECUDA;
}

cudaError_t dfp2s_launch_error() {
  const cudaError_t e = g_launch_err;
  g_launch_err = cudaSuccess;
  return e != cudaSuccess ? e : cudaGetLastError();
}

int dfp2s_fail_cuda(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation) return dfp2s_fail(DFP2S_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
  return dfp2s_fail(DFP2S_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CHECK_ARG(cond, ...)                          \
  do {                                                \
    if (!(cond)) return dfp2s_fail(DFP2S_EINVAL, __VA_ARGS__); \
  } while (0)

#define CHECK_LAUNCH(expr)                                                          \
  do {                                                                              \
    if ((expr) != DFP2S_OK) return dfp2s_fail_cuda(dfp2s_launch_error(), #expr);      \
  } while (0)

extern "C" int dfp2s_last_error(char* buf, size_t n) {
  if (buf && n) {
    strncpy(buf, g_err, n - 1);
    buf[n - 1] = 0;
  }
  return g_err_code;
}

extern "C" const char* dfp2s_version(void) { return "dfp2s 0.1 sm_103a"; }

extern "C" int dfp2s_grid_size(int H, int W, double pix_per_D) {
  CHECK_ARG(H >= 1 && W >= 1 && H <= 4096 && W <= 4096, "image size %dx%d out of range", H, W);
  CHECK_ARG(pix_per_D > 0 && pix_per_D <= 64, "pix_per_D %g out of range", pix_per_D);
  const int need = (H > W ? H : W) + (int)ceil(4.0 * pix_per_D);
  int N = 1;
  while (N < need) N *= 2;
  CHECK_ARG(N <= 4096, "grid %d exceeds 4096", N);
  return N;
}

// ------------------------------------------------------------ spectral factor
static void factor_free(dfp2s_factor* f) {
  if (!f) return;
  cudaFree(f->d.mult);
  cudaFree(f->d.L64);
  cudaFree(f->d.L32);
  cudaFree(f->d.tw);
  cudaFree(f->d.scratch);
  cudaFree(f->d.fchol);
  cudaFree(f->d.fmode);
  cudaFree(f->d.eta);
  cudaFree(f->d.sh_amp);
  cudaFree(f->d.sh_coef);
  cudaFree(f->d.dense);
  cudaFree(f->d.espec);
  delete f;
}

extern "C" int dfp2s_build_spectral_factor(const dfp2s_factor_params* p, dfp2s_factor** out, void* stream) {
  CHECK_ARG(p && out, "null argument");
  *out = nullptr;
  CHECK_ARG(p->J >= 3 && p->J <= DFP2S_MAX_J, "J = %d out of range [3, %d]", p->J, DFP2S_MAX_J);
  CHECK_ARG(is_pow2(p->N) && p->N >= 16 && p->N <= 4096, "N = %d must be a power of two in [16, 4096]", p->N);
  CHECK_ARG(p->pix_per_D > 0 && p->pix_per_D <= 64, "pix_per_D out of range");
  CHECK_ARG(p->kind == DFP2S_FACTOR_FACTORED || p->kind == DFP2S_FACTOR_DENSE || p->kind == DFP2S_FACTOR_FULL,
            "unknown factor kind");
  if (p->kind == DFP2S_FACTOR_DENSE && p->J > 48)
    return dfp2s_fail(DFP2S_EUNSUPPORTED, "the dense root is built for J <= 48 (J = %d)", p->J);
  CHECK_ARG(p->subharmonic_levels >= 0 && p->subharmonic_levels <= 12, "subharmonic levels %d out of [0, 12]",
            p->subharmonic_levels);
  if (p->kind != DFP2S_FACTOR_FACTORED && p->subharmonic_levels > 0)
    return dfp2s_fail(DFP2S_EUNSUPPORTED, "subharmonics are built for the factored sampler only");
  dfp2s_factor* f = new dfp2s_factor();
  memset(&f->d, 0, sizeof(f->d));
  f->d.J = p->J;
  f->d.N = p->N;
  f->d.pix_per_D = p->pix_per_D;
  f->kind = p->kind;
  f->d.sh_levels = p->subharmonic_levels;
  cudaGetDevice(&f->device);
  const size_t half = (size_t)(p->N / 2 + 1) * p->N;
  cudaError_t e;
  if ((e = dfp2s_device_malloc((void**)&f->d.mult, (size_t)p->J * half * sizeof(float))) != cudaSuccess ||
      (e = dfp2s_device_malloc((void**)&f->d.L64, (size_t)p->J * p->J * sizeof(double))) != cudaSuccess ||
      (e = dfp2s_device_malloc((void**)&f->d.L32, (size_t)p->J * p->J * sizeof(float))) != cudaSuccess ||
      (e = dfp2s_device_malloc((void**)&f->d.tw, (size_t)p->N * sizeof(float2))) != cudaSuccess ||
      (e = dfp2s_device_malloc((void**)&f->d.scratch, (size_t)p->J * half * sizeof(float2))) != cudaSuccess) {
    factor_free(f);
    return dfp2s_fail_cuda(e, "factor allocation");
  }
  if (p->kind == DFP2S_FACTOR_DENSE) {
    if ((e = dfp2s_device_malloc((void**)&f->d.dense, (size_t)p->J * p->J * half * sizeof(float))) != cudaSuccess ||
        (e = dfp2s_device_malloc((void**)&f->d.espec, (size_t)p->J * half * sizeof(float2))) != cudaSuccess) {
      factor_free(f);
      return dfp2s_fail_cuda(e, "dense-root table allocation");
    }
  }
  if (p->subharmonic_levels > 0) {
    const size_t n = (size_t)p->J * p->subharmonic_levels * 8;
    if ((e = dfp2s_device_malloc((void**)&f->d.sh_amp, n * sizeof(float))) != cudaSuccess ||
        (e = dfp2s_device_malloc((void**)&f->d.sh_coef, n * sizeof(float2))) != cudaSuccess) {
      factor_free(f);
      return dfp2s_fail_cuda(e, "subharmonic table allocation");
    }
  }
  if (p->kind == DFP2S_FACTOR_FULL) {
    const int R = dfp2s_radial_order_count(p->J);
    const size_t noct = (size_t)(p->N / 2 + 1) * (p->N / 2 + 2) / 2;
    f->d.R = R;
    const size_t trip = (size_t)(R * (R + 1) / 2 + 3) / 4 * 4;  // Cholesky rows padded to whole float4
    if ((e = dfp2s_device_malloc((void**)&f->d.fchol, noct * trip * sizeof(float))) != cudaSuccess ||
        (e = dfp2s_device_malloc((void**)&f->d.fmode, (size_t)p->J * sizeof(dfp2s_full_mode))) != cudaSuccess ||
        (e = dfp2s_device_malloc((void**)&f->d.eta, (size_t)R * (half + p->N + p->N / 2 + 1) * sizeof(float2))) !=
            cudaSuccess) {
      factor_free(f);
      return dfp2s_fail_cuda(e, "full-sampler table allocation");
    }
  }
  const int rc = dfp2s_factor_build_device(&f->d, as_stream(stream));
  if (rc != DFP2S_OK) {
    factor_free(f);
    return rc;
  }
  *out = f;
  return DFP2S_OK;
}

extern "C" int dfp2s_factor_destroy(dfp2s_factor* f) {
  factor_free(f);
  return DFP2S_OK;
}

extern "C" int dfp2s_factor_copy_multiplier(const dfp2s_factor* f, float* dst, void* stream) {
  CHECK_ARG(f && dst, "null argument");
  const size_t n = (size_t)f->d.J * (f->d.N / 2 + 1) * f->d.N;
  DFP2S_CUDA_TRY(cudaMemcpyAsync(dst, f->d.mult, n * sizeof(float), cudaMemcpyDeviceToDevice, as_stream(stream)));
  return DFP2S_OK;
}

extern "C" int dfp2s_factor_copy_cholesky(const dfp2s_factor* f, double* dst_host) {
  CHECK_ARG(f && dst_host, "null argument");
  DFP2S_CUDA_TRY(cudaMemcpy(dst_host, f->d.L64, (size_t)f->d.J * f->d.J * sizeof(double), cudaMemcpyDeviceToHost));
  return DFP2S_OK;
}

extern "C" int dfp2s_factor_info(const dfp2s_factor* f, int* J, int* N, size_t* scratch_bytes) {
  CHECK_ARG(f, "null factor");
  if (J) *J = f->d.J;
  if (N) *N = f->d.N;
  if (scratch_bytes) *scratch_bytes = (size_t)f->d.J * (f->d.N / 2 + 1) * f->d.N * sizeof(float2);
  return DFP2S_OK;
}

extern "C" int dfp2s_sample_zernike_fields(const dfp2s_factor* f, double D_over_r0, uint64_t seed, uint32_t frame,
                                           int H, int W, float* fields, void* stream) {
  CHECK_ARG(f && fields, "null argument");
  CHECK_ARG(H >= 1 && W >= 1 && H <= f->d.N && W <= f->d.N, "frame %dx%d does not fit the %d grid", H, W, f->d.N);
  CHECK_ARG(D_over_r0 >= 0 && D_over_r0 <= 1e4, "D/r0 = %g out of range", D_over_r0);
  const float scale = (float)pow(D_over_r0, 5.0 / 6.0);
  CHECK_LAUNCH(dfp2s_launch_sample_fields(f->d.scratch, f->d.mult, f->d.tw, f->d.N, f->d.J, H, W, seed, frame,
                                          f->d.L32, scale, fields, as_stream(stream), nullptr, 0.f, true, -1,
                                          &f->d));
  return DFP2S_OK;
}

extern "C" int dfp2s_sample_zernike_fields_full(const dfp2s_factor* f, double D_over_r0, uint64_t seed,
                                                uint32_t frame, int H, int W, float* fields, void* stream) {
  CHECK_ARG(f && fields, "null argument");
  CHECK_ARG(f->kind == DFP2S_FACTOR_FULL, "the factor was not built with DFP2S_FACTOR_FULL");
  CHECK_ARG(H >= 1 && W >= 1 && H <= f->d.N && W <= f->d.N, "frame %dx%d does not fit the %d grid", H, W, f->d.N);
  CHECK_ARG(D_over_r0 >= 0 && D_over_r0 <= 1e4, "D/r0 = %g out of range", D_over_r0);
  const float scale = (float)pow(D_over_r0, 5.0 / 6.0);
  CHECK_LAUNCH(dfp2s_launch_sample_fields_full(&f->d, H, W, seed, frame, scale, fields, as_stream(stream)));
  return DFP2S_OK;
}

extern "C" int dfp2s_sample_zernike_fields_dense(const dfp2s_factor* f, double D_over_r0, uint64_t seed,
                                                 uint32_t frame, int H, int W, float* fields, void* stream) {
  CHECK_ARG(f && fields, "null argument");
  CHECK_ARG(f->kind == DFP2S_FACTOR_DENSE, "the factor was not built with DFP2S_FACTOR_DENSE");
  CHECK_ARG(H >= 1 && W >= 1 && H <= f->d.N && W <= f->d.N, "frame %dx%d does not fit the %d grid", H, W, f->d.N);
  CHECK_ARG(D_over_r0 >= 0 && D_over_r0 <= 1e4, "D/r0 = %g out of range", D_over_r0);
  const float scale = (float)pow(D_over_r0, 5.0 / 6.0);
  CHECK_LAUNCH(dfp2s_launch_sample_fields_dense(&f->d, H, W, seed, frame, scale, fields, as_stream(stream)));
  return DFP2S_OK;
}

extern "C" int dfp2s_factor_copy_dense_root(const dfp2s_factor* f, float* dst_dev, void* stream) {
  CHECK_ARG(f && dst_dev, "null argument");
  CHECK_ARG(f->kind == DFP2S_FACTOR_DENSE, "the factor was not built with DFP2S_FACTOR_DENSE");
  const size_t n = (size_t)f->d.J * f->d.J * (f->d.N / 2 + 1) * f->d.N;
  DFP2S_CUDA_TRY(cudaMemcpyAsync(dst_dev, f->d.dense, n * sizeof(float), cudaMemcpyDeviceToDevice, as_stream(stream)));
  return DFP2S_OK;
}

extern "C" int dfp2s_sample_zernike_fields_ar1(const dfp2s_factor* f, double D_over_r0, uint64_t seed, uint32_t frame,
                                               double alpha, int H, int W, const float* prev, float* fields,
                                               void* stream) {
  CHECK_ARG(f && fields, "null argument");
  CHECK_ARG(H >= 1 && W >= 1 && H <= f->d.N && W <= f->d.N, "frame %dx%d does not fit the %d grid", H, W, f->d.N);
  CHECK_ARG(D_over_r0 >= 0 && D_over_r0 <= 1e4, "D/r0 = %g out of range", D_over_r0);
  CHECK_ARG(alpha >= 0 && alpha < 1, "alpha = %g out of [0, 1)", alpha);
  CHECK_ARG(prev != fields, "prev must not alias fields");
  const float scale = (float)pow(D_over_r0, 5.0 / 6.0);
  CHECK_LAUNCH(dfp2s_launch_sample_fields(f->d.scratch, f->d.mult, f->d.tw, f->d.N, f->d.J, H, W, seed, frame,
                                          f->d.L32, scale, fields, as_stream(stream), prev, (float)alpha, true, -1,
                                          &f->d));
  return DFP2S_OK;
}

extern "C" int dfp2s_gaussian_noise(uint64_t seed, uint32_t tag, uint32_t frame, uint32_t mode, int rows, int cols,
                                    float* out, void* stream) {
  CHECK_ARG(out && rows >= 1 && cols >= 4 && cols % 4 == 0, "bad noise shape %dx%d", rows, cols);
  CHECK_ARG(mode < 256 && tag < (1u << 24), "mode/tag out of range");
  const uint64_t sub = ((uint64_t)tag << 40) | ((uint64_t)frame << 8) | mode;
  CHECK_LAUNCH(dfp2s_launch_gaussian(seed, sub, (size_t)rows * cols / 4, out, as_stream(stream)));
  return DFP2S_OK;
}

extern "C" int dfp2s_philox_words(uint64_t seed, uint64_t sub, uint64_t q0, int n, uint32_t* out, void* stream) {
  CHECK_ARG(out && n >= 4 && n % 4 == 0, "n must be a positive multiple of 4");
  CHECK_LAUNCH(dfp2s_launch_philox_words(seed, sub, q0, n / 4, out, as_stream(stream)));
  return DFP2S_OK;
}

extern "C" int dfp2s_build_basis(const dfp2s_factor* f, int K, int n_psf, const double* dr, int n_dr, uint64_t seed,
                                 float* basis, double* sigma_host, int* sweeps_host, void* stream) {
  CHECK_ARG(f && dr && basis, "null argument");
  CHECK_ARG(K >= 1 && K <= DFP2S_MAX_K, "K = %d out of range", K);
  CHECK_ARG(n_psf >= K && n_psf <= (1 << 16), "n_psf = %d out of range", n_psf);
  CHECK_ARG(n_dr >= 1 && n_dr <= 8, "n_dr out of range");
  for (int i = 0; i < n_dr; ++i) CHECK_ARG(dr[i] > 0 && dr[i] < 1e3, "bad D/r0");
  const int rc = dfp2s_basis_build_device(f->d.J, f->d.L32, K, n_psf, dr, n_dr, seed, basis, sigma_host, sweeps_host,
                                          as_stream(stream));
  if (rc == DFP2S_ENOMEM) return dfp2s_fail(rc, "basis allocation");
  if (rc) return dfp2s_fail_cuda(dfp2s_launch_error(), "basis build");
  return DFP2S_OK;
}

// ---------------------------------------------------------------------- P2S

static void p2s_free(dfp2s_p2s* p) {
  if (!p) return;
  void* bufs[] = {p->d.basis, p->d.phiT, p->d.zt,    p->d.mask, p->d.dft,  p->d.flux,     p->d.W1,        p->d.b1,
                  p->d.W2,    p->d.b2,   p->d.W3,    p->d.b3,   p->d.in_scale, p->d.out_scale, p->d.out_shift,
                  p->d.bt,    p->d.pad,  p->d.err,   p->d.bsum,     p->d.tc_w1,     p->d.tc_w2,     p->d.tc_w3,
                  p->d.tc_c3, p->d.tc_bias};
  for (void* b : bufs)
    if (b) cudaFree(b);
  delete p;
}

extern "C" int dfp2s_p2s_create(int J, int K, const float* basis, dfp2s_p2s** out) {
  CHECK_ARG(out && basis, "null argument");
  *out = nullptr;
  CHECK_ARG(J >= 3 && J <= DFP2S_MAX_J, "J = %d out of range", J);
  CHECK_ARG(K >= 1 && K <= DFP2S_MAX_K, "K = %d out of range [1, %d]", K, DFP2S_MAX_K);
  dfp2s_p2s* p = new dfp2s_p2s();
  memset(&p->d, 0, sizeof(p->d));
  p->d.J = J;
  p->d.K = K;
  const size_t n2 = DFP2S_KS * DFP2S_KS;
  cudaError_t e;
  if ((e = dfp2s_device_malloc((void**)&p->d.basis, K * n2 * sizeof(float))) != cudaSuccess ||
      (e = dfp2s_device_malloc((void**)&p->d.phiT, K * n2 * sizeof(float))) != cudaSuccess ||
      (e = dfp2s_device_malloc((void**)&p->d.zt, (J - 2) * n2 * sizeof(float))) != cudaSuccess ||
      (e = dfp2s_device_malloc((void**)&p->d.mask, n2 * sizeof(float))) != cudaSuccess ||
      (e = dfp2s_device_malloc((void**)&p->d.dft, n2 * sizeof(float2))) != cudaSuccess ||
      (e = dfp2s_device_malloc((void**)&p->d.flux, 2 * K * sizeof(float))) != cudaSuccess) {
    p2s_free(p);
    return dfp2s_fail_cuda(e, "p2s allocation");
  }
  if ((e = cudaMemcpy(p->d.basis, basis, K * n2 * sizeof(float), cudaMemcpyDefault)) != cudaSuccess) {
    p2s_free(p);
    return dfp2s_fail_cuda(e, "basis copy");
  }
  if (dfp2s_p2s_build_tables(&p->d, 0) != DFP2S_OK || (e = cudaDeviceSynchronize()) != cudaSuccess) {
    p2s_free(p);
    return dfp2s_fail_cuda(dfp2s_launch_error(), "p2s tables");
  }
  *out = p;
  return DFP2S_OK;
}

extern "C" int dfp2s_p2s_check(dfp2s_p2s* p) {
  CHECK_ARG(p, "null handle");
  if (!p->d.err) return DFP2S_OK;
  int h = 0;
  DFP2S_CUDA_TRY(cudaMemcpy(&h, p->d.err, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) {
    cudaMemset(p->d.err, 0, sizeof(int));
    return dfp2s_fail(DFP2S_ETIMEOUT, "a tensor-core kernel gave up waiting on a barrier (device error word %d)", h);
  }
  return DFP2S_OK;
}

extern "C" int dfp2s_p2s_destroy(dfp2s_p2s* p) {
  p2s_free(p);
  return DFP2S_OK;
}

// copies an (rows x cols) row-major device matrix to a newly allocated transposed (cols x rows) one
static cudaError_t copy_transposed(float** dst, const float* src, int rows, int cols) {
  std::vector<float> h((size_t)rows * cols), t((size_t)rows * cols);
  cudaError_t e = cudaMemcpy(h.data(), src, h.size() * sizeof(float), cudaMemcpyDefault);
  if (e != cudaSuccess) return e;
  for (int r = 0; r < rows; ++r)
    for (int c = 0; c < cols; ++c) t[(size_t)c * rows + r] = h[(size_t)r * cols + c];
  if ((e = dfp2s_device_malloc((void**)dst, t.size() * sizeof(float))) != cudaSuccess) return e;
  return cudaMemcpy(*dst, t.data(), t.size() * sizeof(float), cudaMemcpyHostToDevice);
}

static cudaError_t copy_vec(float** dst, const float* src, int n) {
  cudaError_t e = dfp2s_device_malloc((void**)dst, n * sizeof(float));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, src, n * sizeof(float), cudaMemcpyDefault);
}

int dfp2s_p2s_install_mlp(dfp2s_p2s_dev* d, const float* W1, const float* b1, const float* W2, const float* b2,
                          const float* W3, const float* b3, const float* in_scale, const float* out_scale,
                          const float* out_shift) {
  const int J = d->J, K = d->K;
  float** olds[] = {&d->W1, &d->b1, &d->W2, &d->b2, &d->W3, &d->b3, &d->in_scale, &d->out_scale, &d->out_shift};
  for (float** o : olds)
    if (*o) {
      cudaFree(*o);
      *o = nullptr;
    }
  d->has_mlp = 0;
  cudaError_t e;
  if ((e = copy_transposed(&d->W1, W1, 256, J)) != cudaSuccess || (e = copy_vec(&d->b1, b1, 256)) != cudaSuccess ||
      (e = copy_transposed(&d->W2, W2, 256, 256)) != cudaSuccess || (e = copy_vec(&d->b2, b2, 256)) != cudaSuccess ||
      (e = copy_transposed(&d->W3, W3, K, 256)) != cudaSuccess || (e = copy_vec(&d->b3, b3, K)) != cudaSuccess ||
      (e = copy_vec(&d->in_scale, in_scale, J)) != cudaSuccess ||
      (e = copy_vec(&d->out_scale, out_scale, K)) != cudaSuccess ||
      (e = copy_vec(&d->out_shift, out_shift, K)) != cudaSuccess)
    return dfp2s_fail_cuda(e, "mlp weights");
  if (!d->err) {
    if ((e = dfp2s_device_malloc((void**)&d->err, sizeof(int))) != cudaSuccess) return dfp2s_fail_cuda(e, "error word");
    cudaMemset(d->err, 0, sizeof(int));
  }
  const int rc = dfp2s_mlp_tc_pack(d, 0);
  if (rc == DFP2S_ENOMEM) return dfp2s_fail(rc, "tensor-core weight allocation");
  if (rc) return dfp2s_fail_cuda(dfp2s_launch_error(), "tensor-core weight packing");
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return dfp2s_fail_cuda(e, "tensor-core weight packing");
  d->has_mlp = 1;
  ++d->mlp_version;
  return DFP2S_OK;
}

extern "C" int dfp2s_p2s_set_mlp(dfp2s_p2s* p, const float* W1, const float* b1, const float* W2, const float* b2,
                                 const float* W3, const float* b3, const float* in_scale, const float* out_scale,
                                 const float* out_shift) {
  CHECK_ARG(p && W1 && b1 && W2 && b2 && W3 && b3 && in_scale && out_scale && out_shift, "null argument");
  return dfp2s_p2s_install_mlp(&p->d, W1, b1, W2, b2, W3, b3, in_scale, out_scale, out_shift);
}

// ---- statistics
extern "C" int dfp2s_field_covariance(const float* fields, int J, int H, int W, const int* lags, int n_lags,
                                      double* out, void* stream) {
  CHECK_ARG(fields && lags && out, "null argument");
  CHECK_ARG(J >= 1 && J <= DFP2S_MAX_J && H >= 1 && W >= 1 && (long long)H * W <= (1LL << 31),
            "field shape %d x %d x %d out of range", J, H, W);
  CHECK_ARG(n_lags >= 1 && n_lags <= 64, "%d lags out of range", n_lags);
  for (int l = 0; l < n_lags; ++l)
    CHECK_ARG(abs(lags[2 * l]) < H && abs(lags[2 * l + 1]) < W, "lag (%d, %d) does not fit %d x %d", lags[2 * l],
              lags[2 * l + 1], H, W);
  const int rc = dfp2s_launch_field_covariance(fields, J, H, W, lags, n_lags, out, as_stream(stream));
  if (rc == DFP2S_ENOMEM) return dfp2s_fail(rc, "covariance scratch allocation");
  if (rc != DFP2S_OK) return dfp2s_fail_cuda(dfp2s_launch_error(), "field covariance");
  return DFP2S_OK;
}

extern "C" int dfp2s_aperture_statistics(const float* fields, int J, int H, int W, int step, double* out,
                                         void* stream) {
  CHECK_ARG(fields && out, "null argument");
  CHECK_ARG(J >= 2 && J <= DFP2S_MAX_J && H >= 1 && W >= 1 && (long long)H * W <= (1LL << 31),
            "field shape %d x %d x %d out of range", J, H, W);
  CHECK_ARG(step >= 1 && step <= (H > W ? H : W) + 1, "step %d out of range", step);
  const int rc = dfp2s_launch_aperture_statistics(fields, J, H, W, step, out, as_stream(stream));
  if (rc == DFP2S_ENOMEM) return dfp2s_fail(rc, "aperture statistics scratch allocation");
  if (rc != DFP2S_OK) return dfp2s_fail_cuda(dfp2s_launch_error(), "aperture statistics");
  return DFP2S_OK;
}

extern "C" int dfp2s_tilt_statistics(const float* fields, int H, int W, int max_lag, double* out, void* stream) {
  CHECK_ARG(fields && out, "null argument");
  CHECK_ARG(H >= 1 && W >= 1 && (long long)H * W <= (1LL << 31), "field shape %d x %d out of range", H, W);
  CHECK_ARG(max_lag >= 0 && max_lag < H && max_lag < W && max_lag <= 1024, "max_lag %d out of range", max_lag);
  const int rc = dfp2s_launch_tilt_statistics(fields, H, W, max_lag, out, as_stream(stream));
  if (rc == DFP2S_ENOMEM) return dfp2s_fail(rc, "tilt statistics scratch allocation");
  if (rc != DFP2S_OK) return dfp2s_fail_cuda(dfp2s_launch_error(), "tilt statistics");
  return DFP2S_OK;
}

// ---- network files
static const char kMlpMagic[8] = {'D', 'F', 'P', '2', 'S', 'M', 'L', 'P'};

extern "C" int dfp2s_mlp_save(const dfp2s_p2s* p, const char* path) {
  CHECK_ARG(p && path, "null argument");
  const dfp2s_p2s_dev& d = p->d;
  CHECK_ARG(d.has_mlp, "no surrogate network installed");
  const int J = d.J, K = d.K;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return dfp2s_fail_cuda(e, "network save");
  // the handle keeps W1, W2, W3 transposed; the file holds them as dfp2s_p2s_set_mlp takes them
  auto fetch = [&](const float* src, size_t n, std::vector<float>& h) {
    h.resize(n);
    return cudaMemcpy(h.data(), src, n * sizeof(float), cudaMemcpyDeviceToHost);
  };
  auto untranspose = [](const std::vector<float>& t, int rows, int cols) {  // t is cols x rows
    std::vector<float> h((size_t)rows * cols);
    for (int r = 0; r < rows; ++r)
      for (int c = 0; c < cols; ++c) h[(size_t)r * cols + c] = t[(size_t)c * rows + r];
    return h;
  };
  std::vector<float> w1t, b1, w2t, b2, w3t, b3, isc, osc, osh;
  if ((e = fetch(d.W1, (size_t)256 * J, w1t)) != cudaSuccess || (e = fetch(d.b1, 256, b1)) != cudaSuccess ||
      (e = fetch(d.W2, (size_t)256 * 256, w2t)) != cudaSuccess || (e = fetch(d.b2, 256, b2)) != cudaSuccess ||
      (e = fetch(d.W3, (size_t)K * 256, w3t)) != cudaSuccess || (e = fetch(d.b3, K, b3)) != cudaSuccess ||
      (e = fetch(d.in_scale, J, isc)) != cudaSuccess || (e = fetch(d.out_scale, K, osc)) != cudaSuccess ||
      (e = fetch(d.out_shift, K, osh)) != cudaSuccess)
    return dfp2s_fail_cuda(e, "network save");
  const std::vector<float> W1 = untranspose(w1t, 256, J), W2 = untranspose(w2t, 256, 256),
                           W3 = untranspose(w3t, K, 256);
  FILE* fp = fopen(path, "wb");
  CHECK_ARG(fp, "cannot write %s", path);
  const uint32_t version = 1;
  const int32_t jk[2] = {J, K};
  bool ok = fwrite(kMlpMagic, 1, 8, fp) == 8 && fwrite(&version, 4, 1, fp) == 1 && fwrite(jk, 4, 2, fp) == 2;
  const std::vector<float>* parts[] = {&W1, &b1, &W2, &b2, &W3, &b3, &isc, &osc, &osh};
  for (const std::vector<float>* v : parts) ok = ok && fwrite(v->data(), sizeof(float), v->size(), fp) == v->size();
  ok = (fclose(fp) == 0) && ok;
  CHECK_ARG(ok, "short write to %s", path);
  return DFP2S_OK;
}

extern "C" int dfp2s_mlp_load(dfp2s_p2s* p, const char* path) {
  CHECK_ARG(p && path, "null argument");
  const int J = p->d.J, K = p->d.K;
  FILE* fp = fopen(path, "rb");
  CHECK_ARG(fp, "cannot read %s", path);
  char magic[8];
  uint32_t version = 0;
  int32_t jk[2] = {0, 0};
  bool ok = fread(magic, 1, 8, fp) == 8 && fread(&version, 4, 1, fp) == 1 && fread(jk, 4, 2, fp) == 2 &&
            memcmp(magic, kMlpMagic, 8) == 0 && version == 1 && jk[0] == J && jk[1] == K;
  std::vector<float> W1((size_t)256 * J), b1(256), W2((size_t)256 * 256), b2(256), W3((size_t)K * 256), b3(K),
      isc(J), osc(K), osh(K);
  std::vector<float>* parts[] = {&W1, &b1, &W2, &b2, &W3, &b3, &isc, &osc, &osh};
  for (std::vector<float>* v : parts) ok = ok && fread(v->data(), sizeof(float), v->size(), fp) == v->size();
  ok = ok && fgetc(fp) == EOF;
  fclose(fp);
  CHECK_ARG(ok, "%s is not a J = %d, K = %d network file", path, J, K);
  return dfp2s_p2s_install_mlp(&p->d, W1.data(), b1.data(), W2.data(), b2.data(), W3.data(), b3.data(), isc.data(),
                               osc.data(), osh.data());
}

extern "C" int dfp2s_mlp_param_count(int J, int K) {
  CHECK_ARG(J >= 3 && J <= DFP2S_MAX_J && K >= 1 && K <= DFP2S_MAX_K, "J/K out of range");
  return (int)dfp2s_mlp_nparams(J, K);
}

extern "C" int dfp2s_mlp_loss_grad(int J, int K, int B, const float* params, const float* X, const float* T,
                                   const float* lw, const float* G, float* grads, float* loss, void* stream) {
  CHECK_ARG(params && X && T && (lw || G) && grads, "null argument");
  CHECK_ARG(J >= 3 && J <= DFP2S_MAX_J && K >= 1 && K <= DFP2S_MAX_K && B >= 1 && B <= (1 << 20), "bad shape");
  const int rc = dfp2s_mlp_loss_grad_device(J, K, B, params, X, T, lw, G, grads, loss, as_stream(stream));
  if (rc == DFP2S_ENOMEM) return dfp2s_fail(rc, "mlp scratch allocation");
  if (rc) return dfp2s_fail_cuda(dfp2s_launch_error(), "mlp loss/grad");
  return DFP2S_OK;
}

extern "C" int dfp2s_mlp_image_prior_gram(const dfp2s_p2s* p, const float* sd, float* G, void* stream) {
  CHECK_ARG(p && sd && G, "null argument");
  const int rc = dfp2s_prior_gram_device(p->d.basis, p->d.K, sd, G, as_stream(stream));
  if (rc == DFP2S_ENOMEM) return dfp2s_fail(rc, "gram scratch allocation");
  if (rc) return dfp2s_fail_cuda(dfp2s_launch_error(), "image-prior loss form");
  return DFP2S_OK;
}

extern "C" int dfp2s_mlp_train(dfp2s_p2s* p, const dfp2s_factor* f, const dfp2s_mlp_train_params* tp, float* report,
                               float* params_out_host, void* stream) {
  CHECK_ARG(p && f && tp, "null argument");
  CHECK_ARG(f->d.J == p->d.J, "factor J %d != p2s J %d", f->d.J, p->d.J);
  CHECK_ARG(tp->n_pairs >= 1024 && tp->n_pairs <= (1 << 24), "n_pairs out of range");
  CHECK_ARG(tp->n_dr >= 1 && tp->n_dr <= 8, "n_dr out of range");
  for (int i = 0; i < tp->n_dr; ++i) CHECK_ARG(tp->D_over_r0[i] > 0 && tp->D_over_r0[i] < 1e3, "bad D/r0");
  CHECK_ARG(tp->batch >= 64 && tp->batch <= 8192, "batch out of range");
  CHECK_ARG(tp->steps >= 1 && tp->steps <= 10000000, "steps out of range");
  CHECK_ARG(tp->lr > 0 && tp->lr < 1, "lr out of range");
  CHECK_ARG(tp->val_fraction >= 0 && tp->val_fraction < 0.5, "val_fraction out of range");
  CHECK_ARG(tp->image_prior_loss == 0 || tp->image_prior_loss == 1, "image_prior_loss must be 0 or 1");
  const int rc = dfp2s_mlp_train_device(&p->d, f->d.L32, tp, report, params_out_host, as_stream(stream));
  if (rc == DFP2S_ENOMEM) return dfp2s_fail(rc, "training allocation");
  if (rc) return dfp2s_fail_cuda(dfp2s_launch_error(), "mlp training");
  return DFP2S_OK;
}

extern "C" int dfp2s_p2s_weights(const dfp2s_p2s* p, int mode, const float* fields, int H, int W, void* w,
                                 int w_dtype, void* stream) {
  CHECK_ARG(p && fields && w, "null argument");
  CHECK_ARG(H >= 1 && W >= 1 && (size_t)H * W <= (1u << 26), "frame %dx%d out of range", H, W);
  CHECK_ARG(w_dtype == DFP2S_W_F32 || w_dtype == DFP2S_W_BF16, "unknown weight dtype");
  if (mode == DFP2S_P2S_EXACT) {
    CHECK_LAUNCH(dfp2s_launch_p2s_exact(&p->d, fields, H, W, w, w_dtype, as_stream(stream)));
  } else if (mode == DFP2S_P2S_LEARNED) {
    CHECK_ARG(p->d.has_mlp, "no surrogate network installed");
    CHECK_ARG(p->d.J <= 48, "the tensor-core surrogate takes J <= 48 fields (J = %d); use LEARNED_FP32", p->d.J);
    CHECK_LAUNCH(dfp2s_launch_mlp_tc(&p->d, fields, H * W, w, w_dtype, as_stream(stream)));
  } else if (mode == DFP2S_P2S_LEARNED_FP32) {
    CHECK_ARG(p->d.has_mlp, "no surrogate network installed");
    CHECK_LAUNCH(dfp2s_launch_p2s_mlp(&p->d, fields, H, W, w, w_dtype, as_stream(stream)));
  } else {
    return dfp2s_fail(DFP2S_EINVAL, "unknown P2S mode %d", mode);
  }
  return DFP2S_OK;
}

extern "C" int dfp2s_tilt_warp(const float* img, int C, int H, int W, const float* a2, const float* a3, float* out,
                               void* stream) {
  CHECK_ARG(img && a2 && a3 && out, "null argument");
  CHECK_ARG(img != out, "out must not alias img");
  CHECK_ARG(C >= 1 && C <= 64 && H >= 1 && W >= 1 && H <= 65535 && W <= (1 << 20), "bad image shape");
  CHECK_LAUNCH(dfp2s_launch_tilt_warp(img, C, H, W, a2, a3, out, as_stream(stream)));
  return DFP2S_OK;
}

extern "C" int dfp2s_basis_blur(const dfp2s_p2s* p, const float* img, int C, int H, int W, const void* w,
                                int w_dtype, float* out, void* stream) {
  CHECK_ARG(p && img && w && out, "null argument");
  CHECK_ARG(img != out, "out must not alias img");
  CHECK_ARG(C >= 1 && C <= 64 && H >= 1 && W >= 1 && H <= 65535 * 4 && W <= (1 << 20), "bad image shape");
  CHECK_ARG(w_dtype == DFP2S_W_F32 || w_dtype == DFP2S_W_BF16, "unknown weight dtype");
  if (w_dtype == DFP2S_W_BF16) return dfp2s_basis_blur_tc(p, img, C, H, W, w, w_dtype, out, stream);
  CHECK_LAUNCH(dfp2s_launch_blur(&p->d, img, C, H, W, w, w_dtype, out, as_stream(stream)));
  return DFP2S_OK;
}

extern "C" int dfp2s_basis_blur_tc(const dfp2s_p2s* p, const float* img, int C, int H, int W, const void* w,
                                   int w_dtype, float* out, void* stream) {
  CHECK_ARG(p && img && w && out, "null argument");
  CHECK_ARG(img != out, "out must not alias img");
  CHECK_ARG(C >= 1 && C <= 64 && H >= 1 && W >= 1 && H <= 65535 - 32 && W <= (1 << 20), "bad image shape");
  CHECK_ARG(w_dtype == DFP2S_W_F32 || w_dtype == DFP2S_W_BF16, "unknown weight dtype");
  const int rc = dfp2s_launch_blur_tc(const_cast<dfp2s_p2s_dev*>(&p->d), img, C, H, W, w, w_dtype, out,
                                      as_stream(stream));
  if (rc == DFP2S_ENOMEM) return dfp2s_fail(rc, "blur scratch allocation");
  if (rc == DFP2S_EUNSUPPORTED) return dfp2s_fail(rc, "tensor-core blur supports K <= 128");
  if (rc != DFP2S_OK) return dfp2s_fail_cuda(dfp2s_launch_error(), "tensor-core blur launch");
  return DFP2S_OK;
}

extern "C" int dfp2s_basis_blur_tc_prepare(const dfp2s_p2s* p, const float* img, int C, int H, int W, void* stream) {
  CHECK_ARG(p && img, "null argument");
  CHECK_ARG(C >= 1 && C <= 64 && H >= 1 && W >= 1 && H <= 65535 - 32 && W <= (1 << 20), "bad image shape");
  const int rc = dfp2s_launch_blur_tc_prepare(const_cast<dfp2s_p2s_dev*>(&p->d), img, C, H, W, as_stream(stream));
  if (rc == DFP2S_ENOMEM) return dfp2s_fail(rc, "blur scratch allocation");
  if (rc == DFP2S_EUNSUPPORTED) return dfp2s_fail(rc, "tensor-core blur supports K <= 128");
  if (rc != DFP2S_OK) return dfp2s_fail_cuda(dfp2s_launch_error(), "tensor-core blur image preparation");
  return DFP2S_OK;
}

extern "C" int dfp2s_tilt_warp_blur_tc_prepare(const dfp2s_p2s* p, const float* img, int C, int H, int W,
                                               const float* a2, const float* a3, void* stream) {
  CHECK_ARG(p && img && a2 && a3, "null argument");
  CHECK_ARG(C >= 1 && C <= 64 && H >= 1 && W >= 1 && H <= 65535 - 32 && W <= (1 << 20), "bad image shape");
  const int rc = dfp2s_launch_blur_tc_prepare_warp(const_cast<dfp2s_p2s_dev*>(&p->d), img, C, H, W, a2, a3,
                                                   as_stream(stream));
  if (rc == DFP2S_ENOMEM) return dfp2s_fail(rc, "blur scratch allocation");
  if (rc == DFP2S_EUNSUPPORTED) return dfp2s_fail(rc, "tensor-core blur supports K <= 128");
  if (rc != DFP2S_OK) return dfp2s_fail_cuda(dfp2s_launch_error(), "warp + tensor-core blur preparation");
  return DFP2S_OK;
}

extern "C" int dfp2s_basis_blur_tc_run(const dfp2s_p2s* p, int C, int H, int W, const void* w, int w_dtype, float* out,
                                       void* stream) {
  CHECK_ARG(p && w && out, "null argument");
  CHECK_ARG(C >= 1 && C <= 64 && H >= 1 && W >= 1 && H <= 65535 - 32 && W <= (1 << 20), "bad image shape");
  CHECK_ARG(w_dtype == DFP2S_W_F32 || w_dtype == DFP2S_W_BF16, "unknown weight dtype");
  const int rc = dfp2s_launch_blur_tc_run(const_cast<dfp2s_p2s_dev*>(&p->d), C, H, W, w, w_dtype, out, as_stream(stream));
  if (rc == DFP2S_EINVAL) return dfp2s_fail(rc, "no prepared image of shape %dx%dx%d on this handle", C, H, W);
  if (rc == DFP2S_EUNSUPPORTED) return dfp2s_fail(rc, "tensor-core blur supports K <= 128 (and needs TMA)");
  if (rc != DFP2S_OK) return dfp2s_fail_cuda(dfp2s_launch_error(), "tensor-core blur launch");
  return DFP2S_OK;
}

// ------------------------------------------------------------------ frames
struct dfp2s_ctx {
  const dfp2s_factor* f;
  const dfp2s_p2s* p;
  int maxC, maxH, maxW;
  float* fields;
  float* warped;
  void* w;
  // learned frames: the first layer for unmixed fields, W1 diag(in_scale) L, and the network version it was
  // packed for; the top-left 2 x 2 block of L (host copy) for the tilt rows
  __nv_bfloat16* w1_mixed;
  unsigned w1_mixed_version;
  float l00, l10, l11;
  // stage timing: a ring of nev frames x 5 events, frames recorded so far
  cudaEvent_t* ev;
  int nev;
  unsigned long long frames;
  int field_variant;  // column-pass kernel of the field sampler (-1: the default)
  int field_sampler;  // DFP2S_FIELDS_FACTORED, _DENSE or _FULL
};

extern "C" int dfp2s_ctx_set_field_sampler(dfp2s_ctx* c, int sampler) {
  CHECK_ARG(c, "null context");
  CHECK_ARG(sampler == DFP2S_FIELDS_FACTORED || sampler == DFP2S_FIELDS_DENSE || sampler == DFP2S_FIELDS_FULL,
            "unknown field sampler %d", sampler);
  CHECK_ARG(sampler != DFP2S_FIELDS_DENSE || c->f->kind == DFP2S_FACTOR_DENSE,
            "the dense sampler needs a DFP2S_FACTOR_DENSE factor");
  CHECK_ARG(sampler != DFP2S_FIELDS_FULL || c->f->kind == DFP2S_FACTOR_FULL,
            "the full sampler needs a DFP2S_FACTOR_FULL factor");
  c->field_sampler = sampler;
  return DFP2S_OK;
}

// The mixed fields a (J x H x W) of a frame by the dense or the full sampler (no mixing pass follows).
static int ctx_mixed_fields(dfp2s_ctx* c, int H, int W, uint64_t seed, uint32_t frame, float scale, cudaStream_t st) {
  if (c->field_sampler == DFP2S_FIELDS_DENSE)
    return dfp2s_launch_sample_fields_dense(&c->f->d, H, W, seed, frame, scale, c->fields, st);
  return dfp2s_launch_sample_fields_full(&c->f->d, H, W, seed, frame, scale, c->fields, st);
}

extern "C" int dfp2s_ctx_set_field_variant(dfp2s_ctx* c, int variant) {
  if (!c || variant < -1 || variant > 1) return dfp2s_fail(DFP2S_EINVAL, "bad field-sampler variant %d", variant);
  c->field_variant = variant;
  return DFP2S_OK;
}

static void ctx_free_events(dfp2s_ctx* c) {
  for (int i = 0; i < 5 * c->nev; ++i) cudaEventDestroy(c->ev[i]);
  delete[] c->ev;
  c->ev = nullptr;
  c->nev = 0;
  c->frames = 0;
}

extern "C" int dfp2s_ctx_create(const dfp2s_factor* f, const dfp2s_p2s* p, int maxC, int maxH, int maxW,
                                dfp2s_ctx** out) {
  CHECK_ARG(f && p && out, "null argument");
  *out = nullptr;
  CHECK_ARG(f->d.J == p->d.J, "factor J %d != p2s J %d", f->d.J, p->d.J);
  CHECK_ARG(maxC >= 1 && maxC <= 64 && maxH >= 1 && maxW >= 1 && maxH <= f->d.N && maxW <= f->d.N,
            "context shape does not fit the factor grid");
  dfp2s_ctx* c = new dfp2s_ctx();
  c->f = f;
  c->p = p;
  c->maxC = maxC;
  c->maxH = maxH;
  c->maxW = maxW;
  c->fields = nullptr;
  c->warped = nullptr;
  c->w = nullptr;
  c->w1_mixed = nullptr;
  c->w1_mixed_version = 0;
  c->ev = nullptr;
  c->nev = 0;
  c->frames = 0;
  c->field_variant = -1;
  c->field_sampler = DFP2S_FIELDS_FACTORED;
  const size_t npix = (size_t)maxH * maxW;
  const int J = f->d.J;
  float lt[4] = {1.f, 0.f, 0.f, 1.f};
  cudaError_t e;
  if ((e = dfp2s_device_malloc((void**)&c->fields, (size_t)J * npix * sizeof(float))) != cudaSuccess ||
      (e = dfp2s_device_malloc((void**)&c->warped, (size_t)maxC * npix * sizeof(float))) != cudaSuccess ||
      (e = dfp2s_device_malloc(&c->w, (size_t)p->d.K * npix * sizeof(float))) != cudaSuccess ||
      (e = dfp2s_device_malloc((void**)&c->w1_mixed, dfp2s_mlp_tc_w1_elems() * sizeof(__nv_bfloat16))) != cudaSuccess ||
      (J >= 2 && ((e = cudaMemcpy(lt, f->d.L32, 2 * sizeof(float), cudaMemcpyDeviceToHost)) != cudaSuccess ||
                  (e = cudaMemcpy(lt + 2, f->d.L32 + J, 2 * sizeof(float), cudaMemcpyDeviceToHost)) != cudaSuccess))) {
    cudaFree(c->fields);
    cudaFree(c->warped);
    cudaFree(c->w);
    cudaFree(c->w1_mixed);
    delete c;
    return dfp2s_fail_cuda(e, "context allocation");
  }
  c->l00 = lt[0];
  c->l10 = lt[2];
  c->l11 = lt[3];
  *out = c;
  return DFP2S_OK;
}

extern "C" int dfp2s_ctx_destroy(dfp2s_ctx* c) {
  if (!c) return DFP2S_OK;
  cudaFree(c->fields);
  cudaFree(c->warped);
  cudaFree(c->w);
  cudaFree(c->w1_mixed);
  ctx_free_events(c);
  delete c;
  return DFP2S_OK;
}

extern "C" int dfp2s_ctx_stage_timing(dfp2s_ctx* c, int n) {
  CHECK_ARG(c && n >= 0 && n <= 100000, "bad stage-timing request");
  ctx_free_events(c);
  if (n == 0) return DFP2S_OK;
  c->ev = new cudaEvent_t[5 * (size_t)n]();
  for (int i = 0; i < 5 * n; ++i) {
    const cudaError_t e = cudaEventCreate(&c->ev[i]);
    if (e != cudaSuccess) {
      for (int k = 0; k < i; ++k) cudaEventDestroy(c->ev[k]);
      delete[] c->ev;
      c->ev = nullptr;
      return dfp2s_fail_cuda(e, "stage-timing events");
    }
  }
  c->nev = n;
  c->frames = 0;
  return DFP2S_OK;
}

extern "C" int dfp2s_ctx_stage_times(dfp2s_ctx* c, int count, float* out) {
  CHECK_ARG(c && out, "null argument");
  CHECK_ARG(c->nev > 0 && count >= 1 && count <= c->nev && (unsigned long long)count <= c->frames,
            "%d frames requested, %llu recorded in a ring of %d", count, c->frames, c->nev);
  for (int i = 0; i < count; ++i) {
    const unsigned long long fr = c->frames - (unsigned long long)count + (unsigned long long)i;
    cudaEvent_t* e = c->ev + 5 * (size_t)(fr % (unsigned long long)c->nev);
    cudaError_t r = cudaEventSynchronize(e[4]);
    if (r != cudaSuccess) return dfp2s_fail_cuda(r, "stage-timing wait");
    for (int s = 0; s < 4; ++s) {
      r = cudaEventElapsedTime(out + 4 * (size_t)i + s, e[s], e[s + 1]);
      if (r != cudaSuccess) return dfp2s_fail_cuda(r, "stage-timing read");
    }
  }
  return DFP2S_OK;
}

extern "C" int dfp2s_ctx_buffers(const dfp2s_ctx* c, float** fields, float** warped, void** w) {
  CHECK_ARG(c, "null context");
  if (fields) *fields = c->fields;
  if (warped) *warped = c->warped;
  if (w) *w = c->w;
  return DFP2S_OK;
}

extern "C" int dfp2s_simulate_frame(dfp2s_ctx* c, const float* img, int C, int H, int W, double D_over_r0,
                                    uint64_t seed, uint32_t frame, int p2s_mode, float* out, void* stream) {
  CHECK_ARG(c && img && out, "null argument");
  CHECK_ARG(img != out, "out must not alias img");
  CHECK_ARG(C >= 1 && C <= c->maxC && H >= 1 && H <= c->maxH && W >= 1 && W <= c->maxW,
            "frame %dx%dx%d exceeds the context's %dx%dx%d", C, H, W, c->maxC, c->maxH, c->maxW);
  CHECK_ARG(p2s_mode == DFP2S_P2S_EXACT || p2s_mode == DFP2S_P2S_LEARNED || p2s_mode == DFP2S_P2S_LEARNED_FP32,
            "unknown P2S mode");
  const size_t npix = (size_t)H * W;
  int rc;
  // stage events (when enabled): start, fields, warp, P2S weights, blur
  cudaEvent_t* ev = c->nev > 0 ? c->ev + 5 * (size_t)(c->frames % (unsigned long long)c->nev) : nullptr;
  auto mark = [&](int s) {
    if (ev) cudaEventRecord(ev[s], as_stream(stream));
  };
  mark(0);
  if (p2s_mode == DFP2S_P2S_LEARNED) {
    // The mixing a = scale L u of Sec. III-C is linear, so it moves into its two consumers: the warp forms the
    // tilt rows of a from u0, u1 (in the mixing kernel's operation order, bit for bit), and the network's first
    // layer takes W1 diag(in_scale) L with the fields scaled on loading.  The unit fields u stay in c->fields.
    const dfp2s_p2s_dev* pd = &c->p->d;
    CHECK_ARG(pd->has_mlp, "no surrogate network installed");
    CHECK_ARG(pd->J <= 48 && pd->J >= 2, "the tensor-core surrogate takes 2 <= J <= 48 fields (J = %d)", pd->J);
    CHECK_ARG(H <= c->f->d.N && W <= c->f->d.N && D_over_r0 >= 0 && D_over_r0 <= 1e4, "bad frame arguments");
    cudaStream_t st = as_stream(stream);
    const float scale = (float)pow(D_over_r0, 5.0 / 6.0);
    if (c->field_sampler != DFP2S_FIELDS_FACTORED) {
      // the dense and the full samplers give the mixed fields a: the warp reads their tilt rows as they are and the
      // network takes its own first layer W1 diag(in_scale)
      CHECK_LAUNCH(ctx_mixed_fields(c, H, W, seed, frame, scale, st));
      mark(1);
      rc = dfp2s_launch_blur_tc_prepare_warp(const_cast<dfp2s_p2s_dev*>(pd), img, C, H, W, c->fields,
                                             c->fields + npix, st, nullptr);
      if (rc == DFP2S_ENOMEM) return dfp2s_fail(rc, "blur scratch allocation");
      if (rc == DFP2S_EUNSUPPORTED) return dfp2s_fail(rc, "tensor-core blur supports K <= 128");
      if (rc != DFP2S_OK) return dfp2s_fail_cuda(dfp2s_launch_error(), "warp + tensor-core blur preparation");
      mark(2);
      CHECK_LAUNCH(dfp2s_launch_mlp_tc(pd, c->fields, H * W, c->w, DFP2S_W_F32, st));
      mark(3);
      rc = dfp2s_basis_blur_tc_run(c->p, C, H, W, c->w, DFP2S_W_F32, out, stream);
      if (rc) return rc;
      mark(4);
      if (ev) ++c->frames;
      return DFP2S_OK;
    }
    CHECK_LAUNCH(dfp2s_launch_sample_fields(c->f->d.scratch, c->f->d.mult, c->f->d.tw, c->f->d.N, c->f->d.J, H, W,
                                            seed, frame, c->f->d.L32, scale, c->fields, st, nullptr, 0.f, false,
                                            c->field_variant, &c->f->d));
    if (c->w1_mixed_version != pd->mlp_version) {
      CHECK_LAUNCH(dfp2s_mlp_tc_pack_w1_mixed(pd, c->f->d.L32, c->w1_mixed, st));
      c->w1_mixed_version = pd->mlp_version;
    }
    mark(1);
    const float m[3] = {c->l00 * scale, c->l10 * scale, c->l11 * scale};
    rc = dfp2s_launch_blur_tc_prepare_warp(const_cast<dfp2s_p2s_dev*>(pd), img, C, H, W, c->fields,
                                           c->fields + npix, st, m);
    if (rc == DFP2S_ENOMEM) return dfp2s_fail(rc, "blur scratch allocation");
    if (rc == DFP2S_EUNSUPPORTED) return dfp2s_fail(rc, "tensor-core blur supports K <= 128");
    if (rc != DFP2S_OK) return dfp2s_fail_cuda(dfp2s_launch_error(), "warp + tensor-core blur preparation");
    mark(2);
    CHECK_LAUNCH(dfp2s_launch_mlp_tc(pd, c->fields, H * W, c->w, DFP2S_W_F32, st, c->w1_mixed, scale));
    mark(3);
    rc = dfp2s_basis_blur_tc_run(c->p, C, H, W, c->w, DFP2S_W_F32, out, stream);
  } else {
    CHECK_ARG(D_over_r0 >= 0 && D_over_r0 <= 1e4, "D/r0 = %g out of range", D_over_r0);
    const float scale = (float)pow(D_over_r0, 5.0 / 6.0);
    if (c->field_sampler != DFP2S_FIELDS_FACTORED) {
      CHECK_ARG(H <= c->f->d.N && W <= c->f->d.N, "frame does not fit the %d grid", c->f->d.N);
      CHECK_LAUNCH(ctx_mixed_fields(c, H, W, seed, frame, scale, as_stream(stream)));
    } else {
      CHECK_LAUNCH(dfp2s_launch_sample_fields(c->f->d.scratch, c->f->d.mult, c->f->d.tw, c->f->d.N, c->f->d.J, H,
                                              W, seed, frame, c->f->d.L32, scale, c->fields, as_stream(stream),
                                              nullptr, 0.f, true, c->field_variant, &c->f->d));
    }
    mark(1);
    rc = dfp2s_tilt_warp(img, C, H, W, c->fields, c->fields + npix, c->warped, stream);
    if (rc) return rc;
    mark(2);
    rc = dfp2s_p2s_weights(c->p, p2s_mode, c->fields, H, W, c->w, DFP2S_W_F32, stream);
    if (rc) return rc;
    mark(3);
    if (p2s_mode == DFP2S_P2S_EXACT) rc = dfp2s_basis_blur(c->p, c->warped, C, H, W, c->w, DFP2S_W_F32, out, stream);
    else rc = dfp2s_basis_blur_tc(c->p, c->warped, C, H, W, c->w, DFP2S_W_F32, out, stream);
  }
  if (rc) return rc;
  mark(4);
  if (ev) ++c->frames;
  return DFP2S_OK;
}
