// Internal launcher declarations shared by the translation units of libdfp2s.
// Every launcher enqueues work on `st` and returns DFP2S_OK or DFP2S_ECUDA.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/dfp2s.h"

// fields.cu -- Sec. III-C sampler passes
// prev != nullptr: fields = alpha prev + sqrt(1 - alpha^2) (this frame's fields), the auto-regressive form;
// mix = false: the unit fields before the mixing by scale L (prev must be null)
// sh: the factor whose subharmonic levels (if any) are added to the unit fields before the mixing
struct dfp2s_factor_dev;
int dfp2s_launch_sample_fields(float2* S, const float* mult, const float2* tw, int N, int J, int H, int W,
                               uint64_t seed, uint32_t frame, const float* L, float scale, float* fields,
                               cudaStream_t st, const float* prev = nullptr, float alpha = 0.f, bool mix = true,
                               int variant = -1, const dfp2s_factor_dev* sh = nullptr);
// the row pass alone (S as the column passes leave it), for the full sampler
int dfp2s_launch_rowifft(const float2* S, float* out, const float2* tw, int N, int J, int H, int W, cudaStream_t st);
int dfp2s_launch_philox_words(uint64_t seed, uint64_t sub, uint64_t q0, int nq, uint32_t* out, cudaStream_t st);
int dfp2s_launch_gaussian(uint64_t seed, uint64_t sub, size_t nq, float* out, cudaStream_t st);

// factor.cu -- FP64 spectral factor build
struct dfp2s_factor_dev {
  int J, N;
  double pix_per_D;
  float* mult;     // J x (N/2+1) x N, sqrt(lambda)/N^2
  double* L64;     // J x J, D/r0 = 1
  float* L32;      // J x J
  float2* tw;      // N twiddles exp(-2 pi i m / N)
  float2* scratch; // J x (N/2+1) x N spectrum
  // the full cross-spectral sampler (factor kind DFP2S_FACTOR_FULL; null otherwise)
  int R;                          // distinct radial orders of Noll 2..J+1
  float* fchol;                   // octant bins x R(R+1)/2 (padded to a multiple of 4): Cholesky factor of Gamma(|k|),
                                  // [a(a+1)/2 + b][o(o+1)/2 + r]
  struct dfp2s_full_mode* fmode;  // J mode constants
  float2* eta;                    // R x (N/2+1) x N order fields, then R x (N + N/2 + 1) for the Nyquist lines
  // the dense per-frequency root (factor kind DFP2S_FACTOR_DENSE; null otherwise)
  float* dense;                   // F[j * J + i][bin], bin = kx * N + ky over the half plane, FP32
  float2* espec;                  // J x (N/2+1) x N: this frame's E = F xi (per-frame scratch)
  // subharmonic levels of the factored sampler (0: none)
  int sh_levels;
  float* sh_amp;                  // J x levels x 8: s_{j,p,d}, normalised with lambda to unit variance
  float2* sh_coef;                // J x levels x 8: this frame's complex amplitudes (per-frame scratch)
};
// Per-mode constants of the full sampler: order slot, azimuthal frequency m, sin (odd Noll index) or cos, Noll's
// angular prefactor (complex) and kappa0 = sqrt(A0_jj (n+1) / sum_k P_jj(k)).
struct dfp2s_full_mode {
  int o, m, odd, pad;
  float pre_re, pre_im, kappa0, pad2;
};
// fields_dense.cu -- the dense-root sampler's per-frame passes (needs a factor built with DFP2S_FACTOR_DENSE)
int dfp2s_launch_sample_fields_dense(const dfp2s_factor_dev* f, int H, int W, uint64_t seed, uint32_t frame,
                                     float scale, float* fields, cudaStream_t st);
// Number of distinct radial orders among Noll modes 2..J+1.
int dfp2s_radial_order_count(int J);
// fields_full.cu -- the full sampler's per-frame passes (needs a factor built with the full tables)
int dfp2s_launch_sample_fields_full(const dfp2s_factor_dev* f, int H, int W, uint64_t seed, uint32_t frame,
                                    float scale, float* fields, cudaStream_t st);
int dfp2s_factor_build_device(dfp2s_factor_dev* f, cudaStream_t st);

// The opaque handle of include/dfp2s.h.
struct dfp2s_factor {
  dfp2s_factor_dev d;
  int kind;
  int device;  // device the factor's memory lives on
};

// warp.cu
int dfp2s_launch_tilt_warp(const float* img, int C, int H, int W, const float* a2, const float* a3, float* out,
                           cudaStream_t st);

// p2s.cu -- exact P2S constants and kernel
struct dfp2s_p2s_dev {
  int J, K;
  float* basis;   // K x 1089
  float* phiT;    // 1089 x K (transposed basis)
  float* zt;      // (J-2) x 1089 Zernike values of Noll 4..J+1 on the 33 x 33 pupil window
  float* mask;    // 1089 aperture mask
  float2* dft;    // 33 x 33, exp(-2 pi i (k-16)(i-16) / 64)
  float* flux;    // 2 K: s_k = sum_u phi_k(u), then s_k / (s^T s) (the unit-flux projection of the weights)
  // surrogate network (optional)
  int has_mlp;
  float *W1, *b1, *W2, *b2, *W3, *b3, *in_scale, *out_scale, *out_shift;
  // tensor-core blur: basis tiles, padded BF16 image scratch, device error word
  __nv_bfloat16* bt;
  __nv_bfloat16* pad;
  size_t pad_cap;
  int* err;
  float* bsum;  // centre * sum of each bfloat16 basis function (tensor-core blur)
  int prep_C, prep_H, prep_W;  // image shape whose shifted planes `pad` holds (tensor-core blur)
  // tensor-core surrogate: packed BF16 weights and the folded output offset
  __nv_bfloat16 *tc_w1, *tc_w2, *tc_w3;
  float* tc_c3;
  __nv_bfloat16* tc_bias;
  unsigned mlp_version;  // incremented by every network install  // hidden biases as the B operand of the bias MMAs
};
int dfp2s_p2s_build_tables(dfp2s_p2s_dev* p, cudaStream_t st);
// The opaque handle of include/dfp2s.h.
struct dfp2s_p2s {
  dfp2s_p2s_dev d;
};
// w_dtype for dfp2s_launch_p2s_exact that writes the normalised 33 x 33 PSFs (npix x 1089 FP32) instead of weights
#define DFP2S_W_PSF 2
int dfp2s_launch_p2s_exact(const dfp2s_p2s_dev* p, const float* fields, int H, int W, void* w, int w_dtype,
                           cudaStream_t st);
int dfp2s_launch_p2s_mlp(const dfp2s_p2s_dev* p, const float* fields, int H, int W, void* w, int w_dtype,
                         cudaStream_t st);

// api.cu -- installs surrogate weights (device pointers, row-major W1 256 x J, W2 256 x 256, W3 K x 256)
int dfp2s_p2s_install_mlp(dfp2s_p2s_dev* p, const float* W1, const float* b1, const float* W2, const float* b2,
                          const float* W3, const float* b3, const float* in_scale, const float* out_scale,
                          const float* out_shift);

// mlp_train.cu
size_t dfp2s_mlp_nparams(int J, int K);
int dfp2s_mlp_loss_grad_device(int J, int K, int B, const float* params, const float* X, const float* T,
                               const float* lw, const float* G, float* grads, float* loss, cudaStream_t st);
int dfp2s_prior_gram_device(const float* basis, int K, const float* sd, float* Gh, cudaStream_t st);
int dfp2s_mlp_train_device(dfp2s_p2s_dev* p, const float* L32, const dfp2s_mlp_train_params* tp, float* report,
                           float* params_out_host, cudaStream_t st);
int dfp2s_launch_draw_vectors(int n, int J, const float* L, const float* drs, int nd, uint64_t seed, uint32_t tag,
                              float* out, cudaStream_t st);

// mlp_tc.cu -- tensor-core surrogate inference
int dfp2s_mlp_tc_pack(dfp2s_p2s_dev* p, cudaStream_t st);
// first-layer weights for unmixed input: W1 diag(in_scale) L, packed like tc_w1 (HID x 48 bfloat16)
int dfp2s_mlp_tc_pack_w1_mixed(const dfp2s_p2s_dev* p, const float* L, __nv_bfloat16* out, cudaStream_t st);
size_t dfp2s_mlp_tc_w1_elems();
// w1 != nullptr: first-layer weights to use instead of tc_w1; the fields are multiplied by xscale on loading
int dfp2s_launch_mlp_tc(const dfp2s_p2s_dev* p, const float* fields, int npix, void* w, int w_dtype, cudaStream_t st,
                        const __nv_bfloat16* w1 = nullptr, float xscale = 1.f);

// stats.cu -- lagged covariances of fields (lags_host: n_lags (dy, dx) pairs; out: n_lags x J x J FP64, device)
int dfp2s_launch_field_covariance(const float* a, int J, int H, int W, const int* lags_host, int n_lags, double* out,
                                  cudaStream_t st);

// aperture.cu -- Sec. IV-B statistics (out as include/dfp2s.h documents for the two entry points)
int dfp2s_launch_aperture_statistics(const float* fields, int J, int H, int W, int step, double* out, cudaStream_t st);
int dfp2s_launch_tilt_statistics(const float* fields, int H, int W, int max_lag, double* out, cudaStream_t st);

// basis.cu -- FP64 SVD basis of exact PSFs
int dfp2s_basis_build_device(int J, const float* L32, int K, int n_psf, const double* dr_host, int n_dr, uint64_t seed,
                             float* basis_out, double* sigma_host, int* sweeps_out, cudaStream_t st);

// blur_tc.cu -- BF16 tcgen05 blur (weights in BF16)
int dfp2s_launch_blur_tc_prepare(dfp2s_p2s_dev* p, const float* img, int C, int H, int W, cudaStream_t st);
// m != nullptr: a2/a3 are the unit fields u0, u1 before the mixing, and the tilts are formed as the mixing
// does, t2 = m[0] u0, t3 = m[2] u1 + m[1] u0 (m = scale (L00, L10, L11))
int dfp2s_launch_blur_tc_prepare_warp(dfp2s_p2s_dev* p, const float* img, int C, int H, int W, const float* a2,
                                      const float* a3, cudaStream_t st, const float* m = nullptr);
int dfp2s_launch_blur_tc_run(dfp2s_p2s_dev* p, int C, int H, int W, const void* w, int w_dtype, float* out,
                             cudaStream_t st);
int dfp2s_launch_blur_tc(dfp2s_p2s_dev* p, const float* img, int C, int H, int W, const void* w, int w_dtype,
                         float* out, cudaStream_t st);

// blur.cu
int dfp2s_launch_blur(const dfp2s_p2s_dev* p, const float* img, int C, int H, int W, const void* w, int w_dtype,
                      float* out, cudaStream_t st);

// api.cu -- frame contexts: dfp2s_ctx_set_field_variant is declared in include/dfp2s.h
