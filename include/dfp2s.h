/*
 * dfp2s.h -- C ABI of the GB300 (sm_103a) dense-field phase-to-space (DF-P2S)
 * turbulence simulator.
 *
 * Method: N. Chimitt, X. Zhang, Z. Mao, S. H. Chan, "Real-Time Dense Field
 * Phase-to-Space Simulation of Imaging through Atmospheric Turbulence",
 * arXiv 2210.06713.  One frame is
 *   1. J per-pixel Zernike coefficient fields (Noll modes 2..J+1) drawn from the
 *      homogeneous approximation of the Zernike correlation tensor
 *      (Sec. III-C, Eq. A-tilde): white noise -> 2-D FFT per mode ->
 *      per-frequency multiply by the spectral square root -> inverse FFT ->
 *      pixel-wise mixing with L, L L^T = A_0 (Noll's covariance);
 *   2. a tilt warp by the two tilt fields (the linear-phase part of Eq. 2);
 *   3. phase-to-space (Sec. II-C): each pixel's Zernike vector -> weights w on K
 *      basis PSFs -> out(x) = sum_k w_k(x) (phi_k (*) I)(x) (Eq. varying blur).
 *
 * Conventions (all entry points):
 *   - Every function returns an int status: DFP2S_OK (0) or a negative
 *     DFP2S_E* code.  A failed call sets a thread-local message readable with
 *     dfp2s_last_error().  No C++ exception crosses this boundary.
 *   - Pointers named *_dev are CUDA device pointers owned by the caller; *_host
 *     are host pointers.  Handles (dfp2s_factor, dfp2s_p2s, dfp2s_ctx) are owned
 *     by the library and released by their *_destroy call.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Work is enqueued asynchronously; argument and launch errors are reported
 *     synchronously, device-side results are ready after the stream is
 *     synchronised.  Calls sharing one handle must be ordered on one stream.
 *   - Layouts are row-major: images planar C x H x W float32; fields J x H x W
 *     float32 with index 0 = Noll mode 2 (x tilt), 1 = Noll 3 (y tilt);
 *     weights pixel-major H x W x K (float32 or bfloat16); basis K x 33 x 33.
 *   - x is the image column, y the image row.
 *   - The library never falls back to host computation: without a usable
 *     sm_103a device every compute call fails with DFP2S_ECUDA.
 */
#ifndef DFP2S_H
#define DFP2S_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define DFP2S_OK 0
#define DFP2S_EINVAL (-1)      /* bad argument: null pointer, size out of range */
#define DFP2S_ENOMEM (-2)      /* device allocation failed */
#define DFP2S_ECUDA (-3)       /* CUDA runtime or launch error */
#define DFP2S_ETIMEOUT (-4)    /* a bounded device-side wait gave up */
#define DFP2S_EUNSUPPORTED (-5) /* valid request this build does not handle */

#define DFP2S_W_F32 0   /* weight storage: float32 */
#define DFP2S_W_BF16 1  /* weight storage: bfloat16 */

#define DFP2S_P2S_EXACT 0    /* pupil-FFT PSF + projection (Eq. 2, Sec. II-C) */
#define DFP2S_P2S_LEARNED 1  /* the trained surrogate network (Sec. II-C), BF16 tensor cores */
#define DFP2S_P2S_LEARNED_FP32 2 /* the same network in FP32 on CUDA cores (check mode) */

#define DFP2S_FACTOR_FACTORED 0 /* sqrt(lambda_j(f)) per mode, then mixing by L (Sec. III-C) */
#define DFP2S_FACTOR_DENSE 1    /* FACTORED, plus the per-frequency J x J symmetric root F(f) of
                                   S~(f) = L diag(lambda(f)) L^T (Sec. III-A's eigen-root form per frequency:
                                   FP64 Jacobi eigendecomposition on the device, eigenvalues clamped at 0,
                                   stored FP32; J <= 48, else DFP2S_EUNSUPPORTED): the sampler
                                   dfp2s_sample_zernike_fields_dense.  FACTORED applies the other J x J root
                                   L diag(sqrt(lambda(f))) of the same density (same covariance, other
                                   samples) */
#define DFP2S_FACTOR_FULL 2     /* FACTORED, plus the tables of the exact sampler of the full cross-spectral
                                   density (Sec. III-B, no approximation): dfp2s_sample_zernike_fields_full */

#define DFP2S_KS 33       /* PSF / basis support is 33 x 33 pixels */
#define DFP2S_MAX_J 64    /* at most 64 Zernike fields (Noll 2..65) */
#define DFP2S_MAX_K 128   /* at most 128 basis PSFs */

/* Copies the message of the calling thread's last failure (NUL-terminated,
 * truncated to n bytes).  Returns the status of that failure (0 if none). */
int dfp2s_last_error(char* buf, size_t n);

/* Library build description (sm target, version); static string. */
const char* dfp2s_version(void);

/* N = next power of two >= max(H, W) + 4 pix_per_D: the FFT grid side for an
 * H x W frame; a margin of 4 aperture diameters keeps the periodic wrap-around
 * of the Fourier sampler (Sec. III-A) beyond the range s > 4 where the paper
 * finds the cross-correlations vanished (Sec. III-D).  Returns N, or
 * DFP2S_EINVAL for sizes outside 1..4096 or pix_per_D outside (0, 64]. */
int dfp2s_grid_size(int H, int W, double pix_per_D);

/* ---------------------------------------------------------- spectral factor
 * Built once per (J, N, pix_per_D, kind) on the device (FP64 arithmetic) and
 * reused for every frame and every D/r0: the spectra are normalised so that
 * each field has unit variance (Sec. III-C step 1), and D/r0 only scales the
 * mixing matrix L by (D/r0)^{5/6}.
 *   lambda_j(f) follows the path-integrated point-source model of the
 *   auto-correlation A_jj(s) (the paper defers its form to its reference
 *   [Chimitt 2020]); L is the lower Cholesky factor of Noll's matrix A_0
 *   (Eq. A matrix at s = 0, Fig. rand_gen). */
typedef struct dfp2s_factor dfp2s_factor;

typedef struct {
  int J;            /* number of fields, Noll modes 2..J+1; 3 <= J <= DFP2S_MAX_J */
  int N;            /* FFT grid side, power of two, 16 <= N <= 4096 */
  double pix_per_D; /* image pixels per aperture diameter of displacement s */
  int kind;         /* DFP2S_FACTOR_FACTORED, DFP2S_FACTOR_DENSE or DFP2S_FACTOR_FULL */
  int subharmonic_levels; /* 0 (the paper's sampler) .. 12: subharmonic levels of the factored sampler
                       (Sec. IV-B: the low-frequency deficit of the FFT method).  The DC cell of the
                       torus is split into 3 x 3 sub-cells of side df/3 (df = pix_per_D / N), the eight
                       outer ones represented by their centres f = (n, m) df/3 with weight 1/9 of a
                       bin, the centre split again, for `levels` levels; the per-mode normalisation to
                       unit variance covers bins and subharmonics together.  Each level adds to every
                       unit field sum_d Re[(g_re + i g_im) s_{j,p,d} e^{2 pi i (n x + m y) / (N 3^p)}]
                       (pixel (y, x); Gaussians from Philox tag 6, subsequence mode j, counter
                       4 (p - 1) + k for directions 2k, 2k + 1 of (n, m) = (-1,-1), (0,-1), (1,-1),
                       (-1,0), (1,0), (-1,1), (0,1), (1,1)).  Only with DFP2S_FACTOR_FACTORED
                       (else DFP2S_EUNSUPPORTED). */
} dfp2s_factor_params;

/* Builds the factor (allocates device memory, synchronises `stream` before
 * returning).  *out receives the handle.  Errors: EINVAL (params), ENOMEM,
 * ECUDA. */
int dfp2s_build_spectral_factor(const dfp2s_factor_params* params, dfp2s_factor** out, void* stream);
int dfp2s_factor_destroy(dfp2s_factor* f);
/* Copies the per-mode spectral multiplier sqrt(lambda_j(ky, kx)) / N^2
 * (float32, layout J x (N/2+1) x N, kx-major: [j][kx][ky]) to dst_dev. */
int dfp2s_factor_copy_multiplier(const dfp2s_factor* f, float* dst_dev, void* stream);
/* Copies L (J x J, row-major, FP64, D/r0 = 1) to dst_host (synchronous). */
int dfp2s_factor_copy_cholesky(const dfp2s_factor* f, double* dst_host);
/* Bytes of device scratch the factor holds for one frame's FFTs. */
int dfp2s_factor_info(const dfp2s_factor* f, int* J, int* N, size_t* scratch_bytes);

/* Sec. III-C: draws the J x H x W fields a of frame `frame` of stream `seed`
 * at strength D/r0 into fields_dev (device, J*H*W floats, caller-owned).
 * The white noise is drawn in the Fourier domain (its distribution is that of
 * FFT2 of real white noise, Sec. III-A): for mode j, Philox-4x32-10 with
 * key = seed, subsequence (0 << 40) | (frame << 8) | j, FP32 Box-Muller, gives
 * rows kx = 0 .. N/2 of 2N Gaussians, (Re, Im) of E(kx, ky) at 2 ky, 2 ky + 1
 * (counter (kx N + ky)/2 for ky even), scaled by N / sqrt 2; columns kx = 0 and
 * N/2 are completed to Hermitian symmetry in ky (their bins ky = 0 and N/2 real,
 * scaled by N).  Requires H, W <= factor N (crop of the periodic N x N field)
 * and uses the factor's scratch.  Errors: EINVAL, ECUDA. */
int dfp2s_sample_zernike_fields(const dfp2s_factor* f, double D_over_r0, uint64_t seed, uint32_t frame,
                                int H, int W, float* fields_dev, void* stream);

/* The dense-root form of the sampler (Sec. III-A per frequency, Eq. A tilde):
 * E(f) = F(f) xi(f), F the symmetric root of L diag(lambda(f)) L^T, xi the
 * Fourier-domain noise of dfp2s_sample_zernike_fields (the same Philox
 * streams), then the inverse FFT per mode, times (D/r0)^{5/6}.  Same
 * covariance as the factored form, other samples; the fields come out mixed.
 * Needs a DFP2S_FACTOR_DENSE factor (else EINVAL); uses its scratch and the
 * J^2 (N/2+1) N floats of F (read once per frame).  Errors: EINVAL, ECUDA. */
int dfp2s_sample_zernike_fields_dense(const dfp2s_factor* f, double D_over_r0, uint64_t seed, uint32_t frame,
                                      int H, int W, float* fields_dev, void* stream);
/* Copies F (float32, [j * J + i][kx * N + ky], kx = 0..N/2, D/r0 = 1) of a
 * DFP2S_FACTOR_DENSE factor to dst_dev.  Errors: EINVAL, ECUDA. */
int dfp2s_factor_copy_dense_root(const dfp2s_factor* f, float* dst_dev, void* stream);

/* The exact sampler (Sec. III-B): fields whose every auto- and cross-covariance
 * at every displacement is the full homogeneous tensor A (the slices A_{i,j}(s)
 * of Sec. III-B, not the approximation of Eq. A tilde), at strength D/r0.
 * Under the path-integrated model the angular part of Q_i(u) conj Q_j(u)
 * leaves the path integral, so the J x J cross-spectral density is
 * S(k) = D(k) P Gamma(|f_k|) P^T D(k)^H with D = diag(c_j sqrt(n_j+1) Theta_j(phi_k)),
 * P the J x R indicator of each mode's radial order (R distinct orders: 5 for
 * J = 15, 8 for J = 36) and Gamma the R x R matrix of the radial spectra
 * G_{n n'}(|f|); its root D P chol(Gamma) needs R complex Gaussians per
 * frequency instead of J.  Noise: Philox-4x32-10, key = seed, subsequence
 * (5 << 40) | (frame << 8) | r for stream r, the element layout of
 * dfp2s_sample_zernike_fields (rows kx = 0 .. N/2 of 2N Gaussians, (Re, Im) of
 * bin ky at 2 ky, 2 ky + 1); streams R .. 2R-1 feed the second half of the root
 * on the lines kx = N/2 and ky = N/2, where index N/2 is the frequency -N/2 for
 * k and -k alike.  The fields are complete: no mixing follows.  Needs a factor
 * built with DFP2S_FACTOR_FULL (else EINVAL); uses the factor's scratch.
 * Errors: EINVAL, ECUDA. */
int dfp2s_sample_zernike_fields_full(const dfp2s_factor* f, double D_over_r0, uint64_t seed, uint32_t frame,
                                     int H, int W, float* fields_dev, void* stream);

/* Temporally correlated fields (Sec. III, spatio-temporally correlated
 * fields: the paper enforces the temporal correlation with an auto-regressive
 * process).  Reading: the white noise of every mode follows
 * e_t = alpha e_{t-1} + sqrt(1 - alpha^2) n_t, n_t the noise of frame t; the
 * sampler is linear and time-invariant, so for a fixed D/r0 this is
 *   fields_dev = alpha * prev_dev + sqrt(1 - alpha^2) * (the fields of `frame`),
 * which is what the call computes.  prev_dev (J x H x W, the previous output)
 * may be NULL for the first frame; it must not alias fields_dev.
 * 0 <= alpha < 1.  Errors: EINVAL, ECUDA. */
int dfp2s_sample_zernike_fields_ar1(const dfp2s_factor* f, double D_over_r0, uint64_t seed, uint32_t frame,
                                    double alpha, int H, int W, const float* prev_dev, float* fields_dev,
                                    void* stream);

/* Same result as dfp2s_sample_zernike_fields, for callers that cannot
 * allocate device memory while they draw frames (a fixed memory plan made at
 * start-up, a plug-in whose host framework owns the device allocator, a
 * latency-bound loop in which an allocation may synchronise the device or
 * fail).  This call allocates nothing: the FFT scratch is a statically sized
 * device array inside the library, DFP2S_NOALLOC_SCRATCH_BYTES (48 MiB) on
 * every GPU that loads the library, held until the process exits.  The paper
 * has no counterpart; this is a deployment variant of the same computation.
 *   - Requires J (N/2+1) N * 8 <= DFP2S_NOALLOC_SCRATCH_BYTES (e.g. N = 512
 *     with J <= 47, N = 256 with J <= 64); larger factors get DFP2S_EINVAL.
 *   - The factor must live on the current device (DFP2S_EINVAL otherwise).
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress with that device current); make that first call
 *     before any stream capture begins.
 *   - Every call on a device shares the one array, and it keeps the previous
 *     call's contents (nothing in it needs clearing: each call writes all it
 *     reads).  Calls whose work overlaps on the GPU (different streams, or
 *     different host threads without ordering) race on the array: order them. */
#define DFP2S_NOALLOC_SCRATCH_BYTES (48u * 1024u * 1024u)
int dfp2s_sample_zernike_fields_noalloc(const dfp2s_factor* f, double D_over_r0, uint64_t seed, uint32_t frame,
                                        int H, int W, float* fields_dev, void* stream);

/* Debug/verification: the FP32 Gaussians of one (seed, tag, frame, mode) stream
 * as rows x cols (cols % 4 == 0), into out_dev.  With tag 0, rows = N/2 + 1 and
 * cols = 2N these are the values the field sampler generates in registers. */
int dfp2s_gaussian_noise(uint64_t seed, uint32_t tag, uint32_t frame, uint32_t mode, int rows, int cols,
                         float* out_dev, void* stream);
/* Debug/verification: n raw Philox words, 4 per counter q = q0 .. q0+n/4-1 of
 * subsequence `sub` (n % 4 == 0), into out_dev. */
int dfp2s_philox_words(uint64_t seed, uint64_t sub, uint64_t q0, int n, uint32_t* out_dev, void* stream);

/* Verification tap for the failure path of the tensor-core kernels (their
 * waits on mbarriers are bounded: a wait that runs out sets the kernel's error
 * word, the kernel still lets its own bulk copies land and releases its tensor
 * memory, and the host reads DFP2S_ETIMEOUT, e.g. from dfp2s_p2s_check).  One
 * kernel takes those steps on a barrier that nothing completes: allocates tensor
 * memory, starts a bulk copy, waits until limit_ns runs out, lets the copy land
 * (bounded by 2 s) and releases the tensor memory.  Returns DFP2S_ETIMEOUT, the
 * expected outcome; DFP2S_ECUDA if the wait did not run out or the copy did not
 * land; DFP2S_EINVAL for limit_ns outside [1 us, 1 s].  Synchronous. */
int dfp2s_check_bounded_wait(uint64_t limit_ns, void* stream);

/* Test hook for the allocation-failure paths: the n-th next device allocation
 * made by the library (1 = the next one; 0 disarms) reports
 * cudaErrorMemoryAllocation without allocating, so that the entry point returns
 * DFP2S_ENOMEM.  Process-wide.  Errors: EINVAL (n < 0). */
int dfp2s_debug_fail_allocation(int n);

/* -------------------------------------------------------- phase-to-space
 * A P2S handle holds the PSF basis phi_k (K x 33 x 33, Sec. II-C Eq. p2s PSF)
 * and, optionally, the surrogate network. */
typedef struct dfp2s_p2s dfp2s_p2s;

/* Creates a handle for J fields and K basis PSFs; copies basis_dev
 * (K x 33 x 33 float32, device).  Errors: EINVAL, ENOMEM. */
int dfp2s_p2s_create(int J, int K, const float* basis_dev, dfp2s_p2s** out);
int dfp2s_p2s_destroy(dfp2s_p2s* p);
/* Reads (synchronously) and clears the handle's device error word: returns
 * DFP2S_ETIMEOUT if a tensor-core kernel launched with this handle gave up on
 * a bounded barrier wait (its output is then invalid), DFP2S_OK otherwise. */
int dfp2s_p2s_check(dfp2s_p2s* p);

/* Sec. II-C (PSF database -> basis; reading: uncentred SVD): draws n_psf
 * Zernike vectors a ~ N(0, A_0(D/r0)) with Philox tag 1 (D/r0 =
 * D_over_r0[i % n_dr] for draw i, tilts zeroed), forms their exact 33 x 33 PSFs
 * and writes the top-K right singular vectors of the n_psf x 1089 PSF matrix
 * (FP64 one-sided Jacobi on the device) to basis_dev (K x 33 x 33 float32),
 * each signed so that its largest-magnitude entry is positive.  sigma_host
 * (optional, 1089 doubles) receives all singular values in descending order;
 * sweeps_host (optional) the Jacobi sweeps used.  Synchronous.
 * Errors: EINVAL, ENOMEM, ECUDA. */
int dfp2s_build_basis(const dfp2s_factor* f, int K, int n_psf, const double* D_over_r0, int n_dr, uint64_t seed,
                      float* basis_dev, double* sigma_host, int* sweeps_host, void* stream);

/* Installs surrogate-network weights (all device float32, copied):
 * W1 256 x J, b1 256, W2 256 x 256, b2 256, W3 K x 256, b3 K; in_scale J
 * (multiplies the Zernike vector before the first layer; 0 on the tilt
 * fields); out_scale, out_shift K (v = y * out_scale + out_shift; the P2S
 * weights are v moved onto unit flux, see dfp2s_p2s_weights). */
int dfp2s_p2s_set_mlp(dfp2s_p2s* p, const float* W1, const float* b1, const float* W2, const float* b2,
                      const float* W3, const float* b3, const float* in_scale, const float* out_scale,
                      const float* out_shift);

/* Surrogate training on the device.  Draws n_pairs Zernike vectors
 * a ~ N(0, A_0(D/r0)) (Philox tag 2, D/r0 cycling over D_over_r0[0..n_dr),
 * tilt fields zeroed), computes their exact P2S weights with the same kernel as
 * dfp2s_p2s_weights(EXACT), standardises inputs and targets, trains
 * J -> 256 -> 256 -> K (GELU, erf form) with Adam on a one-cycle schedule
 * (FP32; one step is a captured CUDA graph), and installs the network in `p`
 * (as dfp2s_p2s_set_mlp would).  The last val_fraction of the pairs is held out:
 * report_host[1] receives the relative L2 error of the network's weights on
 * them, report_host[0] the final training loss, report_host[2] the steps run.
 * params_out_host (optional) receives the flat FP32 parameters
 * [W1 (256 x J), b1, W2 (256 x 256), b2, W3 (K x 256), b3] before the
 * standardisation is folded in.  Synchronous.  Errors: EINVAL, ENOMEM, ECUDA. */
typedef struct {
  int n_pairs;            /* training + validation pairs, >= 1024 */
  int n_dr;               /* 1..8 */
  double D_over_r0[8];    /* turbulence strengths, pooled evenly */
  uint64_t seed;          /* Philox key for the data, the batches and the initial weights */
  int batch;              /* 64..8192 */
  int steps;              /* Adam steps */
  float lr;               /* peak learning rate */
  int psf_weighted_loss;  /* 1: per-k loss weight = variance of w_k / mean variance (error of the PSF);
                             0: plain MSE of the standardised weights (both only if image_prior_loss = 0) */
  float val_fraction;     /* 0 <= val_fraction < 0.5 */
  int image_prior_loss;   /* 1: loss r^T G r / K per pair, G = dfp2s_mlp_image_prior_gram of the targets'
                             standard deviations (the expected error of the blurred image); 0: per-k weights */
} dfp2s_mlp_train_params;
int dfp2s_mlp_train(dfp2s_p2s* p, const dfp2s_factor* f, const dfp2s_mlp_train_params* tp, float* report_host,
                    float* params_out_host, void* stream);
/* Network files: the installed network, as dfp2s_p2s_set_mlp takes it, to a
 * host file and back.  Format: the 8 bytes "DFP2SMLP", uint32 version 1,
 * int32 J, int32 K, then W1 (256 x J), b1 (256), W2 (256 x 256), b2 (256),
 * W3 (K x 256), b3 (K), in_scale (J), out_scale (K), out_shift (K) as
 * little-endian float32, nothing after.  _save: EINVAL without an installed
 * network or when the file cannot be written; _load: EINVAL when the file
 * cannot be read or is not a network for this handle's J and K, then as
 * dfp2s_p2s_set_mlp.  Synchronous.  Errors: EINVAL, ECUDA. */
int dfp2s_mlp_save(const dfp2s_p2s* p, const char* path);
int dfp2s_mlp_load(dfp2s_p2s* p, const char* path);
/* Number of FP32 parameters of the J -> 256 -> 256 -> K network. */
int dfp2s_mlp_param_count(int J, int K);
/* One forward/backward pass on a given batch (for gradient checks): X (B x J)
 * network inputs, T (B x K) targets, params flat as above; the loss is
 * sum_b r_b^T G r_b / (B K), r = y - t, if G_dev (K x K, symmetric) is given,
 * else sum_k lw_k r_k^2 / (B K) with lw_dev (K).  Writes grads (flat, same
 * layout) and loss.  All device pointers.  Synchronous. */
int dfp2s_mlp_loss_grad(int J, int K, int B, const float* params_dev, const float* X_dev, const float* T_dev,
                        const float* lw_dev, const float* G_dev, float* grads_dev, float* loss_dev, void* stream);
/* The training loss's quadratic form for this handle's basis (reading of the
 * training objective, Sec. II-C): G_kl = sum_f S(f) Re(Phi_k(f) conj Phi_l(f)),
 * Phi_k the 64 x 64 DFT of basis function k (33 x 33 at the origin),
 * S(f) = 1 / (fx^2 + fy^2 + 1) for integer frequencies in [-32, 32) -- the
 * expected energy a weight error puts into the blurred image of Eq. (varying
 * blur) for images with that power spectrum -- then G^ = diag(sd) G diag(sd)
 * scaled to a unit mean diagonal.  sd_dev (K): standard deviations of the
 * weights; writes G_dev (K x K float32).  FP64 on the device.  Synchronous.
 * Errors: EINVAL, ENOMEM, ECUDA. */
int dfp2s_mlp_image_prior_gram(const dfp2s_p2s* p, const float* sd_dev, float* G_dev, void* stream);

/* Sec. II-C: per-pixel basis weights from the fields (J x H x W, device).
 * Every form returns weights whose PSF keeps the unit sum of the true PSF:
 * with s_k = sum_u phi_k(u), s^T w = 1 (the least-squares projection of
 * Eq. p2s PSF under that constraint; without it the projected PSF keeps only
 * the part of the flux inside the basis span, and a flat image region changes
 * brightness by 1 - s^T w).
 *   EXACT: PSF h of Eq. (2) from modes Noll 4..J+1 on a 64 x 64 pupil grid
 *          (aperture 32 samples across, P = 1 inside), |DFT|^2, 33 x 33 centre,
 *          unit sum, then w = Phi^T h + s (1 - s^T Phi^T h) / (s^T s), the
 *          nearest weights to h's projection with unit flux;
 *   LEARNED: v = MLP(a * in_scale) * out_scale + out_shift on the tcgen05
 *          tensor cores (BF16 inputs, weights and hidden activations, FP32
 *          accumulation), one fused kernel, then in FP32
 *          w = v + s (1 - s^T v) / (s^T s); J <= 48, K <= 128;
 *   LEARNED_FP32: the same network and projection in FP32 on CUDA cores.
 * Writes w_dev (H x W x K, dtype w_dtype).  Errors: EINVAL (no MLP for
 * LEARNED, J > 48 for LEARNED, sizes), ECUDA. */
int dfp2s_p2s_weights(const dfp2s_p2s* p, int mode, const float* fields_dev, int H, int W, void* w_dev,
                      int w_dtype, void* stream);

/* Tilt warp (Eq. 2's linear phase as a shift, reading of Sec. II-C):
 * out(c, y, x) = bilinear(img_c; x + (4/pi) a2(y,x), y + (4/pi) a3(y,x)),
 * clamp to edge.  a2/a3 are H x W (fields 0 and 1).  img, out: C x H x W.
 * out must not alias img.  Errors: EINVAL, ECUDA. */
int dfp2s_tilt_warp(const float* img_dev, int C, int H, int W, const float* a2_dev, const float* a3_dev,
                    float* out_dev, void* stream);

/* Eq. (varying blur): out_c(x) = sum_k w_k(x) sum_u phi_k(u) img_c(x - u),
 * u in [-16, 16]^2, clamp-to-edge borders.  w_dtype F32: FP32 arithmetic;
 * BF16: image and basis rounded to bfloat16, tensor-core products with FP32
 * accumulation (dfp2s_basis_blur_tc).  Errors: EINVAL, ECUDA. */
int dfp2s_basis_blur(const dfp2s_p2s* p, const float* img_dev, int C, int H, int W, const void* w_dev,
                     int w_dtype, float* out_dev, void* stream);

/* Eq. (varying blur) on the tcgen05 tensor cores: the image enters as
 * bfloat16(I - 0.5) (the constant 0.5 * sum_u phi_k(u) is added back in FP32),
 * the basis as bfloat16, products accumulate in FP32 in tensor memory, and the
 * weights (FP32 or BF16 as stored) are applied in FP32.  Requires K <= 128.
 * Errors: EINVAL, EUNSUPPORTED, ENOMEM (scratch), ECUDA.  A device-side barrier
 * timeout is reported by dfp2s_p2s_check. */
int dfp2s_basis_blur_tc(const dfp2s_p2s* p, const float* img_dev, int C, int H, int W, const void* w_dev,
                        int w_dtype, float* out_dev, void* stream);

/* dfp2s_basis_blur_tc in its two steps, for callers that time or overlap
 * them separately.  _prepare writes the image's BF16 operand (eight copies of
 * bfloat16(I - 0.5), edge-padded by 16 and shifted by 0..7 columns, so that
 * the tensor-core operand tiles of Eq. (varying blur) are 16-byte aligned
 * runs) into scratch owned by the handle; _run contracts the prepared image
 * with the basis and the weights w_dev.  A handle holds one prepared image:
 * issue _prepare and then _run, with the same C, H, W, on one stream; _run on
 * a handle without a prepared image of that shape returns EINVAL.
 * dfp2s_basis_blur_tc(...) is _prepare followed by _run.
 * Errors: EINVAL, EUNSUPPORTED (K > 128), ENOMEM (scratch), ECUDA. */
int dfp2s_basis_blur_tc_prepare(const dfp2s_p2s* p, const float* img_dev, int C, int H, int W, void* stream);
/* dfp2s_tilt_warp (Eq. 2's linear phase as a shift) fused with
 * dfp2s_basis_blur_tc_prepare: prepares the blur operand of the tilt-warped
 * image, bit for bit the one _prepare makes from dfp2s_tilt_warp's output,
 * without writing the FP32 warped image.  a2/a3: H x W tilt fields.  Follow
 * it with dfp2s_basis_blur_tc_run.  Errors as _prepare. */
int dfp2s_tilt_warp_blur_tc_prepare(const dfp2s_p2s* p, const float* img_dev, int C, int H, int W,
                                    const float* a2_dev, const float* a3_dev, void* stream);
int dfp2s_basis_blur_tc_run(const dfp2s_p2s* p, int C, int H, int W, const void* w_dev, int w_dtype, float* out_dev,
                            void* stream);

/* ------------------------------------------------------------ statistics
 * Lagged covariances of J x H x W fields (Sec. III-D: the sampled fields'
 * covariance at separation s is A~(s) of Eq. (A tilde), A_0 at s = 0):
 *   out[l][i][j] = (1/n_l) sum over x with x + d_l inside the frame of
 *                  a_i(x) a_j(x + d_l),   d_l = (lags[2l], lags[2l+1]) = (dy, dx),
 *   n_l = (H - |dy|)(W - |dx|).
 * fields_dev: J x H x W float32 (device); lags_host: 2 n_lags ints (host);
 * out_dev: n_lags x J x J doubles (device, row-major).  Products, runs of 32
 * pixels and each block's compensated (Kahan) sum of its runs in FP32, the
 * blocks' partials in FP64, all in a fixed order (the result does not depend on
 * the launch).  1 <= J <= 64, 1 <= n_lags <= 64, |dy| < H,
 * |dx| < W.  Errors: EINVAL, ENOMEM, ECUDA. */
int dfp2s_field_covariance(const float* fields_dev, int J, int H, int W, const int* lags_host, int n_lags,
                           double* out_dev, void* stream);

/* Sec. IV-B, aperture statistics of sampled fields: the structure function
 * of the pupil phase (to compare with 6.88 (r/r0)^{5/3}, Eq. fried_struct)
 * and the long- and short-exposure OTFs (Eqs. H_LE, H_SE).  The realisations
 * are the Zernike vectors (all J fields, Noll 2..J+1) of the pixels on the
 * sub-grid y = 0, step, 2 step, ..., x likewise; each gives the phase
 * phi = sum_j a_j Z_j on the 64 x 64 pupil grid of the exact P2S (coordinates
 * (i - 32)/16, aperture rho <= 1).
 * out_dev (device, caller-owned), FP64:
 *   [0, 33)     D_x(d), d = 0..32 samples (r = d/32 aperture diameters): the mean
 *               over realisations and aperture pairs (i, k), (i, k + d) of
 *               (phi(i, k) - phi(i, k + d))^2; [33, 66) D_y likewise along rows;
 *   [66, 66 + 4096)         H_LE[nu_y][nu_x] (FFT order, nu/32 diameters): Re
 *               of the inverse DFT of the mean |DFT(P e^{-j phi})|^2, divided
 *               by its value at nu = 0;
 *   [66 + 4096, 66 + 8192)  H_SE: the same with phi minus its least-squares
 *               plane c0 + c1 x + c2 y over the aperture samples.
 * 2 <= J <= DFP2S_MAX_J, step >= 1.  Errors: EINVAL, ENOMEM (scratch), ECUDA. */
#define DFP2S_SF_LAGS 33
#define DFP2S_OTF_N 64
int dfp2s_aperture_statistics(const float* fields_dev, int J, int H, int W, int step, double* out_dev,
                              void* stream);

/* Sec. IV-B, spatial statistics: the tilt correlation and the differential
 * tilt variance of the two tilt fields (the first two H x W planes of
 * fields_dev: Noll 2, then Noll 3) at pixel lags d = 0..max_lag along x
 * (dir 0) and along y (dir 1).  out_dev (FP64) [dir][d][8] holds the means
 * over the pixel pairs (p, p + d) inside the frame of
 *   a2(p) a2(p+d), a3(p) a3(p+d), (a2(p) - a2(p+d))^2, (a3(p) - a3(p+d))^2,
 *   a2(p)^2, a2(p+d)^2, a3(p)^2, a3(p+d)^2,
 * so that the paper's identity DTV = 2 (E[alpha^2] - E[alpha(0) alpha(d)])
 * reads DTV = var(p) + var(p + d) - 2 corr for these window means.
 * 0 <= max_lag < min(H, W), max_lag <= 1024.  Errors: EINVAL, ENOMEM, ECUDA. */
int dfp2s_tilt_statistics(const float* fields_dev, int H, int W, int max_lag, double* out_dev, void* stream);

/* Which field sampler a context's frames use: the factored form of Sec. III-C
 * (the default), the dense per-frequency root (needs a DFP2S_FACTOR_DENSE
 * factor) or the full cross-spectral density without the approximation
 * (needs DFP2S_FACTOR_FULL).  The last two give mixed fields: exact frames
 * skip the mixing pass, learned frames feed the network's own first layer
 * W1 diag(in_scale) and warp by the fields' tilt rows.  Errors: EINVAL. */
#define DFP2S_FIELDS_FACTORED 0
#define DFP2S_FIELDS_DENSE 1
#define DFP2S_FIELDS_FULL 2

/* ---------------------------------------------------------------- frames
 * A context binds a factor and a P2S handle and owns the per-frame scratch
 * (fields, warped image, weights) for frames up to max_C x max_H x max_W. */
typedef struct dfp2s_ctx dfp2s_ctx;
int dfp2s_ctx_create(const dfp2s_factor* f, const dfp2s_p2s* p, int max_C, int max_H, int max_W,
                     dfp2s_ctx** out);
int dfp2s_ctx_destroy(dfp2s_ctx* c);
int dfp2s_ctx_set_field_sampler(dfp2s_ctx* c, int sampler);
/* The factored sampler's column-pass kernel for this context's frames (the
 * batch engine's autotuner sets it per shape class): 0 one FFT group per
 * column at the compiler's register budget, 1 three CTAs per SM (at most 80
 * registers; N <= 2048), -1 the default (1 at N = 1024, else 0).  Same fields
 * bit for bit.  Errors: EINVAL. */
int dfp2s_ctx_set_field_variant(dfp2s_ctx* c, int variant);

/* Fig. dfp2s: one frame.  fields (Sec. III-C) -> tilt warp -> P2S weights
 * (FP32) -> blur (p2s_mode EXACT: FP32 CUDA-core blur; LEARNED: the network's
 * weights and the BF16 tensor-core blur, with the warp fused into the blur's
 * operand, dfp2s_tilt_warp_blur_tc_prepare + dfp2s_basis_blur_tc_run) -> out
 * (C x H x W, device).  LEARNED frames skip the pixel-wise mixing pass: the
 * mixing a = (D/r0)^(5/6) L u is linear, so the warp forms the two tilt rows of
 * a from the unit fields u0, u1 (bit for bit as the mixing pass would) and the
 * network's first layer takes W1 diag(in_scale) L (packed once per installed
 * network) on the scaled unit fields.
 * Errors: EINVAL, ECUDA. */
int dfp2s_simulate_frame(dfp2s_ctx* c, const float* img_dev, int C, int H, int W, double D_over_r0,
                         uint64_t seed, uint32_t frame, int p2s_mode, float* out_dev, void* stream);
/* Device pointers of the context's last fields / warped image / weights
 * (valid until the next call on the context; LEARNED frames do not write the
 * FP32 warped image, and leave the unit fields u before the mixing by
 * (D/r0)^(5/6) L in fields_dev). */
int dfp2s_ctx_buffers(const dfp2s_ctx* c, float** fields_dev, float** warped_dev, void** w_dev);
/* Stage timing of dfp2s_simulate_frame.  n > 0: from now on every frame
 * records five CUDA events on its stream (start, after the fields, after the
 * warp, after the P2S weights, after the blur) into a ring of n frames; n = 0
 * turns it off.  The context owns the events.  Errors: EINVAL, ECUDA. */
int dfp2s_ctx_stage_timing(dfp2s_ctx* c, int n);
/* Stage durations in ms of the last `count` recorded frames, oldest first:
 * out_host[4 i + s] for stage s (fields, warp, P2S weights, blur) of frame i.
 * Waits for those frames.  count <= n and <= the frames recorded since
 * dfp2s_ctx_stage_timing.  Errors: EINVAL, ECUDA. */
int dfp2s_ctx_stage_times(dfp2s_ctx* c, int count, float* out_host);

/* ------------------------------------------------------- batched requests
 * The serving pattern: many requests of mixed image size, J, D/r0 and P2S
 * form, each with several frames (frame numbers first_frame .. first_frame +
 * n_frames - 1 of Philox stream `seed`, so every frame is independent), run
 * by one call.  An engine holds the P2S handles (one per J; not owned) and
 * builds, the first time a shape class (J, C, H, W) appears, its spectral
 * factor (shared by the classes of equal J and grid N) and its frame context.
 *   DFP2S_ENGINE_AUTOTUNE: on a class's first use its field column-pass
 *     kernels are timed on its own frames (CUDA events) and the faster kept
 *     (dfp2s_engine_class_info reports the choice and the times);
 *   DFP2S_ENGINE_GRAPHS: the frames of each class are captured into one CUDA
 *     graph per run and launched once; a class's graph is updated in place
 *     when the next run gives it the same number of frames.
 * Each frame is what dfp2s_simulate_frame gives for the request's arguments
 * (bit for bit: the same kernels, whichever column-pass kernel is chosen). */
typedef struct dfp2s_engine dfp2s_engine;
typedef struct {
  const float* img_dev;  /* C x H x W float32, device */
  int C, H, W;           /* 1 <= C <= 64, 1 <= H, W <= 4096 */
  int J;                 /* fields; the engine holds a P2S handle with this J */
  double D_over_r0;
  uint64_t seed;
  uint32_t first_frame;
  int n_frames;          /* >= 0 */
  int p2s_mode;          /* DFP2S_P2S_EXACT, _LEARNED, _LEARNED_FP32 (a network installed for the last two) */
  float* out_dev;        /* n_frames x C x H x W float32, device */
} dfp2s_request;
#define DFP2S_ENGINE_GRAPHS 1
#define DFP2S_ENGINE_AUTOTUNE 2
/* p2s: n_p2s handles with distinct J (1..16).  Errors: EINVAL, ECUDA. */
int dfp2s_engine_create(const dfp2s_p2s* const* p2s, int n_p2s, double pix_per_D, int flags, dfp2s_engine** out);
/* Enqueues every frame of the n_req requests (stream-ordered after the work
 * already on `stream`, and `stream` waits for them).  New classes are built
 * and warmed (and tuned) synchronously first.  Calls on one engine must not
 * overlap.  Errors: EINVAL (request arguments), ENOMEM, ECUDA. */
int dfp2s_engine_run(dfp2s_engine* e, const dfp2s_request* req, int n_req, void* stream);
/* n_classes (optional); counters_host (optional, 4): frames run, graph launches,
 * graph instantiations, graph updates. */
int dfp2s_engine_info(const dfp2s_engine* e, int* n_classes, long long* counters_host);
/* Class i: shape_host (6 ints) = J, C, H, W, N, column-pass kernel in use
 * (0 or 1; -1 before tuning); tuned_ms_host (2 floats) = ms per frame of each
 * candidate (-1 if not timed).  Errors: EINVAL. */
int dfp2s_engine_class_info(const dfp2s_engine* e, int i, int* shape_host, float* tuned_ms_host);
int dfp2s_engine_destroy(dfp2s_engine* e);

#ifdef __cplusplus
}
#endif
#endif /* DFP2S_H */
