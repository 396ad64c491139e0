// Spectral factor of the homogeneous approximation (Sec. III-C), built on the
// device in FP64.
//
//   A_0  Noll's covariance of modes 2..J+1 (Eq. A matrix at s = 0), closed form
//        K sqrt((n+1)(n'+1)) (-1)^((n+n'-2m)/2) Gamma((n+n'-5/3)/2) /
//        [Gamma((n-n'+17/3)/2) Gamma((n'-n+17/3)/2) Gamma((n+n'+23/3)/2)]
//        for equal m and equal angular function, K = c Gamma(14/3) 2^{-5/3}
//        pi^{8/3}, c = [(24/5)Gamma(6/5)]^{5/6} Gamma(11/6)^2 / (2 pi^{11/3})
//        (the coefficient of the Kolmogorov phase spectrum whose structure
//        function is 6.88 (r/r0)^{5/3}, Eq. fried_struct); L = chol(A_0).
//   lambda_j(f) the spectrum of the auto-correlation A_jj(s) under the
//        path-integrated point-source model: with u = f (1-t)/(2t) for a layer
//        at path fraction t,
//          P_j(f) = (n+1) Theta_j(phi) int_0^1 (1-t)^{5/3} ((1-t)/(2t))^2 u^{-11/3}
//                   [J_{n+1}(2 pi u)/(pi u)]^2 dt,
//        evaluated as G_n(f) = int_0^inf (2v/(2v+f))^{5/3} 2v^2/(f (2v+f)^2) g_n(v) dv,
//        g_n(v) = v^{-11/3} [J_{n+1}(2 pi v)/(pi v)]^2, with a composite
//        Gauss-Legendre rule (8-point panels log-spaced on [1e-7, 1], 16-point
//        panels of width 1/2 on [1, 48]).  Theta_j = 1 (m = 0), 2 cos^2(m phi)
//        (even j), 2 sin^2(m phi) (odd j).  lambda_j = N^2 P_j / sum_{k != 0} P_j
//        over the N x N torus (unit variance), lambda_j(0) = 0.
//   The stored multiplier is sqrt(lambda_j)/N^2, which also carries the 1/N^2
//   of the inverse FFT.
#include <cuda_runtime.h>
#include <math.h>

#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int kMaxOrders = 11;  // radial orders 1..10 cover Noll 2..65

DFP2S_DEV void noll_nm(int j, int* n, int* m) {
  int nn = 0;
  while ((nn + 1) * (nn + 2) / 2 < j) ++nn;
  const int r = j - nn * (nn + 1) / 2 - 1;
  *n = nn;
  *m = (nn % 2 == 0) ? 2 * ((r + 1) / 2) : 2 * (r / 2) + 1;
}

// A_0 (D/r0 = 1) and its lower Cholesky factor; one CTA.
__global__ void k_noll_chol(int J, double* __restrict__ L64, float* __restrict__ L32, int* __restrict__ err) {
  __shared__ double A[64 * 64];
  const double pi = 3.14159265358979323846;
  const double c = pow((24.0 / 5.0) * tgamma(6.0 / 5.0), 5.0 / 6.0) * tgamma(11.0 / 6.0) * tgamma(11.0 / 6.0) /
                   (2.0 * pow(pi, 11.0 / 3.0));
  const double K = c * tgamma(14.0 / 3.0) * pow(2.0, -5.0 / 3.0) * pow(pi, 8.0 / 3.0);
  for (int idx = threadIdx.x; idx < J * J; idx += blockDim.x) {
    const int a = idx / J, b = idx - a * J;
    const int i = a + 2, j = b + 2;
    int ni, mi, nj, mj;
    noll_nm(i, &ni, &mi);
    noll_nm(j, &nj, &mj);
    double v = 0.0;
    if (mi == mj && (mi == 0 || (i & 1) == (j & 1))) {
      const double sign = (((ni + nj - 2 * mi) / 2) & 1) ? -1.0 : 1.0;
      const double lg = lgamma((ni + nj - 5.0 / 3.0) / 2.0) - lgamma((ni - nj + 17.0 / 3.0) / 2.0) -
                        lgamma((nj - ni + 17.0 / 3.0) / 2.0) - lgamma((ni + nj + 23.0 / 3.0) / 2.0);
      v = K * sqrt((double)((ni + 1) * (nj + 1))) * sign * exp(lg);
    }
    A[idx] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // Cholesky-Banachiewicz, lower triangle in place
    for (int i = 0; i < J; ++i) {
      for (int j = 0; j <= i; ++j) {
        double s = A[i * J + j];
        for (int k = 0; k < j; ++k) s -= A[i * J + k] * A[j * J + k];
        if (i == j) {
          if (!(s > 0.0)) {
            *err = 1;
            s = 1e-300;
          }
          A[i * J + i] = sqrt(s);
        } else {
          A[i * J + j] = s / A[j * J + j];
        }
      }
      for (int j = i + 1; j < J; ++j) A[i * J + j] = 0.0;
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < J * J; idx += blockDim.x) {
    L64[idx] = A[idx];
    L32[idx] = (float)A[idx];
  }
}

// g_nn'(v_q) * w_q for every needed pair of radial orders (n, n') = (orders_a[p], orders_b[p]) (layout [q][p]);
// the per-mode spectra take the diagonal pairs.
__global__ void k_gtab(const double* __restrict__ v, const double* __restrict__ w, int Q, const int* __restrict__ orders_a,
                       const int* __restrict__ orders_b, int no, double* __restrict__ gtab) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Q * no) return;
  const int q = i / no, o = i - q * no;
  const double pi = 3.14159265358979323846;
  const double x = v[q];
  const double ja = jn(orders_a[o] + 1, 2.0 * pi * x);
  const double jb = orders_b[o] == orders_a[o] ? ja : jn(orders_b[o] + 1, 2.0 * pi * x);
  gtab[i] = w[q] * pow(x, -11.0 / 3.0) * ja * jb / (pi * pi * x * x);
}

// G_n(f) on the octant 0 <= b <= a <= N/2 of integer frequency pairs, index a(a+1)/2 + b, for the no <= kMaxOrders
// columns of gtab (row stride ld) that start at gtab[0].
__global__ void k_radial(const double* __restrict__ v, const double* __restrict__ gtab, int Q, int no, int ld, int N,
                         double fscale, double* __restrict__ G, int noct) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= noct) return;
  int a = (int)((sqrt(8.0 * i + 1.0) - 1.0) * 0.5);
  while (a * (a + 1) / 2 > i) --a;
  while ((a + 1) * (a + 2) / 2 <= i) ++a;
  const int b = i - a * (a + 1) / 2;
  const double f = sqrt((double)a * a + (double)b * b) * fscale;
  double acc[kMaxOrders];
#pragma unroll
  for (int o = 0; o < kMaxOrders; ++o) acc[o] = 0.0;
  if (f > 0.0) {
    for (int q = 0; q < Q; ++q) {
      const double x = v[q];
      const double d = 2.0 * x + f;
      const double K = exp((5.0 / 3.0) * log(2.0 * x / d)) * 2.0 * x * x / (f * d * d);
      const double* g = gtab + (size_t)q * ld;
#pragma unroll
      for (int o = 0; o < kMaxOrders; ++o)
        if (o < no) acc[o] = fma(K, g[o], acc[o]);
    }
  }
#pragma unroll
  for (int o = 0; o < kMaxOrders; ++o)
    if (o < no) G[(size_t)o * noct + i] = acc[o];
}

// G_n(f) at nf listed frequencies (the subharmonics), the same quadrature as k_radial; G[o * nf + i].
__global__ void k_radial_list(const double* __restrict__ v, const double* __restrict__ gtab, int Q, int no,
                              const double* __restrict__ flist, int nf, double* __restrict__ G) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nf) return;
  const double f = flist[i];
  double acc[kMaxOrders];
#pragma unroll
  for (int o = 0; o < kMaxOrders; ++o) acc[o] = 0.0;
  for (int q = 0; q < Q; ++q) {
    const double x = v[q];
    const double d = 2.0 * x + f;
    const double K = exp((5.0 / 3.0) * log(2.0 * x / d)) * 2.0 * x * x / (f * d * d);
    const double* g = gtab + (size_t)q * no;
#pragma unroll
    for (int o = 0; o < kMaxOrders; ++o)
      if (o < no) acc[o] = fma(K, g[o], acc[o]);
  }
#pragma unroll
  for (int o = 0; o < kMaxOrders; ++o)
    if (o < no) G[(size_t)o * nf + i] = acc[o];
}

struct ModeInfo {
  int n, m, odd, o;  // radial order, azimuthal frequency, sin (odd Noll index), order slot
};

// P_j at half-plane bin (kx, ky) (kx in [0, N/2], ky in [0, N) FFT order).
DFP2S_DEV double mode_power(const ModeInfo& mi, int kx, int ky, int N, const double* __restrict__ G, int noct) {
  const int sky = ky < N / 2 ? ky : ky - N;
  if (kx == 0 && sky == 0) return 0.0;
  const int ay = sky < 0 ? -sky : sky;
  const int a = kx > ay ? kx : ay, b = kx > ay ? ay : kx;
  const double g = G[(size_t)mi.o * noct + a * (a + 1) / 2 + b];
  double ang = 1.0;
  if (mi.m != 0) {
    const double phi = atan2((double)sky, (double)kx);
    double s, c;
    sincos(mi.m * phi, &s, &c);
    ang = mi.odd ? 2.0 * s * s : 2.0 * c * c;
  }
  return (mi.n + 1) * ang * g;
}

__global__ void k_lambda_sums(const ModeInfo* __restrict__ modes, int J, int N, const double* __restrict__ G, int noct,
                              double* __restrict__ sums) {
  __shared__ double part[64];
  for (int j = threadIdx.x; j < J; j += blockDim.x) part[j] = 0.0;
  __syncthreads();
  const int half = N / 2 + 1;
  const size_t total = (size_t)half * N;
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = i < total;
  const int kx = live ? (int)(i / N) : 0, ky = live ? (int)(i - (size_t)kx * N) : 0;
  const double wgt = (kx == 0 || kx == N / 2) ? 1.0 : 2.0;
  for (int j = 0; j < J; ++j) {
    double p = live ? wgt * mode_power(modes[j], kx, ky, N, G, noct) : 0.0;
    for (int off = 16; off > 0; off >>= 1) p += __shfl_down_sync(0xffffffffu, p, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(&part[j], p);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < J; j += blockDim.x) atomicAdd(&sums[j], part[j]);
}

// The subharmonic levels (Sec. IV-B): level p, direction d = (n, m) in {-1, 0, 1}^2 \ {0} (order (-1,-1),
// (0,-1), (1,-1), (-1,0), (1,0), (-1,1), (0,1), (1,1)) at f = (n, m) df / 3^p with weight 1/9^p of a bin; their
// power joins the per-mode sum of the bins (sums[j], so lambda is normalised over both), and the amplitudes are
// s_{j,p,d} = sqrt(P_j(f_{p,d}) / 9^p / sum_j).  Gl holds G_n at |f| = df/3^p (axis) and sqrt2 df/3^p (diagonal),
// [o][2 (p-1) + diagonal].  One thread per mode.
__global__ void k_sh_tables(const ModeInfo* __restrict__ modes, int J, int levels, const double* __restrict__ Gl,
                            double* __restrict__ sums, float* __restrict__ amp) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= J) return;
  const ModeInfo mi = modes[j];
  const int dn[8] = {-1, 0, 1, -1, 1, -1, 0, 1}, dm[8] = {-1, -1, -1, 0, 0, 1, 1, 1};
  double pw[12 * 8];
  double extra = 0.0, w = 1.0;
  for (int p = 0; p < levels; ++p) {
    w /= 9.0;
    for (int d = 0; d < 8; ++d) {
      const bool diag = dn[d] != 0 && dm[d] != 0;
      const double g = Gl[(size_t)mi.o * (2 * levels) + 2 * p + (diag ? 1 : 0)];
      double ang = 1.0;
      if (mi.m != 0) {
        const double phi = atan2((double)dm[d], (double)dn[d]);
        double sn, cs;
        sincos(mi.m * phi, &sn, &cs);
        ang = mi.odd ? 2.0 * sn * sn : 2.0 * cs * cs;
      }
      pw[p * 8 + d] = (mi.n + 1) * ang * g * w;
      extra += pw[p * 8 + d];
    }
  }
  const double total = sums[j] + extra;
  sums[j] = total;
  for (int e = 0; e < levels * 8; ++e) amp[(size_t)j * levels * 8 + e] = (float)sqrt(pw[e] / total);
}

__global__ void k_lambda_write(const ModeInfo* __restrict__ modes, int J, int N, const double* __restrict__ G, int noct,
                               const double* __restrict__ sums, float* __restrict__ mult) {
  const int half = N / 2 + 1;
  const size_t total = (size_t)half * N;
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int kx = (int)(i / N), ky = (int)(i - (size_t)kx * N);
  for (int j = 0; j < J; ++j) {
    const double p = mode_power(modes[j], kx, ky, N, G, noct);
    mult[(size_t)j * total + i] = (float)(sqrt(p / sums[j]) / N);
  }
}

// ---- the full cross-spectral sampler (Sec. III-B; reading R29)
// Per octant bin: Gamma_oo' = G_{n_o n_o'}(|f|) (pairs p(a, b) = a no - a(a-1)/2 + (b - a), a <= b), its lower
// Cholesky factor in FP64, stored in FP32 as C[bin][o(o+1)/2 + r], r <= o (rows padded to a multiple of 4).  Gamma is positive definite off DC (a
// Gram matrix of the J_{n+1}(2 pi v) under a positive weight); a pivot that is not positive (DC, where Gamma = 0)
// zeroes its column.
__global__ void k_full_chol(const double* __restrict__ Gp, int no, int noct, float* __restrict__ C) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= noct) return;
  double A[kMaxOrders * kMaxOrders];
  for (int a = 0; a < no; ++a)
    for (int b = a; b < no; ++b) {
      const double g = Gp[(size_t)(a * no - a * (a - 1) / 2 + (b - a)) * noct + i];
      A[a * no + b] = g;
      A[b * no + a] = g;
    }
  for (int a = 0; a < no; ++a) {
    for (int b = 0; b <= a; ++b) {
      double s = A[a * no + b];
      for (int k = 0; k < b; ++k) s -= A[a * no + k] * A[b * no + k];
      if (a == b) A[a * no + a] = s > 0.0 ? sqrt(s) : 0.0;
      else A[a * no + b] = A[b * no + b] > 0.0 ? s / A[b * no + b] : 0.0;
    }
  }
  const int tri = no * (no + 1) / 2, trip = (tri + 3) / 4 * 4;  // rows padded to whole float4
  float* c = C + (size_t)i * trip;
  for (int a = 0; a < no; ++a)
    for (int b = 0; b <= a; ++b) c[a * (a + 1) / 2 + b] = (float)A[a * no + b];
  for (int e = tri; e < trip; ++e) c[e] = 0.f;
}

// Per mode: the order slot, m, sin/cos, Noll's angular prefactor (-1)^((n-m)/2) i^m sqrt 2 ((-1)^(n/2) for m = 0)
// and kappa0_j = sqrt(A0_jj (n_j + 1) / sum_k P_jj(k)) (A0_jj from the rows of L, D/r0 = 1).
__global__ void k_full_modes(const ModeInfo* __restrict__ modes, int J, const double* __restrict__ L64,
                             const double* __restrict__ sums, dfp2s_full_mode* __restrict__ out) {
  const int j = threadIdx.x;
  if (j >= J) return;
  const ModeInfo mi = modes[j];
  double a0 = 0.0;
  for (int k = 0; k <= j; ++k) a0 += L64[j * J + k] * L64[j * J + k];
  dfp2s_full_mode o;
  o.o = mi.o;
  o.m = mi.m;
  o.odd = mi.odd;
  o.pad = 0;
  if (mi.m == 0) {
    o.pre_re = ((mi.n / 2) & 1) ? -1.f : 1.f;
    o.pre_im = 0.f;
  } else {
    const float sg = (((mi.n - mi.m) / 2) & 1) ? -1.f : 1.f;
    const float r2 = 1.41421356237309505f;
    const int q = mi.m & 3;  // i^m
    o.pre_re = q == 0 ? sg * r2 : (q == 2 ? -sg * r2 : 0.f);
    o.pre_im = q == 1 ? sg * r2 : (q == 3 ? -sg * r2 : 0.f);
  }
  o.kappa0 = (float)sqrt(a0 * (mi.n + 1) / sums[j]);
  o.pad2 = 0.f;
  out[j] = o;
}

// ---- the dense per-frequency root (Sec. III-A's eigen-root form applied per frequency; reading R6)
// For half-plane bin k: S(k) = L diag(lambda(k)) L^T (J x J, FP64, D/r0 = 1), its eigendecomposition by cyclic
// Jacobi rotations, and the symmetric root F = U diag(sqrt(max(ev, 0))) U^T, stored in FP32 as F[j * J + i][bin]
// (bins contiguous).  One warp per matrix: the J/2 disjoint pairs of a round-robin round rotate at once (rows,
// then columns and the eigenvector columns), sweeps until the off-diagonal mass is below 1e-30 of the diagonal's
// (at most kDenseSweeps); the matrix lives in shared memory, J padded to an even JP with a zero row and column.
constexpr int kDenseSweeps = 16;
constexpr int kDenseWarps = 4;  // matrices per CTA

DFP2S_DEV int dense_pair_member(int t, int r, int JP) { return t == 0 ? 0 : ((t - 1 + r) % (JP - 1)) + 1; }

__global__ void __launch_bounds__(32 * kDenseWarps) k_dense_root(const ModeInfo* __restrict__ modes, int J, int JP,
                                                              int N, const double* __restrict__ G, int noct,
                                                              const double* __restrict__ sums,
                                                              const double* __restrict__ L64, float* __restrict__ F,
                                                              long long nbins) {
  extern __shared__ double dsm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int JJ = JP * JP;
  double* A = dsm + (size_t)warp * (2 * JJ + 2 * JP);
  double* V = A + JJ;
  double* lam = V + JJ;  // JP
  double* cs = lam + JP;  // JP: (c, s) per pair
  for (long long bin = (long long)blockIdx.x * kDenseWarps + warp; bin < nbins;
       bin += (long long)gridDim.x * kDenseWarps) {
    const int kx = (int)(bin / N), ky = (int)(bin - (long long)kx * N);
    for (int j = lane; j < JP; j += 32)
      lam[j] = j < J ? (double)N * N * mode_power(modes[j], kx, ky, N, G, noct) / sums[j] : 0.0;
    __syncwarp();
    for (int e = lane; e < JJ; e += 32) {
      const int a = e / JP, b = e - a * JP;
      double v = 0.0;
      if (a < J && b < J) {
        const int kmax = a < b ? a : b;
        for (int k = 0; k <= kmax; ++k) v = fma(L64[a * J + k] * lam[k], L64[b * J + k], v);
      }
      A[e] = v;
      V[e] = a == b ? 1.0 : 0.0;
    }
    __syncwarp();
    for (int sweep = 0; sweep < kDenseSweeps; ++sweep) {
      double off = 0.0, dia = 0.0;
      for (int e = lane; e < JJ; e += 32) {
        const int a = e / JP, b = e - a * JP;
        if (a == b) dia += A[e] * A[e];
        else off += A[e] * A[e];
      }
      for (int o = 16; o > 0; o >>= 1) {
        off += __shfl_xor_sync(0xffffffffu, off, o);
        dia += __shfl_xor_sync(0xffffffffu, dia, o);
      }
      if (!(off > 1e-30 * dia)) break;  // warp-uniform (reduced values)
      for (int r = 0; r < JP - 1; ++r) {
        for (int q2 = lane; q2 < JP / 2; q2 += 32) {
          const int p = dense_pair_member(q2, r, JP), q = dense_pair_member(JP - 1 - q2, r, JP);
          const double apq = A[p * JP + q];
          double c = 1.0, sn = 0.0;
          if (apq != 0.0) {
            const double tau = (A[q * JP + q] - A[p * JP + p]) / (2.0 * apq);
            const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            sn = t * c;
          }
          cs[2 * q2] = c;
          cs[2 * q2 + 1] = sn;
        }
        __syncwarp();
        for (int e = lane; e < (JP / 2) * JP; e += 32) {  // rows p, q of A
          const int q2 = e / JP, k = e - q2 * JP;
          const int p = dense_pair_member(q2, r, JP), q = dense_pair_member(JP - 1 - q2, r, JP);
          const double c = cs[2 * q2], sn = cs[2 * q2 + 1];
          const double x = A[p * JP + k], y = A[q * JP + k];
          A[p * JP + k] = c * x - sn * y;
          A[q * JP + k] = sn * x + c * y;
        }
        __syncwarp();
        for (int e = lane; e < (JP / 2) * JP; e += 32) {  // columns p, q of A and of V
          const int q2 = e / JP, k = e - q2 * JP;
          const int p = dense_pair_member(q2, r, JP), q = dense_pair_member(JP - 1 - q2, r, JP);
          const double c = cs[2 * q2], sn = cs[2 * q2 + 1];
          const double x = A[k * JP + p], y = A[k * JP + q];
          A[k * JP + p] = c * x - sn * y;
          A[k * JP + q] = sn * x + c * y;
          const double u = V[k * JP + p], w = V[k * JP + q];
          V[k * JP + p] = c * u - sn * w;
          V[k * JP + q] = sn * u + c * w;
        }
        __syncwarp();
      }
    }
    for (int j = lane; j < JP; j += 32) {
      const double ev = A[j * JP + j];
      lam[j] = ev > 0.0 ? sqrt(ev) : 0.0;  // rounding of a near-singular matrix: negative eigenvalues clamp to 0
    }
    __syncwarp();
    for (int e = lane; e < J * J; e += 32) {
      const int a = e / J, b = e - a * J;
      double v = 0.0;
      for (int k = 0; k < JP; ++k) v = fma(V[a * JP + k] * lam[k], V[b * JP + k], v);
      F[(size_t)e * nbins + bin] = (float)v;
    }
    __syncwarp();  // the buffers are rewritten by the warp's next matrix
  }
}

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.resize(n);
  w.resize(n);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double z = cos(pi * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

void v_rule(std::vector<double>& v, std::vector<double>& w) {
  std::vector<double> x8, w8, x16, w16;
  gauss_legendre(8, x8, w8);
  gauss_legendre(16, x16, w16);
  const double y0 = log(1e-7), y1 = 0.0;
  const int nlog = 65;
  for (int p = 0; p < nlog; ++p) {
    const double a = y0 + (y1 - y0) * p / nlog, b = y0 + (y1 - y0) * (p + 1) / nlog;
    for (int i = 0; i < 8; ++i) {
      const double y = 0.5 * (b - a) * x8[i] + 0.5 * (a + b);
      const double vv = exp(y);
      v.push_back(vv);
      w.push_back(0.5 * (b - a) * w8[i] * vv);
    }
  }
  for (int p = 0; p < 94; ++p) {
    const double a = 1.0 + 0.5 * p, b = a + 0.5;
    for (int i = 0; i < 16; ++i) {
      v.push_back(0.5 * (b - a) * x16[i] + 0.5 * (a + b));
      w.push_back(0.5 * (b - a) * w16[i]);
    }
  }
}

// The v-rule for frequencies far below the torus bins (the subharmonics): 8-point panels of width <= 0.2 in ln v
// from 1e-14 to 1 (the integrand's mass lies at v >~ f, down to df / 3^12), then the uniform panels of v_rule.
void v_rule_deep(std::vector<double>& v, std::vector<double>& w) {
  std::vector<double> x8, w8, x16, w16;
  gauss_legendre(8, x8, w8);
  gauss_legendre(16, x16, w16);
  const double y0 = log(1e-14);
  const int nlog = (int)ceil(-y0 / 0.2);
  for (int p = 0; p < nlog; ++p) {
    const double a = y0 * (1.0 - (double)p / nlog), b = y0 * (1.0 - (double)(p + 1) / nlog);
    for (int i = 0; i < 8; ++i) {
      const double vv = exp(0.5 * (b - a) * x8[i] + 0.5 * (a + b));
      v.push_back(vv);
      w.push_back(0.5 * (b - a) * w8[i] * vv);
    }
  }
  for (int p = 0; p < 94; ++p) {
    const double a = 1.0 + 0.5 * p, b = a + 0.5;
    for (int i = 0; i < 16; ++i) {
      v.push_back(0.5 * (b - a) * x16[i] + 0.5 * (a + b));
      w.push_back(0.5 * (b - a) * w16[i]);
    }
  }
}

template <typename T>
struct DevBuf {
  T* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  cudaError_t alloc(size_t n) { return dfp2s_device_malloc((void**)&p, n * sizeof(T)); }
};

}  // namespace

int dfp2s_radial_order_count(int J) {
  int count = 0, last = -1;
  for (int j = 2; j <= J + 1; ++j) {
    int n = 0;
    while ((n + 1) * (n + 2) / 2 < j) ++n;
    if (n != last) ++count;  // Noll's index runs through the orders in ascending order
    last = n;
  }
  return count;
}

int dfp2s_factor_build_device(dfp2s_factor_dev* f, cudaStream_t st) {
  const int J = f->J, N = f->N;
  // ---- twiddles (FP64 -> FP32)
  {
    std::vector<float2> tw(N);
    const double pi = 3.14159265358979323846;
    for (int m = 0; m < N; ++m) {
      const double a = -2.0 * pi * m / N;
      tw[m] = make_float2((float)cos(a), (float)sin(a));
    }
    DFP2S_CUDA_TRY(cudaMemcpyAsync(f->tw, tw.data(), N * sizeof(float2), cudaMemcpyHostToDevice, st));
    DFP2S_CUDA_TRY(cudaStreamSynchronize(st));
  }
  // ---- modes and radial orders
  std::vector<ModeInfo> modes(J);
  std::vector<int> orders;
  for (int j = 0; j < J; ++j) {
    const int nj = j + 2;
    int n = 0;
    while ((n + 1) * (n + 2) / 2 < nj) ++n;
    const int r = nj - n * (n + 1) / 2 - 1;
    const int m = (n % 2 == 0) ? 2 * ((r + 1) / 2) : 2 * (r / 2) + 1;
    int o = -1;
    for (size_t k = 0; k < orders.size(); ++k)
      if (orders[k] == n) o = (int)k;
    if (o < 0) {
      o = (int)orders.size();
      orders.push_back(n);
    }
    modes[j] = ModeInfo{n, m, nj & 1, o};
  }
  if ((int)orders.size() > kMaxOrders) return dfp2s_fail(DFP2S_EINVAL, "too many radial orders");
  std::vector<double> hv, hw;
  v_rule(hv, hw);
  const int Q = (int)hv.size();
  const int no = (int)orders.size();
  const int noct = (N / 2 + 1) * (N / 2 + 2) / 2;

  DevBuf<double> dv, dw, gtab, G, sums;
  DevBuf<int> dord, derr;
  DevBuf<ModeInfo> dmodes;
  DFP2S_CUDA_TRY(dv.alloc(Q));
  DFP2S_CUDA_TRY(dw.alloc(Q));
  DFP2S_CUDA_TRY(gtab.alloc((size_t)Q * no));
  DFP2S_CUDA_TRY(G.alloc((size_t)no * noct));
  DFP2S_CUDA_TRY(sums.alloc(J));
  DFP2S_CUDA_TRY(dord.alloc(no));
  DFP2S_CUDA_TRY(derr.alloc(1));
  DFP2S_CUDA_TRY(dmodes.alloc(J));
  DFP2S_CUDA_TRY(cudaMemcpyAsync(dv.p, hv.data(), Q * sizeof(double), cudaMemcpyHostToDevice, st));
  DFP2S_CUDA_TRY(cudaMemcpyAsync(dw.p, hw.data(), Q * sizeof(double), cudaMemcpyHostToDevice, st));
  DFP2S_CUDA_TRY(cudaMemcpyAsync(dord.p, orders.data(), no * sizeof(int), cudaMemcpyHostToDevice, st));
  DFP2S_CUDA_TRY(cudaMemcpyAsync(dmodes.p, modes.data(), J * sizeof(ModeInfo), cudaMemcpyHostToDevice, st));
  DFP2S_CUDA_TRY(cudaMemsetAsync(sums.p, 0, J * sizeof(double), st));
  DFP2S_CUDA_TRY(cudaMemsetAsync(derr.p, 0, sizeof(int), st));

  k_noll_chol<<<1, 256, 0, st>>>(J, f->L64, f->L32, derr.p);
  k_gtab<<<(Q * no + 255) / 256, 256, 0, st>>>(dv.p, dw.p, Q, dord.p, dord.p, no, gtab.p);
  k_radial<<<(noct + 127) / 128, 128, 0, st>>>(dv.p, gtab.p, Q, no, no, N, f->pix_per_D / N, G.p, noct);
  const size_t total = (size_t)(N / 2 + 1) * N;
  const unsigned blocks = (unsigned)((total + 255) / 256);
  k_lambda_sums<<<blocks, 256, 0, st>>>(dmodes.p, J, N, G.p, noct, sums.p);
  DevBuf<double> dfl, Gl, dv2, dw2, gtab2d;
  if (f->sh_levels > 0) {
    const int L = f->sh_levels, nf = 2 * L;
    std::vector<double> fl(nf);
    const double df = f->pix_per_D / N;
    double scale = 1.0;
    for (int p = 0; p < L; ++p) {
      scale /= 3.0;
      fl[2 * p] = df * scale;                          // axis directions
      fl[2 * p + 1] = df * scale * 1.41421356237309505;  // diagonals
    }
    std::vector<double> hv2, hw2;
    v_rule_deep(hv2, hw2);
    const int Q2 = (int)hv2.size();
    DFP2S_CUDA_TRY(dfl.alloc(nf));
    DFP2S_CUDA_TRY(Gl.alloc((size_t)no * nf));
    DFP2S_CUDA_TRY(dv2.alloc(Q2));
    DFP2S_CUDA_TRY(dw2.alloc(Q2));
    DFP2S_CUDA_TRY(gtab2d.alloc((size_t)Q2 * no));
    DFP2S_CUDA_TRY(cudaMemcpyAsync(dfl.p, fl.data(), nf * sizeof(double), cudaMemcpyHostToDevice, st));
    DFP2S_CUDA_TRY(cudaMemcpyAsync(dv2.p, hv2.data(), Q2 * sizeof(double), cudaMemcpyHostToDevice, st));
    DFP2S_CUDA_TRY(cudaMemcpyAsync(dw2.p, hw2.data(), Q2 * sizeof(double), cudaMemcpyHostToDevice, st));
    k_gtab<<<(Q2 * no + 255) / 256, 256, 0, st>>>(dv2.p, dw2.p, Q2, dord.p, dord.p, no, gtab2d.p);
    k_radial_list<<<1, 32, 0, st>>>(dv2.p, gtab2d.p, Q2, no, dfl.p, nf, Gl.p);
    k_sh_tables<<<1, 64, 0, st>>>(dmodes.p, J, L, Gl.p, sums.p, f->sh_amp);
  }
  k_lambda_write<<<blocks, 256, 0, st>>>(dmodes.p, J, N, G.p, noct, sums.p, f->mult);
  DFP2S_CUDA_TRY(cudaGetLastError());
  if (f->dense) {
    const int JP = (J + 1) / 2 * 2;
    const size_t smem = (size_t)kDenseWarps * (2 * JP * JP + 2 * JP) * sizeof(double);
    DFP2S_CUDA_TRY(cudaFuncSetAttribute(k_dense_root, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long nbins = (long long)(N / 2 + 1) * N;
    const long long want = (nbins + kDenseWarps - 1) / kDenseWarps;
    const int grid = (int)(want < 8LL * sms ? want : 8LL * sms);
    k_dense_root<<<grid, 32 * kDenseWarps, smem, st>>>(dmodes.p, J, JP, N, G.p, noct, sums.p, f->L64, f->dense,
                                                      nbins);
    DFP2S_CUDA_TRY(cudaGetLastError());
  }
  DevBuf<double> gtab2, Gp;
  DevBuf<int> dpa, dpb;
  if (f->fchol) {
    // the full sampler: radial spectra of every pair of orders, their Cholesky factor per octant bin, mode constants
    if (f->R != no) return dfp2s_fail(DFP2S_EINVAL, "full sampler: %d radial orders, tables sized for %d", no, f->R);
    std::vector<int> pa, pb;
    for (int a = 0; a < no; ++a)
      for (int b = a; b < no; ++b) {
        pa.push_back(orders[a]);
        pb.push_back(orders[b]);
      }
    const int np = (int)pa.size();
    DFP2S_CUDA_TRY(gtab2.alloc((size_t)Q * np));
    DFP2S_CUDA_TRY(Gp.alloc((size_t)np * noct));
    DFP2S_CUDA_TRY(dpa.alloc(np));
    DFP2S_CUDA_TRY(dpb.alloc(np));
    DFP2S_CUDA_TRY(cudaMemcpyAsync(dpa.p, pa.data(), np * sizeof(int), cudaMemcpyHostToDevice, st));
    DFP2S_CUDA_TRY(cudaMemcpyAsync(dpb.p, pb.data(), np * sizeof(int), cudaMemcpyHostToDevice, st));
    k_gtab<<<(Q * np + 255) / 256, 256, 0, st>>>(dv.p, dw.p, Q, dpa.p, dpb.p, np, gtab2.p);
    for (int c0 = 0; c0 < np; c0 += kMaxOrders) {
      const int nc = np - c0 < kMaxOrders ? np - c0 : kMaxOrders;
      k_radial<<<(noct + 127) / 128, 128, 0, st>>>(dv.p, gtab2.p + c0, Q, nc, np, N, f->pix_per_D / N,
                                                   Gp.p + (size_t)c0 * noct, noct);
    }
    k_full_chol<<<(noct + 127) / 128, 128, 0, st>>>(Gp.p, no, noct, f->fchol);
    k_full_modes<<<1, 64, 0, st>>>(dmodes.p, J, f->L64, sums.p, f->fmode);
    DFP2S_CUDA_TRY(cudaGetLastError());
  }
  int herr = 0;
  DFP2S_CUDA_TRY(cudaMemcpyAsync(&herr, derr.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  DFP2S_CUDA_TRY(cudaStreamSynchronize(st));
  if (herr) return dfp2s_fail(DFP2S_ECUDA, "Noll matrix is not positive definite on the device");
  return DFP2S_OK;
}
