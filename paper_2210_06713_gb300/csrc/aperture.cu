// Aperture and spatial statistics of sampled Zernike fields (Sec. IV-B), the checks the paper applies to its
// simulator: the structure function of the pupil phase against 6.88 (r / r0)^{5/3} (Eq. fried_struct), the long-
// and short-exposure OTFs (Eqs. H_LE, H_SE: the mean autocorrelation of P e^{-j phi}, the second with the plane
// of best fit removed), and the tilt correlation with the differential tilt variance.
//
// Realisations are the Zernike vectors of the pixels on a sub-grid of the frame (every `step`-th row and column).
// The pupil is the 64 x 64 grid of the exact P2S (coordinates (i - 32)/16, aperture rho <= 1: 797 samples inside
// the 33 x 33 window at rows and columns 16..48).  One CTA (256 threads) per SM walks the realisations:
//   phi = sum_j a_j Z_j on the window (FP32, the Zernike table evaluated in FP64 at the call), the plane
//   c0 + c1 x + c2 y of least squares over the aperture (X^T X is diagonal on the symmetric aperture: three block
//   sums), the squared phase differences of every aperture pair at x and y offsets 1..32 (a warp per offset and
//   direction, a lane per window line; folded per realisation into FP64 sums), and two 64 x 64 FFTs at once (64
//   thread pairs per grid, the register FFT of the field sampler): P e^{-j phi} and P e^{-j (phi - plane)}.
//   |X|^2 of each grid point is owned by one thread: summed in FP32 registers over 16 realisations, then into FP64
//   sums in shared memory.  The OTF is the normalised inverse transform of the mean PSF (the mean
//   autocorrelation, by linearity), taken in FP64 by two separable passes after a fixed-order sum over CTAs.
#include <cuda_runtime.h>
#include <math.h>

#include "common.cuh"
#include "fft_reg.cuh"
#include "kernels.h"
#include "zernike.cuh"

namespace {

constexpr int GN = 64;            // pupil grid
constexpr int WS = 33;            // aperture window side (rows / columns 16..48 of the grid)
constexpr int W0 = 16;            // first window row / column on the grid
constexpr int WQ = WS * WS;       // 1089 window samples
constexpr int SFL = DFP2S_SF_LAGS;  // 33 offsets 0..32
constexpr int THREADS = 256;
constexpr int US = GN + 1;        // padded row stride of the pupil grids (complex)
constexpr int GBUF = fftr::Plan<GN>::BUF;  // 66 entries per FFT group
constexpr int NPART = 2 * SFL + 2 * GN * GN;  // per-CTA partial sums
constexpr int QS = (WQ + THREADS - 1) / THREADS;  // window samples per thread
constexpr int PSF_FOLD = 16;  // realisations summed in FP32 before a fold into the FP64 PSF sums

// Z_j on the window for j = Noll 2..J+1 ([j][q], q = row * 33 + column, zero outside the aperture) and the 64
// twiddles exp(-2 pi i m / 64).
__global__ void k_aperture_tables(int J, float* __restrict__ Z, float2* __restrict__ tw) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;  // one table entry (mode j, sample q) per thread
  if (e < GN) {
    double s, c;
    sincospi(-2.0 * e / GN, &s, &c);
    tw[e] = make_float2((float)c, (float)s);
  }
  if (e >= J * WQ) return;
  const int j = e / WQ, q = e - j * WQ;
  const int i = q / WS, l = q - i * WS;
  const int iy = i - 16, ix = l - 16;
  const double x = ix / 16.0, y = iy / 16.0;
  const bool inside = ix * ix + iy * iy <= 256;
  const double rho = sqrt(x * x + y * y), th = atan2(y, x);
  Z[e] = inside ? (float)dfp2s_zernike(j + 2, rho, th) : 0.f;
}

struct ApSmem {
  float2 U[2][GN * US];       // the two pupil grids (LE, SE), rows 16..48 filled
  float2 gbuf[128][GBUF];     // FFT exchange buffers, one per thread pair
  double psf[2][GN * GN];     // the CTA's PSF sums [set][ky * 64 + kx]
  float phi[2][WQ + 3];       // phi and phi - plane on the window
  float a[DFP2S_MAX_J];
  float sf[2 * SFL];          // this realisation's structure-function sums (x offsets, then y)
  float red[THREADS / 32][3];
};

__global__ void __launch_bounds__(THREADS, 1) k_aperture_partial(const float* __restrict__ fields, int J, int H, int W,
                                                              int step, int nx, long long nreal,
                                                              const float* __restrict__ Z,
                                                              const float2* __restrict__ tw,
                                                              double* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ApSmem& s = *reinterpret_cast<ApSmem*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const size_t plane = (size_t)H * W;
  for (int e = tid; e < 2 * GN * GN; e += THREADS) (&s.psf[0][0])[e] = 0.0;
  for (int e = tid; e < 2 * SFL; e += THREADS) s.sf[e] = 0.f;
  double sf_acc = 0.0;  // thread t < 66 owns structure-function entry t
  // the aperture's constants: sample count and sum x^2 (= sum y^2) over rho <= 1 of the window
  int na = 0;
  double sxx = 0.0;
  for (int iy = -16; iy <= 16; ++iy)
    for (int ix = -16; ix <= 16; ++ix)
      if (ix * ix + iy * iy <= 256) {
        ++na;
        sxx += (ix / 16.0) * (ix / 16.0);
      }
  const float inv_na = (float)(1.0 / na), inv_sxx = (float)(1.0 / sxx);
  // |X|^2 of this thread's 32 grid points (column (tid >> 1) & 63, rows (tid & 1) + 2 m of set tid >> 7: the same
  // points in every realisation), summed in FP32 over PSF_FOLD realisations, then added to the FP64 sums
  constexpr int PV = fftr::Plan<GN>::V;
  float pacc[PV];
#pragma unroll
  for (int m = 0; m < PV; ++m) pacc[m] = 0.f;
  int nacc = 0;
  const int pset = (tid >> 1) >> 6, pcol = (tid >> 1) & 63, prow = tid & 1;
  auto fold = [&]() {
#pragma unroll
    for (int m = 0; m < PV; ++m) {
      s.psf[pset][(prow + 2 * m) * GN + pcol] += (double)pacc[m];
      pacc[m] = 0.f;
    }
    nacc = 0;
  };
  // the Zernike vector of a realisation is loaded one realisation ahead
  auto coeff = [&](long long r) {
    const int ry = (int)(r / nx), rx = (int)(r - (long long)ry * nx);
    return __ldg(fields + (size_t)tid * plane + (size_t)(ry * step) * W + (size_t)(rx * step));
  };
  float anext = tid < J && blockIdx.x < nreal ? coeff(blockIdx.x) : 0.f;
  __syncthreads();
  for (long long r = blockIdx.x; r < nreal; r += gridDim.x) {
    if (tid < J) s.a[tid] = anext;
    if (tid < J && r + gridDim.x < nreal) anext = coeff(r + gridDim.x);
    __syncthreads();
    // ---- phase on the window and the plane-fit sums.  Thread t owns samples q = t + 256 k (k < QS); the J loop
    // runs six modes at a time so that 6 QS table loads are in flight together (the table does not fit beside the
    // shared arrays and is read from L2); each sample's FMA chain still runs over j in order.
    float v[QS];
#pragma unroll
    for (int k = 0; k < QS; ++k) v[k] = 0.f;
    int qc[QS];
#pragma unroll
    for (int k = 0; k < QS; ++k) qc[k] = min(tid + THREADS * k, WQ - 1);  // clamped: the tail's loads stay in bounds
    int j = 0;
    for (; j + 6 <= J; j += 6) {
      float z[6][QS];
#pragma unroll
      for (int u = 0; u < 6; ++u)
#pragma unroll
        for (int k = 0; k < QS; ++k) z[u][k] = __ldg(Z + (size_t)(j + u) * WQ + qc[k]);
#pragma unroll
      for (int u = 0; u < 6; ++u) {
        const float aj = s.a[j + u];
#pragma unroll
        for (int k = 0; k < QS; ++k) v[k] = fmaf(aj, z[u][k], v[k]);
      }
    }
    for (; j < J; ++j) {
      const float aj = s.a[j];
#pragma unroll
      for (int k = 0; k < QS; ++k) v[k] = fmaf(aj, __ldg(Z + (size_t)j * WQ + qc[k]), v[k]);
    }
    float p0 = 0.f, p1 = 0.f, p2 = 0.f;
#pragma unroll
    for (int k = 0; k < QS; ++k) {
      const int q = tid + THREADS * k;
      if (q < WQ) {
        const int i = q / WS, l = q - i * WS;
        const bool inside = (i - 16) * (i - 16) + (l - 16) * (l - 16) <= 256;
        const float vq = inside ? v[k] : 0.f;
        s.phi[0][q] = vq;
        p0 += vq;
        p1 = fmaf(vq, (l - 16) * 0.0625f, p1);
        p2 = fmaf(vq, (i - 16) * 0.0625f, p2);
      }
    }
    for (int off = 16; off > 0; off >>= 1) {
      p0 += __shfl_xor_sync(0xffffffffu, p0, off);
      p1 += __shfl_xor_sync(0xffffffffu, p1, off);
      p2 += __shfl_xor_sync(0xffffffffu, p2, off);
    }
    if (lane == 0) {
      s.red[warp][0] = p0;
      s.red[warp][1] = p1;
      s.red[warp][2] = p2;
    }
    __syncthreads();
    float c0 = 0.f, c1 = 0.f, c2 = 0.f;
    for (int w = 0; w < THREADS / 32; ++w) {
      c0 += s.red[w][0];
      c1 += s.red[w][1];
      c2 += s.red[w][2];
    }
    c0 *= inv_na;
    c1 *= inv_sxx;
    c2 *= inv_sxx;
    for (int q = tid; q < WQ; q += THREADS) {
      const int i = q / WS, l = q - i * WS;
      const bool inside = (i - 16) * (i - 16) + (l - 16) * (l - 16) <= 256;
      s.phi[1][q] = inside ? s.phi[0][q] - (c0 + c1 * ((l - 16) * 0.0625f) + c2 * ((i - 16) * 0.0625f)) : 0.f;
    }
    // ---- structure function: warp w takes the (direction, offset d) pairs w, w + 8, ...; lane = window line
    // (line 32 holds one aperture sample, no pairs), its pairs inside the aperture summed in FP32, the lanes folded
    // and the sum written by lane 0 (one writer per entry).  The loop runs over the whole line in every lane, so that
    // the lanes' shared-memory reads fall in distinct banks, and masks the pairs outside the aperture.
    {
      const int t = lane - 16;
      int h = (int)sqrtf((float)(256 - t * t));  // samples 16 - h .. 16 + h of the line are inside
      while (h * h > 256 - t * t) --h;
      while ((h + 1) * (h + 1) <= 256 - t * t) ++h;
      for (int pr = warp; pr < 2 * (SFL - 1); pr += THREADS / 32) {
        const int dir = pr / (SFL - 1), d = 1 + pr - dir * (SFL - 1);
        const int ea = dir == 0 ? lane * WS : lane, st = dir == 0 ? 1 : WS;  // sample u of the line at ea + u st
        float acc = 0.f;
#pragma unroll 4
        for (int u = 0; u + d < WS; ++u) {
          const float df = s.phi[0][ea + u * st] - s.phi[0][ea + (u + d) * st];
          acc = (u >= 16 - h && u + d <= 16 + h) ? fmaf(df, df, acc) : acc;
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) s.sf[dir * SFL + d] = acc;
      }
    }
    __syncthreads();  // phi[1] and the sums complete
    if (tid < 2 * SFL) {
      sf_acc += (double)s.sf[tid];
      s.sf[tid] = 0.f;
    }
    // ---- the two pupil grids, rows 16..48: P e^{-j phi}
    for (int e = tid; e < 2 * WS * GN; e += THREADS) {
      const int set = e / (WS * GN), rem = e - set * WS * GN;
      const int i = rem / GN, k = rem - i * GN;  // window row i, grid column k
      float2 u = make_float2(0.f, 0.f);
      const int l = k - W0;
      if (l >= 0 && l < WS && (i - 16) * (i - 16) + (l - 16) * (l - 16) <= 256) {
        float sn, cs;
        sincosf(s.phi[set][i * WS + l], &sn, &cs);
        u = make_float2(cs, -sn);
      }
      s.U[set][(W0 + i) * US + k] = u;
    }
    __syncthreads();
    // ---- row transforms of the 2 x 33 filled rows (rows 16..48 of each grid): thread pair g < 66 takes row
    // g % 33 of grid g / 33; the FFT synchronises whole warps, so the five warps holding those pairs run it (pairs
    // 66..79 on zeros) and the other three skip it
    {
      const int g = tid >> 1, t = tid & 1;
      const bool live = g < 2 * WS;
      const int set = live ? g / WS : 0, rr = live ? g - set * WS : 0;
      float2* row = s.U[set] + (W0 + rr) * US;
      float2 v[fftr::Plan<GN>::V];
      if (warp < (4 * WS + 31) / 32) {
#pragma unroll
        for (int m = 0; m < fftr::Plan<GN>::V; ++m) v[m] = live ? row[t + 2 * m] : make_float2(0.f, 0.f);
        fftr::fft<GN, false>(v, s.gbuf[g], t, tw);
      }
      __syncthreads();  // every row read before any is written
      if (live) {
#pragma unroll
        for (int m = 0; m < fftr::Plan<GN>::V; ++m) row[t + 2 * m] = v[fftr::OutIndex<GN>::reg(m)];
      }
    }
    __syncthreads();
    // ---- column transforms (rows outside 16..48 are zero) and |X|^2 into the CTA's PSF sums
    {
      const int g = tid >> 1, t = tid & 1, set = g >> 6, col = g & 63;
      float2 v[fftr::Plan<GN>::V];
#pragma unroll
      for (int m = 0; m < fftr::Plan<GN>::V; ++m) {
        const int row = t + 2 * m;
        v[m] = (row >= W0 && row < W0 + WS) ? s.U[set][row * US + col] : make_float2(0.f, 0.f);
      }
      fftr::fft<GN, false>(v, s.gbuf[g], t, tw);
#pragma unroll
      for (int m = 0; m < fftr::Plan<GN>::V; ++m) {
        const float2 x = v[fftr::OutIndex<GN>::reg(m)];
        pacc[m] = fmaf(x.x, x.x, fmaf(x.y, x.y, pacc[m]));
      }
      if (++nacc == PSF_FOLD) fold();
    }
    __syncthreads();  // the grids and buffers are rewritten by the next realisation
  }
  if (nacc > 0) fold();
  __syncthreads();  // every thread's last fold before the sums are written out
  double* out = part + (size_t)blockIdx.x * NPART;
  if (tid < 2 * SFL) out[tid] = sf_acc;
  for (int e = tid; e < 2 * GN * GN; e += THREADS) out[2 * SFL + e] = (&s.psf[0][0])[e];
}

// Fixed-order sum over the CTAs; the structure function divided by its pair counts and realisations.
__global__ void k_aperture_sum(const double* __restrict__ part, int nb, long long nreal, double* __restrict__ sums,
                               double* __restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= NPART) return;
  double acc = 0.0;
  for (int b = 0; b < nb; ++b) acc += part[(size_t)b * NPART + e];
  if (e < 2 * SFL) {
    const int dir = e / SFL, d = e - dir * SFL;
    (void)dir;  // the aperture is symmetric: the pair counts along x and y are equal
    long long pairs = 0;
    for (int i = 0; i < WS; ++i)
      for (int u = 0; u + d < WS; ++u) {
        const bool a = (i - 16) * (i - 16) + (u - 16) * (u - 16) <= 256;
        const bool b = (i - 16) * (i - 16) + (u + d - 16) * (u + d - 16) <= 256;
        pairs += (d > 0 && a && b) ? 1 : 0;
      }
    out[e] = pairs ? acc / ((double)pairs * (double)nreal) : 0.0;
  } else {
    sums[e - 2 * SFL] = acc;
  }
}

// OTF of grid `set` (Eqs. H_LE, H_SE): H(nu) = Re sum_k psf(k) e^{+2 pi i k.nu / 64} / sum_k psf(k), separable,
// FP64.  k_otf_rows: CTA (ky, set), thread nu_x: T1[set][ky][nu_x] = sum_kx psf(ky, kx) e^{+2 pi i kx nu_x / 64};
// k_otf_cols: CTA (nu_y, set), thread nu_x: the transform of T1 over ky, divided by the PSF sum (T1 at nu_x = 0
// summed over ky).  128 CTAs each: the 2 x 2 x 64^3 FP64 multiply-adds spread over the SMs.
__global__ void __launch_bounds__(GN) k_otf_rows(const double* __restrict__ sums, double2* __restrict__ T1) {
  __shared__ double cs[GN], sn[GN], row[GN];
  const int ky = blockIdx.x, set = blockIdx.y, vx = threadIdx.x;
  sincospi(2.0 * vx / GN, &sn[vx], &cs[vx]);
  row[vx] = sums[((size_t)set * GN + ky) * GN + vx];
  __syncthreads();
  double re = 0.0, im = 0.0;
  for (int kx = 0; kx < GN; ++kx) {
    const double v = row[kx];
    const int m = (kx * vx) & (GN - 1);
    re = fma(v, cs[m], re);
    im = fma(v, sn[m], im);
  }
  T1[((size_t)set * GN + ky) * GN + vx] = make_double2(re, im);
}

__global__ void __launch_bounds__(GN) k_otf_cols(const double2* __restrict__ T1, double* __restrict__ out) {
  __shared__ double cs[GN], sn[GN];
  const int vy = blockIdx.x, set = blockIdx.y, vx = threadIdx.x;
  sincospi(2.0 * vx / GN, &sn[vx], &cs[vx]);
  __syncthreads();
  const double2* t1 = T1 + (size_t)set * GN * GN;
  double total = 0.0;
  for (int ky = 0; ky < GN; ++ky) total += t1[ky * GN].x;  // nu = 0: the sum of the PSF
  double re = 0.0;
  for (int ky = 0; ky < GN; ++ky) {
    const double2 t = t1[ky * GN + vx];
    const int m = (ky * vy) & (GN - 1);
    re += t.x * cs[m] - t.y * sn[m];
  }
  out[((size_t)set * GN + vy) * GN + vx] = re / total;
}

// ---- tilt correlation and DTV.  The frame is cut into tiles of TILT_R rows x TILT_C columns; a CTA walks its
// tiles, and on each its eight warps take the (direction, lag) items in turn.  Lane l holds the tile's pixels p in
// columns x0 + l + 32 i of both tilt fields in registers, as two-lane FP32 values (Noll 2, Noll 3), for all its
// items; per item it loads only the partners p + d and forms the eight sums on two-lane FP32 instructions (at most
// TILT_R x TILT_C / 32 = 32 pairs per lane).  No load sits behind a branch: a tile inside the item's window takes
// an unguarded path, an edge tile clamps the addresses of the pairs outside the window and adds zeros for them, so
// that a lane's 64 partner loads are in flight together.  The warp folds its lanes by recursive halving (each step
// exchanges half of the values still held), and the item's eight sums go into the CTA's FP64 accumulators in
// shared memory (an item belongs to one warp: no atomics).  Partner rows are shared by many lags and stay in L1.
// When the frame has fewer tiles than resident CTAs the items are also split over `ig` CTA groups (item = g + ig *
// local index).  k_tilt_sum adds the CTAs' FP64 sums in a fixed order and divides by the pair count.
constexpr int TILT_R = 8, TILT_C = 128, TILT_THREADS = 256;

__global__ void __launch_bounds__(TILT_THREADS) k_tilt_partial(const float* __restrict__ a, int H, int W,
                                                               int max_lag, int ntx, int ntiles, int ig,
                                                               double* __restrict__ part) {
  constexpr int CI = TILT_C / 32;
  extern __shared__ double sacc[];  // [local item][8]
  const int items = 2 * (max_lag + 1);
  const int g = blockIdx.y;
  const int nloc = (items - g + ig - 1) / ig;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < nloc * 8; i += TILT_THREADS) sacc[i] = 0.0;
  __syncthreads();
  const size_t plane = (size_t)H * W;
  const uint64_t zero = dfp2s_pk(0.f, 0.f);
  const int kk = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);  // the sum lane kk ends with
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int ty = tile / ntx, tx = tile - ty * ntx;
    const int y0 = ty * TILT_R, x0 = tx * TILT_C;
    uint64_t u[TILT_R][CI];
#pragma unroll
    for (int r = 0; r < TILT_R; ++r)
#pragma unroll
      for (int i = 0; i < CI; ++i) {
        const int y = y0 + r, x = x0 + lane + 32 * i;
        const bool in = y < H && x < W;
        const size_t o = in ? (size_t)y * W + x : 0;
        const uint64_t v = dfp2s_pk(__ldg(a + o), __ldg(a + plane + o));
        u[r][i] = in ? v : zero;
      }
    for (int li = warp; li < nloc; li += TILT_THREADS / 32) {
      const int item = g + ig * li;
      const int dir = item > max_lag ? 1 : 0, d = item - dir * (max_lag + 1);
      const int xe = min(x0 + TILT_C, dir ? W : W - d);  // pairs need x + d < W (dir 0) ...
      const int ye = min(y0 + TILT_R, dir ? H - d : H);  // ... or y + d < H (dir 1)
      const size_t off = dir ? (size_t)d * W : (size_t)d;
      // (a2 a2', a3 a3'), (da2^2, da3^2), (a2^2, a3^2), (a2'^2, a3'^2)
      uint64_t suv = zero, sdd = zero, suu = zero, svv = zero;
      const int xl = x0 + lane;
      if (y0 + TILT_R <= ye && x0 + TILT_C <= xe) {  // every pair of the tile: no guards, all loads in flight
#pragma unroll
        for (int r = 0; r < TILT_R; ++r)
#pragma unroll
          for (int i = 0; i < CI; ++i) {
            const size_t o = (size_t)(y0 + r) * W + xl + 32 * i + off;
            const uint64_t v = dfp2s_pk(__ldg(a + o), __ldg(a + plane + o));
            const uint64_t dd = dfp2s_sub2(u[r][i], v);
            suv = dfp2s_fma2(u[r][i], v, suv);
            sdd = dfp2s_fma2(dd, dd, sdd);
            suu = dfp2s_fma2(u[r][i], u[r][i], suu);
            svv = dfp2s_fma2(v, v, svv);
          }
      } else {  // the window's edge: pairs outside it load element 0 and add zeros
#pragma unroll
        for (int r = 0; r < TILT_R; ++r)
#pragma unroll
          for (int i = 0; i < CI; ++i) {
            const bool in = y0 + r < ye && xl + 32 * i < xe;
            const size_t o = in ? (size_t)(y0 + r) * W + xl + 32 * i + off : 0;
            uint64_t v = dfp2s_pk(__ldg(a + o), __ldg(a + plane + o));
            v = in ? v : zero;
            const uint64_t uv = in ? u[r][i] : zero;
            const uint64_t dd = dfp2s_sub2(uv, v);
            suv = dfp2s_fma2(uv, v, suv);
            sdd = dfp2s_fma2(dd, dd, sdd);
            suu = dfp2s_fma2(uv, uv, suu);
            svv = dfp2s_fma2(v, v, svv);
          }
      }
      const float2 p0 = dfp2s_upk(suv), p1 = dfp2s_upk(sdd), p2 = dfp2s_upk(suu), p3 = dfp2s_upk(svv);
      const float s[8] = {p0.x, p0.y, p1.x, p1.y, p2.x, p3.x, p2.y, p3.y};
      float t4[4], t2[2];
      const bool h4 = lane & 16, h3 = lane & 8, h2 = lane & 4;
#pragma unroll
      for (int k = 0; k < 4; ++k)
        t4[k] = (h4 ? s[k + 4] : s[k]) + __shfl_xor_sync(0xffffffffu, h4 ? s[k] : s[k + 4], 16);
#pragma unroll
      for (int k = 0; k < 2; ++k)
        t2[k] = (h3 ? t4[k + 2] : t4[k]) + __shfl_xor_sync(0xffffffffu, h3 ? t4[k] : t4[k + 2], 8);
      float t = (h2 ? t2[1] : t2[0]) + __shfl_xor_sync(0xffffffffu, h2 ? t2[0] : t2[1], 4);
      t += __shfl_xor_sync(0xffffffffu, t, 2);
      t += __shfl_xor_sync(0xffffffffu, t, 1);
      if ((lane & 3) == 0) sacc[li * 8 + kk] += (double)t;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nloc * 8; i += TILT_THREADS) {
    const int li = i >> 3, k = i & 7;
    part[((size_t)(g + ig * li) * 8 + k) * gridDim.x + blockIdx.x] = sacc[i];
  }
}

// one CTA per (item, sum): the nb CTA sums of that item in FP64, divided by the item's pair count
__global__ void __launch_bounds__(256) k_tilt_sum(const double* __restrict__ part, int nb, int H, int W,
                                                  int max_lag, double* __restrict__ out) {
  __shared__ double red[8];
  const int e = blockIdx.x;
  const int item = e >> 3;
  const int dir = item > max_lag ? 1 : 0, d = item - dir * (max_lag + 1);
  double acc = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) acc += part[(size_t)e * nb + b];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    const double n = dir == 0 ? (double)H * (W - d) : (double)(H - d) * W;
    out[e] = t / n;
  }
}

}  // namespace

int dfp2s_launch_aperture_statistics(const float* fields, int J, int H, int W, int step, double* out, cudaStream_t st) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int nx = (W + step - 1) / step, ny = (H + step - 1) / step;
  const long long nreal = (long long)nx * ny;
  const int nb = (int)(nreal < sms ? nreal : sms);
  float* Z = nullptr;
  float2* tw = nullptr;
  double *part = nullptr, *sums = nullptr;
  double2* T1 = nullptr;
  auto release = [&]() {
    if (Z) cudaFreeAsync(Z, st);
    if (tw) cudaFreeAsync(tw, st);
    if (part) cudaFreeAsync(part, st);
    if (sums) cudaFreeAsync(sums, st);
    if (T1) cudaFreeAsync(T1, st);
  };
  if (dfp2s_device_malloc_async((void**)&Z, (size_t)J * WQ * sizeof(float), st) != cudaSuccess ||
      dfp2s_device_malloc_async((void**)&tw, GN * sizeof(float2), st) != cudaSuccess ||
      dfp2s_device_malloc_async((void**)&part, (size_t)nb * NPART * sizeof(double), st) != cudaSuccess ||
      dfp2s_device_malloc_async((void**)&sums, (size_t)2 * GN * GN * sizeof(double), st) != cudaSuccess ||
      dfp2s_device_malloc_async((void**)&T1, (size_t)2 * GN * GN * sizeof(double2), st) != cudaSuccess) {
    release();
    return DFP2S_ENOMEM;
  }
  const size_t smem = sizeof(ApSmem);
  cudaFuncSetAttribute(k_aperture_partial, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_aperture_tables<<<(J * WQ + 255) / 256, 256, 0, st>>>(J, Z, tw);
  k_aperture_partial<<<nb, THREADS, smem, st>>>(fields, J, H, W, step, nx, nreal, Z, tw, part);
  k_aperture_sum<<<(NPART + 255) / 256, 256, 0, st>>>(part, nb, nreal, sums, out);
  k_otf_rows<<<dim3(GN, 2), GN, 0, st>>>(sums, T1);
  k_otf_cols<<<dim3(GN, 2), GN, 0, st>>>(T1, out + 2 * SFL);
  const bool ok = dfp2s_launch_status() == DFP2S_OK;
  release();
  return ok ? DFP2S_OK : DFP2S_ECUDA;
}

int dfp2s_launch_tilt_statistics(const float* fields, int H, int W, int max_lag, double* out, cudaStream_t st) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int items = 2 * (max_lag + 1);
  const int ntx = (W + TILT_C - 1) / TILT_C, nty = (H + TILT_R - 1) / TILT_R;
  const int ntiles = ntx * nty;
  // CTAs resident per SM (the kernel is register-limited; the shared accumulators grow with the lags)
  const size_t smem1 = (size_t)items * 8 * sizeof(double);  // one group: at most 2050 x 64 B (max_lag <= 1024)
  if (smem1 > 48 * 1024) cudaFuncSetAttribute(k_tilt_partial, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem1);
  int resident = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, k_tilt_partial, TILT_THREADS, smem1);
  if (resident < 1) resident = 1;
  // fewer tiles than resident CTAs: split the items over CTA groups as well
  int ig = ntiles >= resident * sms ? 1 : (resident * sms + ntiles - 1) / ntiles;
  if (ig > items) ig = items;
  const size_t smem = (size_t)((items + ig - 1) / ig) * 8 * sizeof(double);
  const int nb = ntiles < sms * resident ? ntiles : sms * resident;
  double* part = nullptr;
  if (dfp2s_device_malloc_async((void**)&part, (size_t)items * 8 * nb * sizeof(double), st) != cudaSuccess)
    return DFP2S_ENOMEM;
  k_tilt_partial<<<dim3(nb, ig), TILT_THREADS, smem, st>>>(fields, H, W, max_lag, ntx, ntiles, ig, part);
  k_tilt_sum<<<items * 8, 256, 0, st>>>(part, nb, H, W, max_lag, out);
  const bool ok = dfp2s_launch_status() == DFP2S_OK;
  cudaFreeAsync(part, st);
  return ok ? DFP2S_OK : DFP2S_ECUDA;
}
