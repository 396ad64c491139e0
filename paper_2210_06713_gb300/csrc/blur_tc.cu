// Basis blur on the tcgen05 tensor cores (BF16 operands, FP32 accumulation in
// TMEM), Eq. (varying blur):
//
//   out_c(y, x) = sum_k w_k(y, x) conv_k,c(y, x),
//   conv_k,c(y, x) = sum_{iy, ix} phi_k(iy, ix) I_c(y + 16 - iy, x + 16 - ix)   (clamp to edge)
//
// For one output row y and 128 consecutive pixels x0..x0+127 (M = 128) the
// 33 x 33 taps are split into two dense contractions with N = NP filters:
//
//   rows:    D[p][k] += sum_{kappa < 32} A_iy[p][kappa] B_iy[k][kappa]   for each basis row iy,
//            A_iy[p][kappa] = I_c(y + 16 - iy, x0 - 16 + p + kappa),  B_iy[k][kappa] = phi_k(iy, 32 - kappa)
//            (taps ix = 1..32: K = 32, two K = 16 MMAs, no padding);
//   column:  D[p][k] += sum_iy L[p][iy] C[k][iy],
//            L[p][iy] = I_c(y + 16 - iy, x0 + 16 + p),  C[k][iy] = phi_k(iy, 0)
//            (the remaining tap ix = 0 of every row: K = 33 padded to 48, three MMAs);
//
// 69 MMAs per channel per tile, the fewest K = 16 steps that hold 1089 taps.
// A_iy needs no im2col: its K-major core matrix (8 rows x 16 bytes) at (row
// group i, K group g) is the 8 x 8 block E_{i+g}[s][t] = I_c(r, x0 - 16 +
// 8(i+g) + s + t), so the blocks E_0..E_19 of an image row, back to back,
// serve as A_iy with the same 128-byte stride along M and K.  Row s of E_b is
// the 16-byte run at x0 - 16 + 8b + s, which is 16-byte aligned in the image
// copy shifted left by s columns; with eight shifted copies of the padded image
// in global memory one TMA tile load (box 8 x 8 shifts x 20 blocks) writes the
// blocks of one row and channel straight into shared memory.  L is built by two
// warps of its own from the unshifted copy in global memory (each image row's
// 128 values are one contiguous 256-byte run, resident in L2), transposed in
// registers into its core matrices.
// The row tiles of B for each iy are laid out once per basis in global memory
// and streamed with 1-D bulk copies; C stays in shared memory, and so do the
// tile's weights (one bulk copy per tile).  The epilogue reads D from TMEM (one
// pixel per thread, one warp group per channel) and contracts it with the
// pixel's weights: out = sum_k w_k (D[p][k] + c s_k).
//
// Precision: the image enters as bfloat16(I - c) with c = 0.5 (centring halves
// the magnitudes of [0, 1] images and so the rounding error), and the term
// c s_k, s_k = sum_u bf16(phi_k(u)), is added back inside the column
// contraction: its K columns 33, 34, 35 (padding of the 33 taps) hold ones in
// L and a three-part bfloat16 split of c s_k in C (exact to about 2^-25
// relative); the weights are read in FP32 or BF16 as stored.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "kernels.h"
#include "tilt.cuh"
#include "umma.cuh"

namespace {

constexpr int KS = 33;
constexpr int TM = 128;              // pixels per tile (MMA M)
constexpr int KM = 32;               // row taps ix = 1..32 (two K = 16 steps)
constexpr int KL = 48;               // column taps iy = 0..32 padded to three K = 16 steps
constexpr int NBLK = 19;             // blocks E_0..E_18 per image row (the two K = 16 steps reach E_18)
constexpr int ROWB = NBLK * 128;     // 2432 bytes per row and channel
constexpr int NSHIFT = 8;            // shifted image copies
constexpr int CMAX = 3;              // channels per pass
constexpr int NSLOT = 4;             // TMEM accumulator slots of NP <= 128 columns (512 in all)
// warp 0: copies; warp 1: MMA issue; warps 2-3: column operand; warps 4-15:
// epilogue, one group of four per channel (warp w reads TMEM lanes 32 (w % 4) ..)
constexpr int L_WARP0 = 2;
constexpr int NL_WARPS = 2;
constexpr int EPI_WARP0 = 4;
constexpr int THREADS = (EPI_WARP0 + 4 * CMAX) * 32;
constexpr int NB = 7;                // operand ring: one slot per basis row iy (its image row blocks and basis tile)
constexpr uint64_t kWaitNs = 2000000000ull;  // 2 s bound on any wait
constexpr int B_SLOT = 128 * KM * 2;         // bytes of one basis-tile slot (NP <= 128)
constexpr int L_BYTES = TM * KL * 2;         // column operand of one channel
constexpr int C_BYTES = 128 * KL * 2;        // column taps of the basis

struct Slot {
  uint8_t A[CMAX][ROWB];           // Hankel blocks of one image row per channel (TMA)
  uint8_t B[B_SLOT];               // the basis row tile
};
struct Smem {
  Slot ring[NB];                   // operand ring, one basis row per slot
  uint8_t L[CMAX][L_BYTES];        // column operand of the tile
  uint8_t Cb[C_BYTES];             // column taps (resident)
  float Wt[TM * 128];              // the tile's weights (FP32, K per pixel)
  uint64_t full[NB], empty[NB];
  uint64_t l_full, l_free;
  uint64_t c_full, w_full, w_empty, drain;
  uint64_t acc_full[NSLOT], acc_empty[NSLOT];
  uint32_t tmem_base;
  int abort;
};

// Warp-wide load of 16 TMEM columns without waiting; tmem_wait_ld4 waits for all
// outstanding loads and ties the destination registers to the wait, so that no
// use of them is scheduled before it.
DFP2S_DEV void tmem_ld16_async(uint32_t taddr, float* v) {
  uint32_t* r = reinterpret_cast<uint32_t*>(v);
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
DFP2S_DEV void tmem_wait_ld4(float (&d)[4][16]) {
  uint32_t* r = reinterpret_cast<uint32_t*>(&d[0][0]);
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]),
                 "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]),
                 "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31]),
                 "+r"(r[32]), "+r"(r[33]), "+r"(r[34]), "+r"(r[35]), "+r"(r[36]), "+r"(r[37]), "+r"(r[38]), "+r"(r[39]),
                 "+r"(r[40]), "+r"(r[41]), "+r"(r[42]), "+r"(r[43]), "+r"(r[44]), "+r"(r[45]), "+r"(r[46]), "+r"(r[47]),
                 "+r"(r[48]), "+r"(r[49]), "+r"(r[50]), "+r"(r[51]), "+r"(r[52]), "+r"(r[53]), "+r"(r[54]), "+r"(r[55]),
                 "+r"(r[56]), "+r"(r[57]), "+r"(r[58]), "+r"(r[59]), "+r"(r[60]), "+r"(r[61]), "+r"(r[62]), "+r"(r[63])
               :
               : "memory");
}

// TMA tile load of a rank-5 box into shared memory, completion counted in bytes on `bar`.
DFP2S_DEV void tma_load_5d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3, int c4, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
      "%6}], [%7];" ::"r"(umma::smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(umma::smem_u32(bar))
      : "memory");
}

// Replicate-padded, shifted BF16 copies of the image:
// P[c][sh][r][x] = I[c][clamp(r - 16)][clamp(x + sh - 16)] - centre, sh = 0..7, r < H + 32, x < Wq.
__global__ void k_pad_shifted(const float* __restrict__ img, int C, int H, int W, int Wq, float centre,
                              __nv_bfloat16* __restrict__ P) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  const int c = blockIdx.z;
  if (x >= Wq) return;
  const int R = H + 32;
  const int sy = min(max(r - 16, 0), H - 1);
  const float* row = img + ((size_t)c * H + sy) * W;
  const size_t plane = (size_t)R * Wq;
  __nv_bfloat16* dst = P + (size_t)c * NSHIFT * plane + (size_t)r * Wq + x;
#pragma unroll
  for (int sh = 0; sh < NSHIFT; ++sh) {
    const int sx = min(max(x + sh - 16, 0), W - 1);
    dst[sh * plane] = __float2bfloat16_rn(row[sx] - centre);
  }
}

// The same planes for the tilt-warped image, without the FP32 warped image: the
// value at padded (r, x) of shift sh is the warped pixel (clamp(r - 16),
// clamp(x + sh - 16)) (tilt_sample, as in the warp kernel).  One CTA per padded
// row and channel: the row's warped samples at clamped columns i - 16,
// i < Wq + 7, go to shared memory once (as bfloat16 bits; eight samples per
// thread at a time, their tilt loads and then their gathers all in flight),
// then each thread takes sixteen consecutive samples with two 16-byte loads and
// writes the eight shifted 16-byte runs of its eight columns (funnel shifts for
// the odd shifts; consecutive threads, consecutive runs of each shift plane).
__global__ void __launch_bounds__(128)
    k_warp_pad_shifted(const float* __restrict__ img, int C, int H, int W, const float* __restrict__ a2,
                       const float* __restrict__ a3, int Wq, float centre, __nv_bfloat16* __restrict__ P, int mixed,
                       float m00, float m10, float m11) {
  extern __shared__ __align__(16) unsigned short wrow[];  // Wq + 8 entries
  const int r = blockIdx.x, c = blockIdx.y;
  const int R = H + 32;
  const int yp = min(max(r - 16, 0), H - 1);
  const size_t plane = (size_t)R * Wq;
  const float* t2 = a2 + (size_t)yp * W;
  const float* t3 = a3 + (size_t)yp * W;
  const float* I = img + (size_t)c * H * W;
  const int n = Wq + 7;
  if (threadIdx.x == 0) wrow[n] = 0;
  for (int base = 0; base < n; base += 8 * blockDim.x) {
    float s2[8], s3[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int i = base + k * blockDim.x + threadIdx.x;
      const int x = min(max(i - 16, 0), W - 1);
      s2[k] = i < n ? __ldg(t2 + x) : 0.f;
      s3[k] = i < n ? __ldg(t3 + x) : 0.f;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int i = base + k * blockDim.x + threadIdx.x;
      if (i < n) {
        const int x = min(max(i - 16, 0), W - 1);
        float u2 = s2[k], u3 = s3[k];
        if (mixed) {  // the tilt rows of a = scale L u, in the mixing kernel's operation order
          u3 = fmaf(m11, u3, fmaf(m10, u2, 0.f));
          u2 = fmaf(m00, u2, 0.f);
        }
        const float v = tilt_sample(I, H, W, x, yp, u2, u3);
        wrow[i] = __bfloat16_as_ushort(__float2bfloat16_rn(v - centre));
      }
    }
  }
  __syncthreads();
  const int runs = Wq / 8;
  __nv_bfloat16* dst = P + ((size_t)c * NSHIFT) * plane + (size_t)r * Wq;
  const uint4* w4 = reinterpret_cast<const uint4*>(wrow);
  for (int u = threadIdx.x; u < runs; u += blockDim.x) {
    const uint4 lo = w4[u], hi = w4[u + 1];  // samples 8u .. 8u + 15 (the last run reads up to Wq + 7)
    const uint32_t w[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
    for (int sh = 0; sh < NSHIFT; ++sh) {
      const int m = sh >> 1;
      uint4 v;
      if (sh & 1) {
        v = make_uint4(__funnelshift_r(w[m], w[m + 1], 16), __funnelshift_r(w[m + 1], w[m + 2], 16),
                       __funnelshift_r(w[m + 2], w[m + 3], 16), __funnelshift_r(w[m + 3], w[m + 4], 16));
      } else {
        v = make_uint4(w[m], w[m + 1], w[m + 2], w[m + 3]);
      }
      *reinterpret_cast<uint4*>(dst + sh * plane + 8 * u) = v;
    }
  }
}

// Row tiles: Bt[iy][j][g][n8][k8] = phi_{8j+n8}(iy, 32 - (8g+k8)), g < 4 (taps ix = 1..32),
// then the column taps Ct[j][g][n8][k8] = phi_{8j+n8}(8g+k8, 0), g < 6, with the rows 8g+k8 = 33, 34, 35
// holding the bfloat16 parts hi, mid, lo of the centring term cs_k (cs_k = hi + mid + lo to about 2^-25);
// zero outside.
__global__ void k_build_bt(const float* __restrict__ basis, int K, int NP, const float* __restrict__ cs,
                           __nv_bfloat16* __restrict__ Bt) {
  const int per_iy = NP * KM;
  const int nrow = KS * per_iy;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nrow + NP * KL) return;
  float v = 0.f;
  if (i < nrow) {
    const int iy = i / per_iy;
    int rem = i - iy * per_iy;
    const int j = rem / (KM * 8);
    rem -= j * KM * 8;
    const int g = rem / 64;
    rem -= g * 64;
    const int n8 = rem / 8, k8 = rem - n8 * 8;
    const int k = 8 * j + n8, kap = 8 * g + k8;
    if (k < K) v = basis[((size_t)k * KS + iy) * KS + (KS - 1 - kap)];
  } else {
    int rem = i - nrow;
    const int j = rem / (KL * 8);
    rem -= j * KL * 8;
    const int g = rem / 64;
    rem -= g * 64;
    const int n8 = rem / 8, k8 = rem - n8 * 8;
    const int k = 8 * j + n8, iy = 8 * g + k8;
    if (k < K && iy < KS) v = basis[((size_t)k * KS + iy) * KS];
    if (k < K && iy >= KS && iy < KS + 3) {
      const float c = cs[k];
      const float hi = __bfloat162float(__float2bfloat16_rn(c));
      const float mid = __bfloat162float(__float2bfloat16_rn(c - hi));
      v = iy == KS ? hi : (iy == KS + 1 ? mid : c - hi - mid);
    }
  }
  Bt[i] = __float2bfloat16_rn(v);
}

// s_k = sum over the 33 x 33 taps of the bfloat16-rounded basis function k (zero for k >= K)
__global__ void k_basis_sums(const float* __restrict__ basis, int K, int NP, float* __restrict__ sums) {
  __shared__ float red[8];
  const int k = blockIdx.x;
  float t = 0.f;
  if (k < K)
    for (int i = threadIdx.x; i < KS * KS; i += blockDim.x)
      t += __bfloat162float(__float2bfloat16_rn(basis[(size_t)k * KS * KS + i]));
  for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(0xffffffffu, t, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    float a = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) a += red[i];
    sums[k] = a;
  }
}

template <typename WT>
DFP2S_DEV float wload(const WT* p);
template <>
DFP2S_DEV float wload<float>(const float* p) { return __ldg(p); }
template <>
DFP2S_DEV float wload<__nv_bfloat16>(const __nv_bfloat16* p) { return __bfloat162float(*p); }

__global__ void k_scale(float* __restrict__ v, int n, float a) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] *= a;
}

template <typename WT, int C>
__global__ void __launch_bounds__(THREADS, 1)
    k_blur_tc(const __grid_constant__ CUtensorMap tmap, int H, int W, const __nv_bfloat16* __restrict__ Bt, int K,
              int NP, const __nv_bfloat16* __restrict__ planes, int Wq, size_t chan_stride,
              const WT* __restrict__ w, int w_vec, float* __restrict__ out, int* __restrict__ err) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // 1024-byte aligned base in the shared window (the launch adds 1024 bytes of slack)
  uint8_t* sbase = smem_raw + ((1024u - (umma::smem_u32(smem_raw) & 1023u)) & 1023u);
  Smem& s = *reinterpret_cast<Smem*>(sbase);
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const uint32_t bt_bytes = (uint32_t)NP * KM * 2;
  const uint32_t ct_bytes = (uint32_t)NP * KL * 2;
  const __nv_bfloat16* Ct = Bt + (size_t)KS * NP * KM;
  const uint32_t idesc = umma::idesc_bf16(TM, NP);
  const int nseg = (W + TM - 1) / TM;
  const int ntiles = H * nseg;
  const int my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

  if (tid == 0) {
    for (int i = 0; i < NB; ++i) {
      umma::mbar_init(&s.full[i], 1);   // the producer's expect_tx: image row blocks and basis tile
      umma::mbar_init(&s.empty[i], 1);  // the MMAs' commit
    }
    umma::mbar_init(&s.l_full, NL_WARPS);
    umma::mbar_init(&s.l_free, 1);
    umma::mbar_init(&s.c_full, 1);
    umma::mbar_init(&s.w_full, 1);
    umma::mbar_init(&s.w_empty, 4 * C);
    umma::mbar_init(&s.drain, 1);
    for (int i = 0; i < NSLOT; ++i) {
      umma::mbar_init(&s.acc_full[i], 1);
      umma::mbar_init(&s.acc_empty[i], 4);
    }
    s.abort = 0;
    umma::fence_mbar_init();
  }
  // the column operand's padding K columns (iy = 36..47) stay zero
  for (int i = tid; i < CMAX * L_BYTES / 16; i += THREADS) reinterpret_cast<uint4*>(&s.L[0][0])[i] = make_uint4(0, 0, 0, 0);
  if (warp == 0) {
    umma::tmem_alloc(&s.tmem_base, 512);
    umma::tmem_relinquish();
  }
  umma::fence_proxy_async_smem();
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = s.tmem_base;
  auto tile_xy = [&](int t_local, int& y, int& x0) {
    const int tile = blockIdx.x + t_local * gridDim.x;
    y = tile / nseg;
    x0 = (tile - y * nseg) * TM;
  };

  if (warp == 0) {
    // ---------------------------------------------------------- copies (one lane)
    // The ring position (slot, round) is kept in counters: this thread and the MMA thread run a tight loop
    // each, and the MMA thread's instruction latency bounds the tensor cores' rate.
    if (lane == 0) {
      bool ok = true;
      uint32_t slot = 0, round = 0, issued = 0;  // ring position; operand rows issued
      int w_issued = 0;                          // weight tiles issued
      const uint32_t row_tx = (uint32_t)(C * ROWB) + bt_bytes;
      umma::mbar_arrive_expect_tx(&s.c_full, ct_bytes);
      umma::bulk_g2s(s.Cb, Ct, ct_bytes, &s.c_full);
      auto issue_w = [&](int t) {
        int y, x0;
        tile_xy(t, y, x0);
        const int nlive = min(TM, W - x0);
        const uint32_t bytes = (uint32_t)(nlive * K * 4);
        umma::mbar_arrive_expect_tx(&s.w_full, bytes);
        umma::bulk_g2s(s.Wt, w + ((size_t)y * W + x0) * K, bytes, &s.w_full);
        w_issued = t + 1;
      };
      for (int t = 0; t < my_tiles && ok; ++t) {
        int y, x0;
        tile_xy(t, y, x0);
        const int xb = x0 >> 3;
        const __nv_bfloat16* bsrc = Bt;
        for (int iy = 0; iy < KS; ++iy, bsrc += NP * KM) {
          // (a sleep between polls: a spinning wait slows the MMA thread's barrier operations)
          if (issued >= NB && !umma::mbar_wait_backoff(&s.empty[slot], (round - 1) & 1, kWaitNs, 64)) {
            ok = false;
            break;
          }
          Slot& sl = s.ring[slot];
          umma::mbar_arrive_expect_tx(&s.full[slot], row_tx);
#pragma unroll
          for (int c = 0; c < C; ++c) tma_load_5d(sl.A[c], &tmap, 0, 0, xb, y + (KS - 1 - iy), c, &s.full[slot]);
          umma::bulk_g2s(sl.B, bsrc, bt_bytes, &s.full[slot]);
          ++issued;
          if (++slot == NB) {
            slot = 0;
            ++round;
          }
          // this tile's weights, once the epilogue of the previous tile has released the buffer
          if (w_vec && w_issued == t && iy >= 2) {
            if (t == 0 || umma::mbar_ready(&s.w_empty, (t - 1) & 1)) {
              issue_w(t);
            } else if (iy == KS - 1) {
              if (!umma::mbar_wait(&s.w_empty, (t - 1) & 1, kWaitNs)) {
                ok = false;
                break;
              }
              issue_w(t);
            }
          }
        }
      }
      if (!ok) {
        s.abort = 1;
        atomicExch(err, 1);
      }
      // every issued copy must land before the CTA exits (bounded)
      umma::mbar_wait(&s.c_full, 0, kWaitNs);
      for (uint32_t u = (issued >= NB ? issued - NB : 0); u < issued; ++u)
        umma::mbar_wait(&s.full[u % NB], (u / NB) & 1, kWaitNs);
      if (w_issued > 0) umma::mbar_wait(&s.w_full, (w_issued - 1) & 1, kWaitNs);
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------- MMA issue (whole warp, one elected lane)
    // The warp runs the loop together (its waits and branches are warp-uniform: every wait's outcome goes
    // through a vote) and one elected lane issues the MMAs and commits; the issuing thread's instruction
    // latency, not the tensor cores, bounds a stream of these MMAs, and a loop run by one lane of a warp
    // whose other lanes have left costs it more per MMA.
    {
      const bool leader = umma::elect_one();
      // row blocks: core matrices 128 B apart along M and K (Hankel); row tiles [j][g][8][8]: K-adjacent
      // core matrices 128 B apart, 8-filter groups 512 B apart; column operand [p/8][g][8][8] and
      // column taps [j][g][8][8]: 128 B along K, 768 B along M/N.  Descriptors = base + (byte offset >> 4).
      const uint64_t a_base = umma::sdesc(umma::smem_u32(s.ring[0].A[0]), 128, 128);
      const uint64_t b_base = umma::sdesc(umma::smem_u32(s.ring[0].B), 128, KM / 8 * 128);
      const uint64_t l_base = umma::sdesc(umma::smem_u32(s.L[0]), 128, KL / 8 * 128);
      const uint64_t c_desc = umma::sdesc(umma::smem_u32(s.Cb), 128, KL / 8 * 128);
      constexpr uint32_t SLOT16 = sizeof(Slot) >> 4, ROW16 = ROWB >> 4, L16 = L_BYTES >> 4;
      bool ok = __all_sync(0xffffffffu, my_tiles == 0 || umma::mbar_wait(&s.c_full, 0, kWaitNs));
      uint32_t slot = 0, par = 0;           // ring slot and the parity of its current use
      uint64_t a_s = a_base, b_s = b_base;  // descriptors of the current slot
      for (int t = 0; t < my_tiles && ok; ++t) {
        uint32_t dch[C];
        bool got = true;
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const uint32_t g = (uint32_t)(t * C + c);
          dch[c] = tmem + (g % NSLOT) * NP;
          // a reused accumulator slot: the epilogue has read it out
          if (g >= NSLOT) got = got && umma::mbar_wait(&s.acc_empty[g % NSLOT], ((g / NSLOT) - 1) & 1, kWaitNs);
        }
        if (!__all_sync(0xffffffffu, got)) {
          ok = false;
          break;
        }
        umma::fence_after_sync();
        uint32_t acc = 0;  // the first row starts the accumulators
        for (int iy = 0; iy < KS; ++iy) {
          if (!__all_sync(0xffffffffu, umma::mbar_wait(&s.full[slot], par, kWaitNs))) {
            ok = false;
            break;
          }
          umma::fence_after_sync();
          if (leader) {
#pragma unroll
            for (int c = 0; c < C; ++c) {
              umma::mma_bf16(dch[c], a_s + c * ROW16, b_s, idesc, acc);
              umma::mma_bf16(dch[c], a_s + c * ROW16 + 16, b_s + 16, idesc, 1);
            }
            umma::mma_commit(&s.empty[slot]);
          }
          acc = 1;
          if (++slot == NB) {
            slot = 0;
            par ^= 1;
            a_s = a_base;
            b_s = b_base;
          } else {
            a_s += SLOT16;
            b_s += SLOT16;
          }
        }
        if (!ok) break;
        // the column taps, once the tile's column operand is complete
        if (!__all_sync(0xffffffffu, umma::mbar_wait(&s.l_full, t & 1, kWaitNs))) {
          ok = false;
          break;
        }
        umma::fence_after_sync();
        if (leader) {
#pragma unroll
          for (int c = 0; c < C; ++c) {
            const uint64_t l_c = l_base + c * L16;
            umma::mma_bf16(dch[c], l_c, c_desc, idesc, 1);
            umma::mma_bf16(dch[c], l_c + 16, c_desc + 16, idesc, 1);
            umma::mma_bf16(dch[c], l_c + 32, c_desc + 32, idesc, 1);
          }
          umma::mma_commit(&s.l_free);
#pragma unroll
          for (int c = 0; c < C; ++c) umma::mma_commit(&s.acc_full[(t * C + c) % NSLOT]);
        }
      }
      if (!ok) {
        if (leader) {
          s.abort = 1;
          atomicExch(err, 1);
          // the MMAs issued so far complete before the tensor memory is released (bounded)
          umma::mma_commit(&s.drain);
          umma::mbar_wait(&s.drain, 0, kWaitNs);
        }
      } else if (my_tiles > 0 && leader) {
        const int t = my_tiles - 1;  // the last MMAs have completed before the CTA exits
        umma::mbar_wait(&s.l_free, t & 1, kWaitNs);
      }
    }
  } else if (warp < EPI_WARP0) {
    // ---------------------------------------------------------- column operand L
    // L[p][iy] = P[c][0][y + 32 - iy][x0 + 32 + p] (the unshifted padded plane).  Thread (c, m) loads, for
    // eight basis rows iy = 8 g + e, the pixels p = 8 m .. 8 m + 7 (one 16-byte load per row, 16 threads
    // read a row's 256 contiguous bytes), transposes the 8 x 8 tile in registers and writes the core matrix
    // L[8 m .. 8 m + 7][8 g .. 8 g + 7], its eight 16-byte rows in an order rotated by m so that the 16
    // threads of a channel hit distinct banks.  Columns 33, 34, 35 hold ones (the centring term's factor).
    const int lt = tid - L_WARP0 * 32;
    const int lc = lt >> 4, m = lt & 15;
    const bool active = lc < C;
    const __nv_bfloat16* plane = planes + (size_t)(active ? lc : 0) * chan_stride;
    for (int t = 0; t < my_tiles && !s.abort; ++t) {
      int y, x0;
      tile_xy(t, y, x0);
      const __nv_bfloat16* src = plane + (size_t)(y + 32) * Wq + x0 + 32 + 8 * m;
      // the column operand was last read by the column MMAs of tile t - 1
      if (t >= 1 && !umma::mbar_wait_backoff(&s.l_free, (t - 1) & 1, kWaitNs, 256)) s.abort = 1;
      if (s.abort) break;
      for (int g = 0; g < (KS + 3 + 7) / 8; ++g) {
        uint4 win[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int iy = 8 * g + e;
          if (iy < KS) win[e] = active ? __ldg(reinterpret_cast<const uint4*>(src - (size_t)iy * Wq)) : make_uint4(0, 0, 0, 0);
          else if (iy < KS + 3) win[e] = make_uint4(0x3F803F80u, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u);
          else win[e] = make_uint4(0, 0, 0, 0);
        }
        if (active) {
          // row j of the transposed tile: element e is bf16 j of win[e] (word j / 2, half j % 2)
          uint8_t* dst = s.L[lc] + (m * (KL / 8) + g) * 128;
          auto comp = [](const uint4& v, int q) { return q == 0 ? v.x : (q == 1 ? v.y : (q == 2 ? v.z : v.w)); };
#pragma unroll
          for (int jp = 0; jp < 8; ++jp) {
            const int j = (jp + m) & 7;
            const uint32_t sel = (j & 1) ? 0x7632u : 0x5410u;
            const int wj = j >> 1;
            const uint4 o = make_uint4(__byte_perm(comp(win[0], wj), comp(win[1], wj), sel),
                                       __byte_perm(comp(win[2], wj), comp(win[3], wj), sel),
                                       __byte_perm(comp(win[4], wj), comp(win[5], wj), sel),
                                       __byte_perm(comp(win[6], wj), comp(win[7], wj), sel));
            *reinterpret_cast<uint4*>(dst + j * 16) = o;
          }
        }
      }
      umma::fence_proxy_async_smem();  // L stores -> visible to the tensor cores
      __syncwarp();
      if (lane == 0) umma::mbar_arrive(&s.l_full);
    }
  } else {
    // ---------------------------------------------------------- epilogue: TMEM -> weighted sums, one channel per group
    const int c = (warp - EPI_WARP0) >> 2;
    const int q4 = warp & 3;  // warp w reads TMEM lanes 32 (w % 4) ..
    const int p = q4 * 32 + lane;
    if (c < C) {
      for (int t = 0; t < my_tiles; ++t) {
        int y, x0;
        tile_xy(t, y, x0);
        const int x = x0 + p;
        const bool live = x < W;
        const uint32_t g = (uint32_t)(t * C + c);
        const uint32_t slot = g % NSLOT;
        if (!umma::mbar_wait_backoff(&s.acc_full[slot], (g / NSLOT) & 1, kWaitNs, 128)) s.abort = 1;
        if (w_vec && !umma::mbar_wait_backoff(&s.w_full, t & 1, kWaitNs)) s.abort = 1;
        if (s.abort) break;
        umma::fence_after_sync();
        float acc = 0.f;
        const float* ws = s.Wt + p * K;
        const WT* wg = w + ((size_t)y * W + (live ? x : 0)) * K;
        const uint32_t taddr = tmem + ((uint32_t)(q4 * 32) << 16) + slot * NP;
        const int nq = NP / 16;
        // up to 64 accumulator columns per TMEM round trip (two for NP <= 128)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (4 * h < nq) {
            float d[4][16];
#pragma unroll
            for (int qq = 0; qq < 4; ++qq)
              if (4 * h + qq < nq) tmem_ld16_async(taddr + (4 * h + qq) * 16, d[qq]);
            tmem_wait_ld4(d);
            if (4 * (h + 1) >= nq) {
              // the accumulator is in registers: hand the slot back to the MMAs before the weighted sums
              umma::fence_before_sync();
              __syncwarp();
              if (lane == 0) umma::mbar_arrive(&s.acc_empty[slot]);
            }
#pragma unroll
            for (int qq = 0; qq < 4; ++qq) {
              const int q = 4 * h + qq;
              if (q < nq) {
                float wk[16];
                if (w_vec) {  // the tile's FP32 weights in shared memory
#pragma unroll
                  for (int i4 = 0; i4 < 4; ++i4) {
                    const int k = q * 16 + 4 * i4;
                    const float4 v4 =
                        (k < K && live) ? *reinterpret_cast<const float4*>(ws + k) : make_float4(0.f, 0.f, 0.f, 0.f);
                    wk[4 * i4 + 0] = v4.x;
                    wk[4 * i4 + 1] = v4.y;
                    wk[4 * i4 + 2] = v4.z;
                    wk[4 * i4 + 3] = v4.w;
                  }
                } else {
#pragma unroll
                  for (int i = 0; i < 16; ++i) {
                    const int k = q * 16 + i;
                    wk[i] = k < K ? wload<WT>(wg + k) : 0.f;
                  }
                }
#pragma unroll
                for (int i = 0; i < 16; ++i) acc = fmaf(wk[i], d[qq][i], acc);
              }
            }
          }
        }
        __syncwarp();
        if (lane == 0 && w_vec) umma::mbar_arrive(&s.w_empty);
        if (live) out[((size_t)c * H + y) * W + x] = acc;
      }
    }
  }
  umma::fence_before_sync();
  __syncthreads();
  if (warp == 0) umma::tmem_dealloc(tmem, 512);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)ptr;
  }
  return fn;
}

}  // namespace

// Basis tiles, centring sums and the plane scratch for a C x H x W image (once per handle / size).
static int blur_tc_scratch(dfp2s_p2s_dev* p, int C, int H, int W, cudaStream_t st) {
  const int K = p->K;
  const int NP = (K + 15) / 16 * 16;
  const float centre = 0.5f;
  if (NP > 128) return DFP2S_EUNSUPPORTED;
  if (!p->bt) {
    const int n = KS * NP * KM + NP * KL;  // row tiles, then the column taps
    if (dfp2s_device_malloc((void**)&p->bt, (size_t)n * sizeof(__nv_bfloat16)) != cudaSuccess) return DFP2S_ENOMEM;
    if (dfp2s_device_malloc((void**)&p->bsum, (size_t)NP * sizeof(float)) != cudaSuccess) return DFP2S_ENOMEM;
    k_basis_sums<<<NP, 256, 0, st>>>(p->basis, K, NP, p->bsum);
    k_scale<<<1, 128, 0, st>>>(p->bsum, NP, centre);
    k_build_bt<<<(n + 255) / 256, 256, 0, st>>>(p->basis, K, NP, p->bsum, p->bt);
  }
  if (!p->err) {
    if (dfp2s_device_malloc((void**)&p->err, sizeof(int)) != cudaSuccess) return DFP2S_ENOMEM;
    cudaMemsetAsync(p->err, 0, sizeof(int), st);
  }
  const int nseg = (W + TM - 1) / TM;
  const int Wq = nseg * TM + 64;  // >= x0 + 160 for every tile; a multiple of 8 (16-byte rows)
  const size_t need = (size_t)C * NSHIFT * (H + 32) * Wq;
  if (need > p->pad_cap) {
    if (p->pad) cudaFree(p->pad);
    p->pad = nullptr;
    p->pad_cap = 0;
    if (dfp2s_device_malloc((void**)&p->pad, need * sizeof(__nv_bfloat16)) != cudaSuccess) return DFP2S_ENOMEM;
    p->pad_cap = need;
  }
  return DFP2S_OK;
}

// Shifted BF16 planes of the image in the handle's scratch (k_pad_shifted).
int dfp2s_launch_blur_tc_prepare(dfp2s_p2s_dev* p, const float* img, int C, int H, int W, cudaStream_t st) {
  const int rc = blur_tc_scratch(p, C, H, W, st);
  if (rc != DFP2S_OK) return rc;
  const int Wq = (W + TM - 1) / TM * TM + 64;
  k_pad_shifted<<<dim3((Wq + 255) / 256, H + 32, C), 256, 0, st>>>(img, C, H, W, Wq, 0.5f, p->pad);
  p->prep_C = C;
  p->prep_H = H;
  p->prep_W = W;
  return dfp2s_launch_status();
}

// The same for the tilt-warped image (k_warp_pad_shifted), without writing the warped image.
int dfp2s_launch_blur_tc_prepare_warp(dfp2s_p2s_dev* p, const float* img, int C, int H, int W, const float* a2,
                                      const float* a3, cudaStream_t st, const float* m) {
  const int rc = blur_tc_scratch(p, C, H, W, st);
  if (rc != DFP2S_OK) return rc;
  const int Wq = (W + TM - 1) / TM * TM + 64;
  k_warp_pad_shifted<<<dim3(H + 32, C), 128, (size_t)(Wq + 8) * sizeof(unsigned short), st>>>(
      img, C, H, W, a2, a3, Wq, 0.5f, p->pad, m != nullptr, m ? m[0] : 1.f, m ? m[1] : 0.f, m ? m[2] : 1.f);
  p->prep_C = C;
  p->prep_H = H;
  p->prep_W = W;
  return dfp2s_launch_status();
}

// The tensor-core contraction on the prepared planes.
int dfp2s_launch_blur_tc_run(dfp2s_p2s_dev* p, int C, int H, int W, const void* w, int w_dtype, float* out,
                             cudaStream_t st) {
  const int K = p->K;
  const int NP = (K + 15) / 16 * 16;
  if (NP > 128) return DFP2S_EUNSUPPORTED;
  if (!p->pad || !p->bt || p->prep_C != C || p->prep_H != H || p->prep_W != W) return DFP2S_EINVAL;
  const int nseg = (W + TM - 1) / TM;
  const int Wq = nseg * TM + 64;
  const int R = H + 32;
  const size_t plane = (size_t)R * Wq;
  EncodeTiledFn encode = encode_tiled();
  if (!encode) return DFP2S_EUNSUPPORTED;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int ntiles = H * nseg;
  const int grid = ntiles < sms ? ntiles : sms;
  // more than half of an SM's shared memory: one CTA (and one 512-column TMEM
  // allocation) per SM
  const size_t sm = sizeof(Smem) + 1024;
  static_assert(sizeof(Smem) + 1024 > 116 * 1024 && sizeof(Smem) + 1024 <= 227 * 1024, "smem layout");
  cudaFuncSetAttribute(k_blur_tc<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  cudaFuncSetAttribute(k_blur_tc<float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  cudaFuncSetAttribute(k_blur_tc<float, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  cudaFuncSetAttribute(k_blur_tc<__nv_bfloat16, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  cudaFuncSetAttribute(k_blur_tc<__nv_bfloat16, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  cudaFuncSetAttribute(k_blur_tc<__nv_bfloat16, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  // FP32 weights whose tile rows are 16-byte multiples come in by one bulk copy per tile
  const int w_vec = (w_dtype == DFP2S_W_F32) && (K % 4) == 0 && ((uintptr_t)w & 15) == 0;
  for (int c0 = 0; c0 < C; c0 += CMAX) {
    const int nc = C - c0 < CMAX ? C - c0 : CMAX;
    // rank-5 view of the shifted copies: (t: 8 columns, sh: shift, b: 8-column block, r: row, c: channel)
    CUtensorMap tmap;
    const cuuint64_t dims[5] = {8, NSHIFT, (cuuint64_t)(Wq / 8), (cuuint64_t)R, (cuuint64_t)nc};
    const cuuint64_t strides[4] = {plane * 2, 16, (cuuint64_t)Wq * 2, NSHIFT * plane * 2};
    const cuuint32_t box[5] = {8, NSHIFT, NBLK, 1, 1};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    if (encode(&tmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, p->pad + (size_t)c0 * NSHIFT * plane, dims, strides, box,
               estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return DFP2S_EUNSUPPORTED;
    float* oc = out + (size_t)c0 * H * W;
    const __nv_bfloat16* planes = p->pad + (size_t)c0 * NSHIFT * plane;  // shift 0 of channel c0
#define DFP2S_BLUR_LAUNCH(WT, NC, WPTR, WV)                                                                    \
  k_blur_tc<WT, NC><<<grid, THREADS, sm, st>>>(tmap, H, W, p->bt, K, NP, planes, Wq, (size_t)NSHIFT * plane, WPTR, \
                                               WV, oc, p->err)
    if (w_dtype == DFP2S_W_BF16) {
      const __nv_bfloat16* wb = (const __nv_bfloat16*)w;
      if (nc == 1) DFP2S_BLUR_LAUNCH(__nv_bfloat16, 1, wb, 0);
      else if (nc == 2) DFP2S_BLUR_LAUNCH(__nv_bfloat16, 2, wb, 0);
      else DFP2S_BLUR_LAUNCH(__nv_bfloat16, 3, wb, 0);
    } else {
      const float* wf = (const float*)w;
      if (nc == 1) DFP2S_BLUR_LAUNCH(float, 1, wf, w_vec);
      else if (nc == 2) DFP2S_BLUR_LAUNCH(float, 2, wf, w_vec);
      else DFP2S_BLUR_LAUNCH(float, 3, wf, w_vec);
    }
#undef DFP2S_BLUR_LAUNCH
  }
  return dfp2s_launch_status();
}

int dfp2s_launch_blur_tc(dfp2s_p2s_dev* p, const float* img, int C, int H, int W, const void* w, int w_dtype,
                         float* out, cudaStream_t st) {
  const int rc = dfp2s_launch_blur_tc_prepare(p, img, C, H, W, st);
  if (rc != DFP2S_OK) return rc;
  return dfp2s_launch_blur_tc_run(p, C, H, W, w, w_dtype, out, st);
}
