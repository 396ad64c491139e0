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
// 8(i+g) + s + t), so a staged image row holds the 19 blocks E_0..E_18 back to
// back and the operand descriptor takes the same 128-byte stride along M and K.
// L is gathered once per tile from the same image rows.  B tiles for each iy
// are laid out once per basis in global memory and streamed with 1-D bulk
// copies; C stays in shared memory.  The epilogue reads D from TMEM (one pixel
// per thread, one warp group per channel) and contracts it with the pixel's
// weights: out = sum_k w_k (D[p][k] + c s_k).
//
// Precision: the image enters as bfloat16(I - c) with c = 0.5 (centring halves
// the magnitudes of [0, 1] images and so the rounding error), and the exact
// term c s_k, s_k = sum_u bf16(phi_k(u)), is added back in FP32; the weights
// are read in FP32 or BF16 as stored.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "kernels.h"
#include "umma.cuh"

namespace {

constexpr int KS = 33;
constexpr int TM = 128;                    // pixels per tile (MMA M)
constexpr int KM = 32;                     // row taps ix = 1..32 (two K = 16 steps)
constexpr int KL = 48;                     // column taps iy = 0..32 padded to three K = 16 steps
constexpr int NBLK = TM / 8 + KM / 8 - 1;  // 19 staged 8x8 blocks per image row
constexpr int ROWB = NBLK * 128;           // 2432 bytes per staged row
constexpr int RAWW = TM + KM;              // 160 staged image columns per row (cols p + kappa <= 159)
constexpr int RAWB = RAWW * 2;             // 320 bytes
constexpr int CMAX = 3;                    // channels per pass
constexpr int NSLOT = 4;                   // TMEM accumulator slots of NP <= 128 columns (512 in all)
// warp 0: bulk copies; warp 1: MMA issue; warps 2-7: staging; warps 8-19: epilogue,
// one group of four per channel (warp w reads TMEM lanes 32 (w % 4) ..)
constexpr int STAGE_WARP0 = 2;
constexpr int NSTAGE_WARPS = 6;
constexpr int EPI_WARP0 = STAGE_WARP0 + NSTAGE_WARPS;
constexpr int EPI_WARPS = 4 * CMAX;
constexpr int THREADS = (EPI_WARP0 + EPI_WARPS) * 32;
constexpr int NB = 4;                      // staged-row ring (one slot per basis row iy)
constexpr int NBB = 4;                     // basis-tile ring
constexpr uint64_t kWaitNs = 2000000000ull;  // 2 s bound on any wait
constexpr int B_SLOT = 128 * KM * 2;       // bytes of one basis-tile slot (NP <= 128)
constexpr int L_BYTES = TM * KL * 2;       // column operand of one channel
constexpr int C_BYTES = 128 * KL * 2;      // column taps of the basis

struct Smem {
  uint8_t raw[2][CMAX][KS][RAWB];  // image rows of a tile (bulk copies, prefetched one tile ahead)
  uint8_t A[NB][CMAX][ROWB];       // Hankel-blocked rows
  uint8_t L[CMAX][L_BYTES];        // column operand of the tile
  uint8_t B[NBB][B_SLOT];          // basis tiles of one row each
  uint8_t Cb[C_BYTES];             // column taps (resident)
  float csum[128];
  uint64_t raw_full[2], raw_empty[2];
  uint64_t a_full[NB], slot_free[NB];
  uint64_t b_full[NBB], b_free[NBB];
  uint64_t l_full, l_free, c_full;
  uint64_t acc_full[NSLOT], acc_empty[NSLOT];
  uint32_t tmem_base;
  int abort;
};

// Replicate-padded BF16 copy of the image: P[c][r + 16][x + 16] = I[c][clamp(r)][clamp(x)].
__global__ void k_pad_bf16(const float* __restrict__ img, int C, int H, int W, int Wp, float centre,
                           __nv_bfloat16* __restrict__ P) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  const int c = blockIdx.z;
  if (x >= Wp) return;
  const int sy = min(max(r - 16, 0), H - 1);
  const int sx = min(max(x - 16, 0), W - 1);
  P[((size_t)c * (H + 32) + r) * Wp + x] = __float2bfloat16_rn(img[((size_t)c * H + sy) * W + sx] - centre);
}

// Row tiles: Bt[iy][j][g][n8][k8] = phi_{8j+n8}(iy, 32 - (8g+k8)), g < 4 (taps ix = 1..32),
// then the column taps Ct[j][g][n8][k8] = phi_{8j+n8}(8g+k8, 0), g < 6; zero outside.
__global__ void k_build_bt(const float* __restrict__ basis, int K, int NP, __nv_bfloat16* __restrict__ Bt) {
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
__global__ void __launch_bounds__(THREADS, 1) k_blur_tc(const __nv_bfloat16* __restrict__ P, int H, int W,
                                                        int Wp, const __nv_bfloat16* __restrict__ Bt, int K, int NP,
                                                        const float* __restrict__ csum, const WT* __restrict__ w,
                                                        int w_vec, float* __restrict__ out, int* __restrict__ err) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  Smem& s = *reinterpret_cast<Smem*>(smem_raw);
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
    for (int i = 0; i < 2; ++i) {
      umma::mbar_init(&s.raw_full[i], 1);
      umma::mbar_init(&s.raw_empty[i], NSTAGE_WARPS);
    }
    for (int i = 0; i < NB; ++i) {
      umma::mbar_init(&s.a_full[i], NSTAGE_WARPS);
      umma::mbar_init(&s.slot_free[i], 1);
    }
    for (int i = 0; i < NBB; ++i) {
      umma::mbar_init(&s.b_full[i], 1);
      umma::mbar_init(&s.b_free[i], 1);
    }
    umma::mbar_init(&s.l_full, NSTAGE_WARPS);
    umma::mbar_init(&s.l_free, 1);
    umma::mbar_init(&s.c_full, 1);
    for (int i = 0; i < NSLOT; ++i) {
      umma::mbar_init(&s.acc_full[i], 1);
      umma::mbar_init(&s.acc_empty[i], 4);
    }
    s.abort = 0;
    umma::fence_mbar_init();
  }
  for (int i = tid; i < 128; i += THREADS) s.csum[i] = i < NP ? csum[i] : 0.f;
  if (warp == 0) {
    umma::tmem_alloc(&s.tmem_base, 512);
    umma::tmem_relinquish();
  }
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
    // ---------------------------------------------------------- bulk copies (one lane)
    if (lane == 0) {
      auto issue_raw = [&](int t_local) {
        int y, x0;
        tile_xy(t_local, y, x0);
        const int rb = t_local & 1;
        umma::mbar_arrive_expect_tx(&s.raw_full[rb], (uint32_t)(C * KS * RAWB));
        for (int c = 0; c < C; ++c)
          for (int ri = 0; ri < KS; ++ri)
            umma::bulk_g2s(s.raw[rb][c][ri], P + ((size_t)c * (H + 32) + y + ri) * Wp + x0, RAWB, &s.raw_full[rb]);
      };
      bool ok = true;
      uint32_t v = 0;  // row tiles issued
      int raw_issued = 0;
      umma::mbar_arrive_expect_tx(&s.c_full, ct_bytes);
      umma::bulk_g2s(s.Cb, Ct, ct_bytes, &s.c_full);
      if (my_tiles > 0) {
        issue_raw(0);
        raw_issued = 1;
      }
      for (int t = 0; t < my_tiles && ok; ++t) {
        for (int iy = 0; iy < KS && ok; ++iy, ++v) {
          // the next tile's image rows go out a quarter of the way into this tile, into the raw buffer
          // whose previous tile (t - 1) finished staging before the MMAs of this tile began
          if (iy == KS / 4 && t + 1 < my_tiles) {
            if (t >= 1 && !umma::mbar_wait(&s.raw_empty[(t + 1) & 1], ((t - 1) >> 1) & 1, kWaitNs)) {
              ok = false;
              break;
            }
            issue_raw(t + 1);
            raw_issued = t + 2;
          }
          const int b = v % NBB;
          if (v >= NBB && !umma::mbar_wait(&s.b_free[b], ((v / NBB) - 1) & 1, kWaitNs)) {
            ok = false;
            break;
          }
          umma::mbar_arrive_expect_tx(&s.b_full[b], bt_bytes);
          umma::bulk_g2s(s.B[b], Bt + (size_t)iy * (NP * KM), bt_bytes, &s.b_full[b]);
        }
      }
      if (!ok) {
        s.abort = 1;
        atomicExch(err, 1);
      }
      // every issued copy must land before the CTA exits (bounded)
      umma::mbar_wait(&s.c_full, 0, kWaitNs);
      for (uint32_t u = (v >= NBB ? v - NBB : 0); u < v; ++u) umma::mbar_wait(&s.b_full[u % NBB], (u / NBB) & 1, kWaitNs);
      for (int t = (raw_issued >= 2 ? raw_issued - 2 : 0); t < raw_issued; ++t)
        umma::mbar_wait(&s.raw_full[t & 1], (t >> 1) & 1, kWaitNs);
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------- MMA issue (one lane)
    if (lane == 0) {
      // row operand (slot 0, channel 0): core matrices 128 B apart along M and K (Hankel blocks);
      // row tiles [j][g][8][8]: K-adjacent core matrices 128 B apart, 8-filter groups 512 B apart;
      // column operand [p/8][g][8][8] and column taps [j][g][8][8]: 128 B along K, 768 B along M/N
      const uint64_t a_base = umma::sdesc(umma::smem_u32(s.A[0][0]), 128, 128);
      const uint64_t b_base = umma::sdesc(umma::smem_u32(s.B[0]), 128, KM / 8 * 128);
      const uint64_t l_base = umma::sdesc(umma::smem_u32(s.L[0]), 128, KL / 8 * 128);
      const uint64_t c_desc = umma::sdesc(umma::smem_u32(s.Cb), 128, KL / 8 * 128);
      bool ok = my_tiles == 0 || umma::mbar_wait(&s.c_full, 0, kWaitNs);
      uint32_t it = 0;
      for (int t = 0; t < my_tiles && ok; ++t) {
        for (int iy = 0; iy < KS; ++iy, ++it) {
          const int sb = it % NB;
          const int bb = it % NBB;
          if (!umma::mbar_wait(&s.a_full[sb], (it / NB) & 1, kWaitNs) ||
              !umma::mbar_wait(&s.b_full[bb], (it / NBB) & 1, kWaitNs)) {
            ok = false;
            break;
          }
          if (iy == 0 && !umma::mbar_wait(&s.l_full, t & 1, kWaitNs)) {
            ok = false;
            break;
          }
          umma::fence_after_sync();
          // descriptors = base descriptor + (byte offset >> 4): forming each one from scratch in the
          // issue loop costs more than the MMA itself
          const uint64_t a_it = a_base + (uint64_t)(((uint32_t)sb * (CMAX * ROWB)) >> 4);
          const uint64_t b_it = b_base + (uint64_t)(((uint32_t)bb * B_SLOT) >> 4);
#pragma unroll
          for (int c = 0; c < C; ++c) {
            const uint32_t g = (uint32_t)(t * C + c);
            const uint32_t d = tmem + (g % NSLOT) * NP;
            if (iy == 0) {
              // a fresh accumulator: wait until the epilogue has emptied this slot, then the column taps
              if (g >= NSLOT && !umma::mbar_wait(&s.acc_empty[g % NSLOT], ((g / NSLOT) - 1) & 1, kWaitNs)) {
                ok = false;
                break;
              }
              umma::fence_after_sync();
              const uint64_t l_c = l_base + (uint64_t)((c * L_BYTES) >> 4);
              umma::mma_bf16(d, l_c, c_desc, idesc, 0);
              umma::mma_bf16(d, l_c + 16, c_desc + 16, idesc, 1);
              umma::mma_bf16(d, l_c + 32, c_desc + 32, idesc, 1);
            }
            const uint64_t a_c = a_it + (uint64_t)((c * ROWB) >> 4);
            umma::mma_bf16(d, a_c, b_it, idesc, 1);
            umma::mma_bf16(d, a_c + 16, b_it + 16, idesc, 1);
          }
          if (!ok) break;
          umma::mma_commit(&s.slot_free[sb]);
          umma::mma_commit(&s.b_free[bb]);
          if (iy == 0) umma::mma_commit(&s.l_free);
          if (iy == KS - 1)
#pragma unroll
            for (int c = 0; c < C; ++c) umma::mma_commit(&s.acc_full[(t * C + c) % NSLOT]);
        }
      }
      if (!ok) {
        s.abort = 1;
        atomicExch(err, 1);
      }
      if (it >= 1) umma::mbar_wait(&s.slot_free[(it - 1) % NB], ((it - 1) / NB) & 1, kWaitNs);
    }
  } else if (warp < EPI_WARP0) {
    // ---------------------------------------------------------- staging: Hankel blocks and column operand
    const int st_tid = tid - STAGE_WARP0 * 32;
    uint32_t it = 0;
    for (int t = 0; t < my_tiles; ++t) {
      const int rb = t & 1;
      if (!umma::mbar_wait(&s.raw_full[rb], (t >> 1) & 1, kWaitNs)) s.abort = 1;
      // the column operand of the previous tile has been consumed by its first MMAs
      if (t >= 1 && !umma::mbar_wait(&s.l_free, (t - 1) & 1, kWaitNs)) s.abort = 1;
      if (s.abort) break;
      // L[p][iy] = raw row 32 - iy, column p + 32 (iy < 33; zero up to 48), K-major [p/8][iy/8][8][8]
      for (int item = st_tid; item < C * (KL / 8) * TM; item += NSTAGE_WARPS * 32) {
        const int p = item & (TM - 1);
        const int cg = item >> 7;
        const int c = cg / (KL / 8), g = cg - c * (KL / 8);
        uint32_t wv[4];
#pragma unroll
        for (int e2 = 0; e2 < 4; ++e2) {
          uint32_t lo = 0, hi = 0;
          const int iy0 = 8 * g + 2 * e2;
          if (iy0 < KS) lo = *reinterpret_cast<const uint16_t*>(s.raw[rb][c][KS - 1 - iy0] + 2 * (p + 32));
          if (iy0 + 1 < KS) hi = *reinterpret_cast<const uint16_t*>(s.raw[rb][c][KS - 2 - iy0] + 2 * (p + 32));
          wv[e2] = lo | (hi << 16);
        }
        *reinterpret_cast<uint4*>(s.L[c] + ((p >> 3) * (KL / 8) + g) * 128 + (p & 7) * 16) =
            make_uint4(wv[0], wv[1], wv[2], wv[3]);
      }
      umma::fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) umma::mbar_arrive(&s.l_full);
      for (int iy = 0; iy < KS; ++iy, ++it) {
        const int sb = it % NB;
        if (it >= NB && !umma::mbar_wait(&s.slot_free[sb], ((it / NB) - 1) & 1, kWaitNs)) s.abort = 1;
        if (s.abort) break;
        const int ri = KS - 1 - iy;
        // item = (channel, block, row s of the block), s fastest: 8 lanes write one 128-byte block
        for (int item = st_tid; item < C * NBLK * 8; item += NSTAGE_WARPS * 32) {
          const int sr = item & 7;
          const int cb = item >> 3;
          const int c = cb / NBLK, b = cb - c * NBLK;
          const uint32_t* src = reinterpret_cast<const uint32_t*>(s.raw[rb][c][ri]) + 4 * b + (sr >> 1);
          const uint32_t w0 = src[0], w1 = src[1], w2 = src[2], w3 = src[3], w4 = src[4];
          const uint32_t sh = (sr & 1) * 16;
          const uint4 o = make_uint4(__funnelshift_r(w0, w1, sh), __funnelshift_r(w1, w2, sh),
                                     __funnelshift_r(w2, w3, sh), __funnelshift_r(w3, w4, sh));
          *reinterpret_cast<uint4*>(s.A[sb][c] + b * 128 + sr * 16) = o;
        }
        umma::fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) umma::mbar_arrive(&s.a_full[sb]);
      }
      if (s.abort) break;
      if (lane == 0) umma::mbar_arrive(&s.raw_empty[rb]);
    }
  } else {
    // ---------------------------------------------------------- epilogue: TMEM -> weighted sums, one channel per group
    const int c = (warp - EPI_WARP0) >> 2;
    const int q4 = warp & 3;  // warp w reads TMEM lanes 32 (w % 4) ..
    if (c < C) {
      for (int t = 0; t < my_tiles; ++t) {
        int y, x0;
        tile_xy(t, y, x0);
        const int x = x0 + q4 * 32 + lane;
        const bool live = x < W;
        const size_t pix = (size_t)y * W + (live ? x : 0);
        const WT* wg = w + pix * K;
        const uint32_t g = (uint32_t)(t * C + c);
        const uint32_t slot = g % NSLOT;
        if (!umma::mbar_wait(&s.acc_full[slot], (g / NSLOT) & 1, kWaitNs)) s.abort = 1;
        if (s.abort) break;
        umma::fence_after_sync();
        float acc = 0.f;
        for (int q = 0; q < NP / 16; ++q) {
          float wk[16];
          if (w_vec) {  // 16-byte aligned FP32 rows: four vector loads
#pragma unroll
            for (int i4 = 0; i4 < 4; ++i4) {
              const int k = q * 16 + 4 * i4;
              const float4 v4 = k < K ? __ldg(reinterpret_cast<const float4*>(wg) + (k >> 2)) : make_float4(0.f, 0.f, 0.f, 0.f);
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
          float d[16];
          umma::tmem_ld16(tmem + ((uint32_t)(q4 * 32) << 16) + slot * NP + q * 16, d);
#pragma unroll
          for (int i = 0; i < 16; ++i) acc = fmaf(wk[i], d[i] + s.csum[q * 16 + i], acc);
        }
        umma::fence_before_sync();
        __syncwarp();
        if (lane == 0) umma::mbar_arrive(&s.acc_empty[slot]);
        if (live) out[((size_t)c * H + y) * W + x] = acc;
      }
    }
  }
  umma::fence_before_sync();
  __syncthreads();
  if (warp == 0) umma::tmem_dealloc(tmem, 512);
}

}  // namespace

int dfp2s_launch_blur_tc(dfp2s_p2s_dev* p, const float* img, int C, int H, int W, const void* w, int w_dtype,
                         float* out, cudaStream_t st) {
  const int K = p->K;
  const int NP = (K + 15) / 16 * 16;
  const float centre = 0.5f;
  if (NP > 128) return DFP2S_EUNSUPPORTED;
  // basis tiles and centring sums c * s_k (once per handle)
  if (!p->bt) {
    const int n = KS * NP * KM + NP * KL;  // row tiles, then the column taps
    if (cudaMalloc((void**)&p->bt, (size_t)n * sizeof(__nv_bfloat16)) != cudaSuccess) return DFP2S_ENOMEM;
    if (cudaMalloc((void**)&p->bsum, (size_t)NP * sizeof(float)) != cudaSuccess) return DFP2S_ENOMEM;
    k_build_bt<<<(n + 255) / 256, 256, 0, st>>>(p->basis, K, NP, p->bt);
    k_basis_sums<<<NP, 256, 0, st>>>(p->basis, K, NP, p->bsum);
    k_scale<<<1, 128, 0, st>>>(p->bsum, NP, centre);
  }
  if (!p->err) {
    if (cudaMalloc((void**)&p->err, sizeof(int)) != cudaSuccess) return DFP2S_ENOMEM;
    cudaMemsetAsync(p->err, 0, sizeof(int), st);
  }
  const int nseg = (W + TM - 1) / TM;
  const int Wp = nseg * TM + 64;
  const size_t need = (size_t)C * (H + 32) * Wp;
  if (need > p->pad_cap) {
    if (p->pad) cudaFree(p->pad);
    p->pad = nullptr;
    p->pad_cap = 0;
    if (cudaMalloc((void**)&p->pad, need * sizeof(__nv_bfloat16)) != cudaSuccess) return DFP2S_ENOMEM;
    p->pad_cap = need;
  }
  k_pad_bf16<<<dim3((Wp + 255) / 256, H + 32, C), 256, 0, st>>>(img, C, H, W, Wp, centre, p->pad);
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
  // FP32 weights in 16-byte aligned rows are read with vector loads
  const int w_vec = (w_dtype == DFP2S_W_F32) && (K % 4) == 0 && ((uintptr_t)w & 15) == 0;
  for (int c0 = 0; c0 < C; c0 += CMAX) {
    const int nc = C - c0 < CMAX ? C - c0 : CMAX;
    const __nv_bfloat16* pc = p->pad + (size_t)c0 * (H + 32) * Wp;
    float* oc = out + (size_t)c0 * H * W;
#define DFP2S_BLUR_LAUNCH(WT, NC, WPTR, WSM) \
  k_blur_tc<WT, NC><<<grid, THREADS, sm, st>>>(pc, H, W, Wp, p->bt, K, NP, p->bsum, WPTR, WSM, oc, p->err)
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
  return cudaGetLastError() == cudaSuccess ? DFP2S_OK : DFP2S_ECUDA;
}
