// Basis blur on the tcgen05 tensor cores (BF16 operands, FP32 accumulation in
// TMEM), Eq. (varying blur):
//
//   out_c(y, x) = sum_k w_k(y, x) conv_k,c(y, x),
//   conv_k,c(y, x) = sum_{iy, ix} phi_k(iy, ix) I_c(y + 16 - iy, x + 16 - ix)   (clamp to edge)
//
// For one output row y and 128 consecutive pixels x0..x0+127, the 33 taps of
// basis row iy form a dense contraction over kappa = 32 - ix:
//
//   D[p][k] += sum_kappa A_iy[p][kappa] B_iy[k][kappa],
//   A_iy[p][kappa] = I_c(r, x0 - 16 + p + kappa), r = y + 16 - iy   (Hankel in p + kappa)
//   B_iy[k][kappa] = phi_k(iy, 32 - kappa)                          (kappa padded to 48, k to NP)
//
// with M = 128 pixels, N = NP filters and K = 48 (three K = 16 MMAs) per basis
// row, 99 MMAs per channel per tile.  A needs no im2col: a K-major core matrix
// (8 rows x 16 bytes) of A at (row group i, K group g) is the 8 x 8 block
// E_{i+g}[s][t] = I_c(r, x0 - 16 + 8(i+g) + s + t), so one staged image row
// holds the 21 blocks E_0..E_20 back to back and the operand descriptor uses
// the same 128-byte stride along M and along K.  B tiles for each iy are laid
// out once per basis in global memory and streamed with 1-D bulk copies.
// The epilogue reads D from TMEM (one pixel per thread) and contracts it with
// the pixel's weights: out = sum_k w_k (D[p][k] + c s_k).
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
constexpr int TM = 128;                // pixels per tile (MMA M)
constexpr int KP = 48;                 // taps of one basis row padded to three K = 16 steps
constexpr int NBLK = TM / 8 + KP / 8 - 1;  // 21 staged 8x8 blocks per image row
constexpr int ROWB = NBLK * 128;       // 2688 bytes per staged row
constexpr int CMAX = 3;                // channels per pass
constexpr int NSLOT = 4;               // TMEM accumulator slots of NP <= 128 columns (512 in all)
// warp 0: bulk copies; warp 1: MMA issue; warps 2-7: staging; warps 8-11: epilogue (TMEM lane quarters 0-3)
constexpr int STAGE_WARP0 = 2;
constexpr int NSTAGE_WARPS = 6;
constexpr int EPI_WARP0 = STAGE_WARP0 + NSTAGE_WARPS;
constexpr int THREADS = (EPI_WARP0 + 4) * 32;
constexpr int NB = 4;                  // staged-row ring (one slot per basis row iy)
constexpr int NBB = 4;                 // basis-tile ring
constexpr int RAWW = TM + KP;          // 176 staged image columns per row
constexpr uint64_t kWaitNs = 2000000000ull;  // 2 s bound on any wait
constexpr int B_SLOT = KP / 8 * 16 * 128;  // bytes of one basis-tile slot

struct Smem {
  uint8_t raw[2][CMAX][KS][RAWW * 2];  // image rows of a tile (bulk copies, prefetched one tile ahead)
  uint8_t A[NB][CMAX][ROWB];           // Hankel-blocked rows
  uint8_t B[NBB][B_SLOT];              // basis tiles (up to NP = 128)
  float csum[128];
  uint64_t raw_full[2], raw_empty[2];
  uint64_t a_full[NB], slot_free[NB];
  uint64_t b_full[NBB], b_free[NBB];
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

// B tiles: Bt[iy][j][g][n8][k8] = phi_{8j+n8}(iy, 32 - (8g+k8)), zero outside.
__global__ void k_build_bt(const float* __restrict__ basis, int K, int NP, __nv_bfloat16* __restrict__ Bt) {
  const int per_iy = NP * KP;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= KS * per_iy) return;
  const int iy = i / per_iy;
  int rem = i - iy * per_iy;
  const int j = rem / (6 * 64);
  rem -= j * 6 * 64;
  const int g = rem / 64;
  rem -= g * 64;
  const int n8 = rem / 8, k8 = rem - n8 * 8;
  const int k = 8 * j + n8, kap = 8 * g + k8;
  float v = 0.f;
  if (k < K && kap < KS) v = basis[((size_t)k * KS + iy) * KS + (KS - 1 - kap)];
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
                                                        int w_smem, float* __restrict__ out, int* __restrict__ err) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  Smem& s = *reinterpret_cast<Smem*>(smem_raw);
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const uint32_t bt_bytes = (uint32_t)(NP / 8) * 6 * 128;
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
        umma::mbar_arrive_expect_tx(&s.raw_full[rb], (uint32_t)(C * KS * RAWW * 2));
        for (int c = 0; c < C; ++c)
          for (int ri = 0; ri < KS; ++ri)
            umma::bulk_g2s(s.raw[rb][c][ri], P + ((size_t)c * (H + 32) + y + ri) * Wp + x0, RAWW * 2,
                           &s.raw_full[rb]);
      };
      bool ok = true;
      uint32_t v = 0;  // basis tiles issued
      int raw_issued = 0;
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
          umma::bulk_g2s(s.B[b], Bt + (size_t)iy * (NP * KP), bt_bytes, &s.b_full[b]);
        }
      }
      if (!ok) {
        s.abort = 1;
        atomicExch(err, 1);
      }
      // every issued copy must land before the CTA exits (bounded)
      for (uint32_t u = (v >= NBB ? v - NBB : 0); u < v; ++u) umma::mbar_wait(&s.b_full[u % NBB], (u / NBB) & 1, kWaitNs);
      for (int t = (raw_issued >= 2 ? raw_issued - 2 : 0); t < raw_issued; ++t)
        umma::mbar_wait(&s.raw_full[t & 1], (t >> 1) & 1, kWaitNs);
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------- MMA issue (one lane)
    if (lane == 0) {
      // A tile (slot 0, channel 0): core matrices 128 B apart along M and K (Hankel blocks);
      // B tile [j][g][8][8]: K-adjacent core matrices 128 B apart, 8-filter groups 768 B apart
      const uint64_t a_base = umma::sdesc(umma::smem_u32(s.A[0][0]), 128, 128);
      const uint64_t b_base = umma::sdesc(umma::smem_u32(s.B[0]), 128, 768);
      bool ok = true;
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
          if (iy == 0) {
#pragma unroll
            for (int c = 0; c < C; ++c) {
              const uint32_t g = (uint32_t)(t * C + c);
              if (g >= NSLOT && !umma::mbar_wait(&s.acc_empty[g % NSLOT], ((g / NSLOT) - 1) & 1, kWaitNs)) ok = false;
            }
            if (!ok) break;
          }
          umma::fence_after_sync();
          // descriptors = base descriptor + (byte offset >> 4): forming each one from scratch in the
          // issue loop costs more than the MMA itself
          const uint64_t a_it = a_base + (uint64_t)(((uint32_t)sb * (CMAX * ROWB)) >> 4);
          const uint64_t b_it = b_base + (uint64_t)(((uint32_t)bb * B_SLOT) >> 4);
          const uint32_t acc = iy != 0;
#pragma unroll
          for (int c = 0; c < C; ++c) {
            const uint32_t d = tmem + ((uint32_t)(t * C + c) % NSLOT) * NP;
            const uint64_t a_c = a_it + (uint64_t)((c * ROWB) >> 4);
            umma::mma_bf16(d, a_c, b_it, idesc, acc);
            umma::mma_bf16(d, a_c + 16, b_it + 16, idesc, 1);
            umma::mma_bf16(d, a_c + 32, b_it + 32, idesc, 1);
          }
          umma::mma_commit(&s.slot_free[sb]);
          umma::mma_commit(&s.b_free[bb]);
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
    // ---------------------------------------------------------- staging: Hankel blocks from raw rows
    const int st_tid = tid - STAGE_WARP0 * 32;
    uint32_t it = 0;
    for (int t = 0; t < my_tiles; ++t) {
      const int rb = t & 1;
      if (!umma::mbar_wait(&s.raw_full[rb], (t >> 1) & 1, kWaitNs)) s.abort = 1;
      if (s.abort) break;
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
    // ---------------------------------------------------------- epilogue: TMEM -> weighted sums
    const int q4 = warp & 3;  // warp w reads TMEM lanes 32 (w % 4) ..
    for (int t = 0; t < my_tiles; ++t) {
      int y, x0;
      tile_xy(t, y, x0);
      const int x = x0 + q4 * 32 + lane;
      const bool live = x < W;
      const size_t pix = (size_t)y * W + (live ? x : 0);
      const WT* wg = w + pix * K;
      int slot[CMAX];
      for (int c = 0; c < C; ++c) {
        const uint32_t g = (uint32_t)(t * C + c);
        slot[c] = g % NSLOT;
        if (!umma::mbar_wait(&s.acc_full[slot[c]], (g / NSLOT) & 1, kWaitNs)) s.abort = 1;
      }
      if (s.abort) break;
      umma::fence_after_sync();
      float acc[CMAX] = {0.f, 0.f, 0.f};
      for (int q = 0; q < NP / 16; ++q) {
        float wk[16];
        if (w_smem) {  // 16-byte aligned FP32 rows: four vector loads
#pragma unroll
          for (int i4 = 0; i4 < 4; ++i4) {
            const int k = q * 16 + 4 * i4;
            const float4 v = k < K ? __ldg(reinterpret_cast<const float4*>(wg) + (k >> 2)) : make_float4(0.f, 0.f, 0.f, 0.f);
            wk[4 * i4 + 0] = v.x;
            wk[4 * i4 + 1] = v.y;
            wk[4 * i4 + 2] = v.z;
            wk[4 * i4 + 3] = v.w;
          }
        } else {
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int k = q * 16 + i;
            wk[i] = k < K ? wload<WT>(wg + k) : 0.f;
          }
        }
#pragma unroll
        for (int c = 0; c < CMAX; ++c) {
          if (c < C) {
            float d[16];
            umma::tmem_ld16(tmem + ((uint32_t)(q4 * 32) << 16) + slot[c] * NP + q * 16, d);
#pragma unroll
            for (int i = 0; i < 16; ++i) acc[c] = fmaf(wk[i], d[i] + s.csum[q * 16 + i], acc[c]);
          }
        }
      }
      umma::fence_before_sync();
      __syncwarp();
      if (lane == 0)
        for (int c = 0; c < C; ++c) umma::mbar_arrive(&s.acc_empty[slot[c]]);
      if (live) {
#pragma unroll
        for (int c = 0; c < CMAX; ++c)
          if (c < C) out[((size_t)c * H + y) * W + x] = acc[c];
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
    if (cudaMalloc((void**)&p->bt, (size_t)KS * NP * KP * sizeof(__nv_bfloat16)) != cudaSuccess) return DFP2S_ENOMEM;
    if (cudaMalloc((void**)&p->bsum, (size_t)NP * sizeof(float)) != cudaSuccess) return DFP2S_ENOMEM;
    const int n = KS * NP * KP;
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
  static_assert(sizeof(Smem) + 1024 > 116 * 1024 && sizeof(Smem) + 1024 < 227 * 1024, "smem layout");
  cudaFuncSetAttribute(k_blur_tc<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  cudaFuncSetAttribute(k_blur_tc<float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  cudaFuncSetAttribute(k_blur_tc<float, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  cudaFuncSetAttribute(k_blur_tc<__nv_bfloat16, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  cudaFuncSetAttribute(k_blur_tc<__nv_bfloat16, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  cudaFuncSetAttribute(k_blur_tc<__nv_bfloat16, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  // FP32 weights in 16-byte aligned rows are read with vector loads
  const int w_smem = (w_dtype == DFP2S_W_F32) && (K % 4) == 0 && ((uintptr_t)w & 15) == 0;
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
      if (nc == 1) DFP2S_BLUR_LAUNCH(float, 1, wf, w_smem);
      else if (nc == 2) DFP2S_BLUR_LAUNCH(float, 2, wf, w_smem);
      else DFP2S_BLUR_LAUNCH(float, 3, wf, w_smem);
    }
#undef DFP2S_BLUR_LAUNCH
  }
  return cudaGetLastError() == cudaSuccess ? DFP2S_OK : DFP2S_ECUDA;
}
