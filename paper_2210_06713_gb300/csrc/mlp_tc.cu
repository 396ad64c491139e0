// Surrogate P2S network (Sec. II-C) on the tcgen05 tensor cores: one fused
// kernel per frame, BF16 operands, FP32 accumulation in tensor memory.
//
// A tile is 128 consecutive pixels (MMA M = 128):
//   layer 1: X [128 x 48] (the J fields, zero-padded) x W1'^T -> TMEM columns [0, 256)
//            (W1' = W1 diag(in_scale), resident in shared memory)
//   GELU(z + b1) -> H [128 x 256] BF16 in shared memory (K-major core matrices)
//   layer 2: H x W2^T -> TMEM [256, 512), W2 streamed in four 64-wide K chunks
//   GELU(z + b2) -> H
//   layer 3: H x W3^T -> TMEM [0, NP3), W3 streamed in four K chunks
//   w = y * out_scale + (b3 * out_scale + out_shift) -> global (FP32 or BF16)
// Weight chunks arrive by 1-D bulk copies into a three-deep ring; the MMAs of a
// chunk release its buffer through tcgen05.commit.  All waits are bounded.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "kernels.h"
#include "umma.cuh"

namespace {

constexpr int TM = 128;
constexpr int HID = 256;
constexpr int KX = 48;           // J padded to three K = 16 steps
constexpr int THREADS = 256;     // 8 warps: warps w and w + 4 share TMEM lanes 32 (w % 4) ..
constexpr int NRING = 3;
constexpr int CHUNK_BYTES = HID * 64 * 2;  // one 64-wide K chunk of W2 (the largest)
constexpr uint64_t kWaitNs = 2000000000ull;

struct Smem {
  uint8_t ring[NRING][CHUNK_BYTES];  // 96 KB
  uint8_t H[TM * HID * 2];           // 64 KB
  uint8_t W1[HID * KX * 2];          // 24 KB
  uint8_t X[TM * KX * 2];            // 12 KB
  float b1[HID], b2[HID];
  float c3[128], s3[128];            // output bias and scale
  uint64_t full[NRING], empty[NRING];
  uint64_t w1_full, layer_done;
  uint32_t tmem_base;
  int abort;
};

DFP2S_DEV float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }

// byte offset of element (row, k) in a K-major no-swizzle tile with `kgroups` 8-element K groups per row group
DFP2S_DEV uint32_t kmajor_off(int row, int k, int kgroups) {
  return (uint32_t)(((row >> 3) * kgroups + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

template <typename WT>
DFP2S_DEV void wstore(WT* p, float v);
template <>
DFP2S_DEV void wstore<float>(float* p, float v) { *p = v; }
template <>
DFP2S_DEV void wstore<__nv_bfloat16>(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }

// TMEM columns [col0, col0 + 128) of this thread's pixel -> GELU(z + b) -> H row (K = col - col0 + kbase)
DFP2S_DEV void epilogue_gelu(uint32_t tmem, int warp, int lane, int col0, int kbase, const float* bias, uint8_t* H) {
  const int p = (warp & 3) * 32 + lane;
  for (int q = 0; q < 8; ++q) {
    float d[16];
    umma::tmem_ld16(tmem + ((uint32_t)((warp & 3) * 32) << 16) + col0 + q * 16, d);
    uint32_t packed[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int k = kbase + q * 16 + 2 * i;
      const float g0 = gelu(d[2 * i] + bias[k]);
      const float g1 = gelu(d[2 * i + 1] + bias[k + 1]);
      __nv_bfloat162 h2 = __floats2bfloat162_rn(g0, g1);
      packed[i] = *reinterpret_cast<uint32_t*>(&h2);
    }
    const int k0 = kbase + q * 16;
    *reinterpret_cast<uint4*>(H + kmajor_off(p, k0, HID / 8)) = make_uint4(packed[0], packed[1], packed[2], packed[3]);
    *reinterpret_cast<uint4*>(H + kmajor_off(p, k0 + 8, HID / 8)) =
        make_uint4(packed[4], packed[5], packed[6], packed[7]);
  }
}

template <typename WT>
__global__ void __launch_bounds__(THREADS, 1)
    k_mlp_tc(const float* __restrict__ fields, int J, int npix, int K, int NP3, const __nv_bfloat16* __restrict__ w1t,
             const __nv_bfloat16* __restrict__ w2c, const __nv_bfloat16* __restrict__ w3c, const float* __restrict__ b1,
             const float* __restrict__ b2, const float* __restrict__ c3, const float* __restrict__ s3,
             WT* __restrict__ wout, int* __restrict__ err) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  Smem& s = *reinterpret_cast<Smem*>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t w2_bytes = (uint32_t)CHUNK_BYTES;
  const uint32_t w3_bytes = (uint32_t)(NP3 * 64 * 2);
  const int ntiles = (npix + TM - 1) / TM;

  if (tid == 0) {
    for (int i = 0; i < NRING; ++i) {
      umma::mbar_init(&s.full[i], 1);
      umma::mbar_init(&s.empty[i], 1);
    }
    umma::mbar_init(&s.w1_full, 1);
    umma::mbar_init(&s.layer_done, 1);
    s.abort = 0;
    umma::fence_mbar_init();
  }
  for (int i = tid; i < HID; i += THREADS) {
    s.b1[i] = b1[i];
    s.b2[i] = b2[i];
  }
  for (int i = tid; i < 128; i += THREADS) {
    s.c3[i] = i < K ? c3[i] : 0.f;
    s.s3[i] = i < K ? s3[i] : 0.f;
  }
  // zero X once (the padded K columns stay zero)
  for (int i = tid; i < TM * KX * 2 / 16; i += THREADS) reinterpret_cast<uint4*>(s.X)[i] = make_uint4(0, 0, 0, 0);
  if (warp == 0) {
    umma::tmem_alloc(&s.tmem_base, 512);
    umma::tmem_relinquish();
  }
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = s.tmem_base;
  if (tid == 0) {
    umma::mbar_arrive_expect_tx(&s.w1_full, HID * KX * 2);
    umma::bulk_g2s(s.W1, w1t, HID * KX * 2, &s.w1_full);
  }
  // operand descriptors (K-major, no swizzle): X and W1 with 6 K groups per 8-row group,
  // H with 32, weight chunks with 8; per-MMA descriptors add (byte offset >> 4)
  const uint64_t x_desc = umma::sdesc(umma::smem_u32(s.X), 128, 768);
  const uint64_t w1_desc = umma::sdesc(umma::smem_u32(s.W1), 128, 768);
  const uint64_t h_desc = umma::sdesc(umma::smem_u32(s.H), 128, 4096);
  const uint64_t ring_desc = umma::sdesc(umma::smem_u32(s.ring[0]), 128, 1024);
  const uint32_t idesc1 = umma::idesc_bf16(TM, HID);
  const uint32_t idesc3 = umma::idesc_bf16(TM, NP3);
  uint32_t u_issue = 0;  // weight chunks issued (bulk copies)
  uint32_t u_use = 0;    // weight chunks consumed by MMAs
  uint32_t ndone = 0;    // completions of layer_done
  bool ok = true;

  // issue the copy of weight chunk number u (8 per tile: 4 of W2 then 4 of W3)
  auto issue = [&](uint32_t u) {
    const int b = u % NRING;
    if (u >= NRING) {
      if (!umma::mbar_wait(&s.empty[b], ((u / NRING) - 1) & 1, kWaitNs)) s.abort = 1;
    }
    const int c = u % 8;
    if (c < 4) {
      umma::mbar_arrive_expect_tx(&s.full[b], w2_bytes);
      umma::bulk_g2s(s.ring[b], w2c + (size_t)c * (HID * 64), w2_bytes, &s.full[b]);
    } else {
      umma::mbar_arrive_expect_tx(&s.full[b], w3_bytes);
      umma::bulk_g2s(s.ring[b], w3c + (size_t)(c - 4) * (NP3 * 64), w3_bytes, &s.full[b]);
    }
  };

  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int p0 = tile * TM;
    // prefetch the first chunks of this tile
    if (tid == 0) {
      while (u_issue < u_use + NRING && !s.abort) issue(u_issue++);
    }
    // X tile: fields[j][p0 + p] -> bf16 at (p, j)
    for (int idx = tid; idx < J * TM; idx += THREADS) {
      const int j = idx / TM, p = idx - j * TM;
      const float v = (p0 + p < npix) ? __ldg(fields + (size_t)j * npix + p0 + p) : 0.f;
      *reinterpret_cast<__nv_bfloat16*>(s.X + kmajor_off(p, j, KX / 8)) = __float2bfloat16_rn(v);
    }
    umma::fence_proxy_async_smem();
    __syncthreads();
    if (s.abort) {
      ok = false;
      break;
    }
    // layer 1
    if (tid == 0) {
      if (!umma::mbar_wait(&s.w1_full, 0, kWaitNs)) {
        s.abort = 1;
      } else {
        umma::fence_after_sync();
#pragma unroll
        for (int ks = 0; ks < KX / 16; ++ks) umma::mma_bf16(tmem, x_desc + 16 * ks, w1_desc + 16 * ks, idesc1, ks != 0);
        umma::mma_commit(&s.layer_done);
      }
    }
    if (!umma::mbar_wait(&s.layer_done, ndone & 1, kWaitNs)) s.abort = 1;
    ++ndone;
    umma::fence_after_sync();
    epilogue_gelu(tmem, warp, lane, (warp >> 2) * 128, (warp >> 2) * 128, s.b1, s.H);
    umma::fence_proxy_async_smem();
    umma::fence_before_sync();
    __syncthreads();
    if (s.abort) {
      ok = false;
      break;
    }
    // layers 2 and 3: 8 weight chunks
    for (int layer = 2; layer <= 3; ++layer) {
      if (tid == 0) {
        umma::fence_after_sync();
        for (int c = 0; c < 4; ++c) {
          const uint32_t u = u_use++;
          const int b = u % NRING;
          if (!umma::mbar_wait(&s.full[b], (u / NRING) & 1, kWaitNs)) {
            s.abort = 1;
            break;
          }
          // descriptors = base + (byte offset >> 4)
          const uint64_t a_c = h_desc + (uint64_t)(c * 8 * 8);
          const uint64_t b_c = ring_desc + (uint64_t)(b * (CHUNK_BYTES >> 4));
          const uint32_t d = layer == 2 ? tmem + 256 : tmem;
          const uint32_t id = layer == 2 ? idesc1 : idesc3;
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) umma::mma_bf16(d, a_c + 16 * ks, b_c + 16 * ks, id, (c | ks) != 0);
          umma::mma_commit(&s.empty[b]);
          // keep the ring full (the next tile's chunks too)
          while (u_issue < u_use + NRING && !s.abort) issue(u_issue++);
        }
        umma::mma_commit(&s.layer_done);
      }
      if (!umma::mbar_wait(&s.layer_done, ndone & 1, kWaitNs)) s.abort = 1;
      ++ndone;
      umma::fence_after_sync();
      if (layer == 2) {
        epilogue_gelu(tmem, warp, lane, 256 + (warp >> 2) * 128, (warp >> 2) * 128, s.b2, s.H);
        umma::fence_proxy_async_smem();
      } else {
        // stage this tile's outputs in H (free now), then one contiguous coalesced copy
        float* stage = reinterpret_cast<float*>(s.H);
        if (warp < 4) {
          const int p = warp * 32 + lane;
          for (int q = 0; q < NP3 / 16; ++q) {
            float d[16];
            umma::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + q * 16, d);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const int k = q * 16 + i;
              if (k < K) stage[p * K + k] = fmaf(d[i], s.s3[k], s.c3[k]);
            }
          }
        }
        __syncthreads();
        const int nlive = min(TM, npix - p0);
        WT* dst = wout + (size_t)p0 * K;
        for (int i = tid; i < nlive * K; i += THREADS) wstore<WT>(dst + i, stage[i]);
      }
      umma::fence_before_sync();
      __syncthreads();
      if (s.abort) {
        ok = false;
        break;
      }
    }
    if (!ok) break;
  }
  if (!ok && tid == 0) atomicExch(err, 2);
  // drain outstanding copies (bounded) before the CTA exits
  if (tid == 0) {
    for (uint32_t u = u_use; u < u_issue; ++u) umma::mbar_wait(&s.full[u % NRING], (u / NRING) & 1, kWaitNs);
    if (u_use > 0) {
      const uint32_t u = u_use - 1;
      umma::mbar_wait(&s.empty[u % NRING], (u / NRING) & 1, kWaitNs);
    }
  }
  umma::fence_before_sync();
  __syncthreads();
  if (warp == 0) umma::tmem_dealloc(tmem, 512);
}

// ---- weight layouts (built once per installed network)
// W1' [n][j] * in_scale[j] -> K-major tile [n/8][j/8][8][8], j padded to 48
__global__ void k_pack_w1(const float* __restrict__ W1t, const float* __restrict__ in_scale, int J,
                          __nv_bfloat16* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // over 256 x 48
  if (i >= HID * KX) return;
  const int n = i / KX, j = i - n * KX;
  // W1t is stored transposed (J x 256): W1[n][j] = W1t[j * 256 + n]
  const float v = j < J ? W1t[(size_t)j * HID + n] * in_scale[j] : 0.f;
  out[kmajor_off(n, j, KX / 8) / 2] = __float2bfloat16_rn(v);
}

// W[n][k] (given transposed: Wt[k * ncols + n]) -> chunks [kc][n/8][k%64/8][8][8] for n < nrows_pad
__global__ void k_pack_chunks(const float* __restrict__ Wt, int nrows, int nrows_pad, int ncols_t,
                              __nv_bfloat16* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // over 4 chunks x nrows_pad x 64
  if (i >= 4 * nrows_pad * 64) return;
  const int kc = i / (nrows_pad * 64);
  const int rem = i - kc * nrows_pad * 64;
  const int n = rem / 64, kk = rem - n * 64;
  const int k = kc * 64 + kk;
  const float v = n < nrows ? Wt[(size_t)k * ncols_t + n] : 0.f;
  out[(size_t)kc * nrows_pad * 64 + kmajor_off(n, kk, 8) / 2] = __float2bfloat16_rn(v);
}

__global__ void k_out_affine(const float* __restrict__ b3, const float* __restrict__ sc,
                             const float* __restrict__ sh, int K, float* __restrict__ c3) {
  const int k = threadIdx.x;
  if (k < K) c3[k] = b3[k] * sc[k] + sh[k];
}

}  // namespace

int dfp2s_mlp_tc_pack(dfp2s_p2s_dev* p, cudaStream_t st) {
  const int K = p->K;
  const int NP3 = (K + 15) / 16 * 16;
  if (NP3 > 128) return DFP2S_EUNSUPPORTED;
  if (!p->tc_w1 && (cudaMalloc((void**)&p->tc_w1, HID * KX * sizeof(__nv_bfloat16)) != cudaSuccess ||
                    cudaMalloc((void**)&p->tc_w2, 4 * HID * 64 * sizeof(__nv_bfloat16)) != cudaSuccess ||
                    cudaMalloc((void**)&p->tc_w3, 4 * 128 * 64 * sizeof(__nv_bfloat16)) != cudaSuccess ||
                    cudaMalloc((void**)&p->tc_c3, 128 * sizeof(float)) != cudaSuccess))
    return DFP2S_ENOMEM;
  // the SIMT layout keeps W1, W2, W3 transposed: W1t (J x 256), W2t (256 x 256), W3t (256 x K)
  k_pack_w1<<<(HID * KX + 255) / 256, 256, 0, st>>>(p->W1, p->in_scale, p->J, p->tc_w1);
  k_pack_chunks<<<(4 * HID * 64 + 255) / 256, 256, 0, st>>>(p->W2, HID, HID, HID, p->tc_w2);
  k_pack_chunks<<<(4 * NP3 * 64 + 255) / 256, 256, 0, st>>>(p->W3, K, NP3, K, p->tc_w3);
  k_out_affine<<<1, 128, 0, st>>>(p->b3, p->out_scale, p->out_shift, K, p->tc_c3);
  return cudaGetLastError() == cudaSuccess ? DFP2S_OK : DFP2S_ECUDA;
}

int dfp2s_launch_mlp_tc(const dfp2s_p2s_dev* p, const float* fields, int npix, void* w, int w_dtype, cudaStream_t st) {
  const int K = p->K;
  const int NP3 = (K + 15) / 16 * 16;
  const int ntiles = (npix + TM - 1) / TM;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = ntiles < sms ? ntiles : sms;
  const size_t sm = sizeof(Smem) + 1024;
  cudaFuncSetAttribute(k_mlp_tc<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  cudaFuncSetAttribute(k_mlp_tc<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (w_dtype == DFP2S_W_BF16)
    k_mlp_tc<__nv_bfloat16><<<grid, THREADS, sm, st>>>(fields, p->J, npix, K, NP3, p->tc_w1, p->tc_w2, p->tc_w3, p->b1,
                                                      p->b2, p->tc_c3, p->out_scale, (__nv_bfloat16*)w, p->err);
  else
    k_mlp_tc<float><<<grid, THREADS, sm, st>>>(fields, p->J, npix, K, NP3, p->tc_w1, p->tc_w2, p->tc_w3, p->b1, p->b2,
                                              p->tc_c3, p->out_scale, (float*)w, p->err);
  return cudaGetLastError() == cudaSuccess ? DFP2S_OK : DFP2S_ECUDA;
}
