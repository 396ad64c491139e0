// Surrogate P2S network (Sec. II-C) on the tcgen05 tensor cores: one fused
// kernel per frame, BF16 operands, FP32 accumulation in tensor memory, GELU by a
// logistic fit accurate far beyond the BF16 rounding of the activations.
//
// A tile is 128 consecutive pixels (MMA M = 128).  Tensor memory (512 columns)
// holds two 256-column regions; tile t computes in P = region t % 2 and
// Q = the other:
//   layer 1: X [128 x 48] (the J fields, zero-padded) x W1'^T + b1 -> P
//            (W1' = W1 diag(in_scale), resident in shared memory)
//   2 GELU(z) -> H1 (BF16), written back into P: each 16-column quarter of a
//            64-column chunk keeps its 16 activations in its first 8 columns
//   layer 2: H1 (A operand from tensor memory) x (W2 / 2)^T + b2 -> Q, W2 streamed
//            in four 64-wide K chunks
//   2 GELU(z) -> H2 in Q, the same way
//   layer 3: H2 (from tensor memory) x (W3 / 2)^T -> P columns [0, NP3)
//   w = y * out_scale + (b3 * out_scale + out_shift) -> staging rows in shared
//            memory; each pixel's flux s^T w (s_k = sum_u phi_k(u), four
//            partial sums per pixel) -> w += (1 - s^T w) s / (s^T s) in the
//            staging rows (reading R28: the P2S weights keep the PSF's unit
//            sum) -> global memory by one bulk copy (FP32 or BF16)
//
// The hidden biases enter the accumulators through one extra K = 16 MMA per
// layer (a tile of ones against the bias split into high and low bfloat16
// parts, exact to about 2^-17 relative), and the activations are stored doubled
// against halved weights of the next layer (both scalings by a power of two are
// exact).  The activations never touch shared memory, so the MMAs read only
// their weights there.
//
// Warp roles: warps 0-15 run the epilogues (warp w reads TMEM lanes 32 (w % 4)
// .. and a quarter of each chunk's columns), warp 16 issues the MMAs, warps 17
// and 19 convert the next tile's fields into X, warp 18 issues the weight copies.
// The epilogues hand each layer over in 64-column chunks (one mbarrier per
// chunk), so the next layer's MMAs start on a chunk while the epilogue works on
// the following one; every warp writes its activations only over accumulator
// columns it has read itself.  Layer 1 of the next tile runs on the tensor
// cores while the epilogues write out the current tile.  Weight chunks arrive
// by 1-D bulk copies into a three-deep ring; their MMAs release a slot through
// tcgen05.commit.  The copies have a warp of their own because a bulk copy can
// hold its issuing thread until the copy engine takes it, which would stall the
// MMA issue.  All waits are bounded; a wait that runs out sets the kernel's
// error word.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "gelu_fit.h"
#include "kernels.h"
#include "umma.cuh"

namespace {

constexpr int TM = 128;
constexpr int HID = 256;
constexpr int KX = 48;           // J padded to three K = 16 steps
constexpr int EPI_WARPS = 16;
constexpr int EPI_THREADS = EPI_WARPS * 32;
constexpr int PRODUCER_WARP = EPI_WARPS;
constexpr int LOADER_WARP = EPI_WARPS + 1;
constexpr int COPY_WARP = EPI_WARPS + 2;
constexpr int LOADER_WARP2 = EPI_WARPS + 3;
constexpr int THREADS = EPI_THREADS + 128;  // + MMA, copy and two loader warps
constexpr int NRING = 3;
constexpr int CHUNK_BYTES = HID * 64 * 2;  // one 64-wide K chunk of W2 (the largest)
constexpr int STAGE_BYTES = TM * 132 * 4;  // FP32 output rows of up to 128 (+4) weights
constexpr int ONES_BYTES = TM * 16 * 2;    // a 128 x 16 A operand, ones in two K columns
constexpr int BIAS_BYTES = HID * 16 * 2;   // the 256 x 16 B operand of the hidden biases
constexpr uint64_t kWaitNs = 2000000000ull;

struct Smem {
  uint8_t ring[NRING][CHUNK_BYTES];  // 96 KB
  uint8_t stage[STAGE_BYTES];        // 66 KB: the tile's output rows
  uint8_t W1[HID * KX * 2];          // 24 KB
  uint8_t X[TM * KX * 2];            // 12 KB
  uint8_t ONES[2][ONES_BYTES];       // 8 KB: ones in K columns 0, 1 (layer 1) and 2, 3 (layer 2)
  uint8_t BIAS[BIAS_BYTES];          // 8 KB: K columns 0, 1 = b1 (high and low bfloat16 parts), 2, 3 = b2
  float c3[128], s3[128];            // output bias and scale
  float fs[128], fg[128];            // s_k and s_k / (s^T s) of the unit-flux projection
  float mpart[4][TM];                // partial flux sums of the tile's pixels, one per epilogue slice
  uint64_t full[NRING], empty[NRING];
  uint64_t w1_full, x_ready, l1_done, l2_done, l3_done;
  uint64_t h_ready[4];
  uint32_t tmem_base;
  int abort;
};

// 2 GELU(z) = 2 z Phi(z) with the logistic fit of Phi in gelu_fit.h (max error
// 1.9e-5 in Phi), written as z (1 + tanh(z q ln2 / 2)) and evaluated with the
// hardware tanh.approx (one special-function instruction per activation; its
// absolute error, measured on sm_103a at 7.8e-6, leaves the 5.5e-5 GELU error of
// the fit unchanged).  tanh saturates to -1 for z -> -inf, so GELU -> 0 there.
DFP2S_DEV float tanh_approx(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// Per activation: s = min(z^2, Z2MAX), q = (c2 s + c1) s + c0 (the fit's coefficients times ln2 / 2), and
// 2 GELU(z) = z tanh(z q) + z; two activations at a time with the two-lane FP32 instructions (fma/mul .rn.f32x2,
// each lane rounded as the scalar instruction is), so the multiplies and the polynomial issue once per pair.
DFP2S_DEV uint64_t pack2(float a, float b) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
DFP2S_DEV float2 unpack2(uint64_t v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}
DFP2S_DEV uint64_t mul2(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
DFP2S_DEV uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
DFP2S_DEV float2 gelu2x_pair(float za, float zb) {
  constexpr float h = DFP2S_GELU_TANH_SCALE;
  constexpr float c0 = DFP2S_GELU_C0 * h, c1 = DFP2S_GELU_C1 * h, c2 = DFP2S_GELU_C2 * h;
  const uint64_t z = pack2(za, zb);
  const float2 zz = unpack2(mul2(z, z));
  const uint64_t sv = pack2(fminf(zz.x, DFP2S_GELU_Z2MAX), fminf(zz.y, DFP2S_GELU_Z2MAX));
  const uint64_t q = fma2(fma2(pack2(c2, c2), sv, pack2(c1, c1)), sv, pack2(c0, c0));
  const float2 a = unpack2(mul2(z, q));
  return unpack2(fma2(z, pack2(tanh_approx(a.x), tanh_approx(a.y)), z));
}

// byte offset of element (row, k) in a K-major no-swizzle tile with `kgroups` 8-element K groups per row group
DFP2S_DEV uint32_t kmajor_off(int row, int k, int kgroups) {
  return (uint32_t)(((row >> 3) * kgroups + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// Barrier of the epilogue warps (named barrier 1) that also ORs a flag over
// them, so that every epilogue thread takes the same abort decision.
DFP2S_DEV bool bar_epi_any(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, 1, %2, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(EPI_THREADS)
      : "memory");
  return r != 0;
}

// Barrier of the four epilogue warps that read TMEM lane quarter q4 (warps q4, q4 + 4, q4 + 8, q4 + 12):
// named barriers 2..5, 128 threads each.
DFP2S_DEV void bar_quarter(int q4) { asm volatile("bar.sync %0, 128;" ::"r"(2 + q4) : "memory"); }

// 1-D bulk copy shared -> global (both 16-byte aligned, size a multiple of 16) in a bulk group; wait until
// its source may be overwritten, or until every issued copy has completed.
DFP2S_DEV void bulk_s2g(void* dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(umma::smem_u32(src)),
               "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
DFP2S_DEV void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
DFP2S_DEV void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

template <typename WT>
DFP2S_DEV void wstore(WT* p, float v);
template <>
DFP2S_DEV void wstore<float>(float* p, float v) { *p = v; }
template <>
DFP2S_DEV void wstore<__nv_bfloat16>(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }

// Warp-wide load of 16 TMEM columns without waiting; tmem_wait16 waits for every
// outstanding load and ties the destination registers to the wait, so that no
// use of them is scheduled before it.
DFP2S_DEV void tmem_ld16_async(uint32_t taddr, float (&v)[16]) {
  uint32_t* r = reinterpret_cast<uint32_t*>(v);
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
DFP2S_DEV void tmem_wait16(float (&v)[16]) {
  uint32_t* r = reinterpret_cast<uint32_t*>(v);
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
               :
               : "memory");
}

// Hidden-layer epilogue of one epilogue warp (lane quarter q4, slice sl): for
// each 64-column chunk c of the 256-column region R, this warp's 16 columns
// [64 c + 16 sl, +16) (biases included) -> 2 GELU -> 8 columns of BF16 pairs
// written over the first 8 of those same columns (so no other warp reads what
// it writes), then the chunk is handed to the MMA warp.  Chunk c's K = 16 step
// ks therefore sits in columns [64 c + 16 ks, +8).  The next chunk's load is in
// flight meanwhile.
DFP2S_DEV void epilogue_gelu(Smem& s, uint32_t R, int warp, int lane, bool skip) {
  const int q4 = warp & 3, sl = warp >> 2;
  const uint32_t base = R + ((uint32_t)(q4 * 32) << 16) + 16 * sl;
  float d[2][16];
  tmem_ld16_async(base, d[0]);
  tmem_wait16(d[0]);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    float(&cur)[16] = d[c & 1];
    if (c < 3) tmem_ld16_async(base + 64 * (c + 1), d[(c + 1) & 1]);
    if (!skip) {
      uint32_t packed[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const float2 g = gelu2x_pair(cur[2 * e], cur[2 * e + 1]);
        __nv_bfloat162 h2 = __floats2bfloat162_rn(g.x, g.y);
        packed[e] = *reinterpret_cast<uint32_t*>(&h2);
      }
      umma::tmem_st8(base + 64 * c, packed);
      umma::tmem_wait_st();
    }
    umma::fence_before_sync();  // TMEM reads and writes ordered before the hand-over
    __syncwarp();
    if (lane == 0) umma::mbar_arrive(&s.h_ready[c]);
    if (c < 3) tmem_wait16(d[(c + 1) & 1]);
  }
}

template <typename WT, bool SCALED>
__global__ void __launch_bounds__(THREADS, 1)
    k_mlp_tc(const float* __restrict__ fields, int J, int npix, int K, int NP3, const __nv_bfloat16* __restrict__ w1t,
             const __nv_bfloat16* __restrict__ w2c, const __nv_bfloat16* __restrict__ w3c,
             const __nv_bfloat16* __restrict__ bias, const float* __restrict__ c3, const float* __restrict__ s3,
             const float* __restrict__ flux, WT* __restrict__ wout, int KS, int vec_out, int* __restrict__ err,
             float xscale) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  Smem& s = *reinterpret_cast<Smem*>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntiles = (npix + TM - 1) / TM;
  const int my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

  if (tid == 0) {
    for (int i = 0; i < NRING; ++i) {
      umma::mbar_init(&s.full[i], 1);
      umma::mbar_init(&s.empty[i], 1);
    }
    umma::mbar_init(&s.w1_full, 1);
    umma::mbar_init(&s.x_ready, 2);
    umma::mbar_init(&s.l1_done, 1);
    umma::mbar_init(&s.l2_done, 1);
    umma::mbar_init(&s.l3_done, 1);
    for (int c = 0; c < 4; ++c) umma::mbar_init(&s.h_ready[c], EPI_WARPS);
    s.abort = 0;
    umma::fence_mbar_init();
  }
  for (int i = tid; i < 128; i += THREADS) {
    s.c3[i] = i < K ? c3[i] : 0.f;
    s.s3[i] = i < K ? s3[i] : 0.f;
    s.fs[i] = i < K ? flux[i] : 0.f;
    s.fg[i] = i < K ? flux[K + i] : 0.f;
  }
  // zero X once (the padded K columns stay zero); the ones tiles of the bias MMAs
  for (int i = tid; i < TM * KX * 2 / 16; i += THREADS) reinterpret_cast<uint4*>(s.X)[i] = make_uint4(0, 0, 0, 0);
  for (int i = tid; i < 2 * TM * 16; i += THREADS) {
    const int g = i / (TM * 16), r = (i / 16) % TM, k = i % 16;
    const __nv_bfloat16 v = __float2bfloat16_rn((k >> 1) == g ? 1.f : 0.f);
    *reinterpret_cast<__nv_bfloat16*>(s.ONES[g] + kmajor_off(r, k, 2)) = v;
  }
  umma::fence_proxy_async_smem();  // X and the ones tiles -> the tensor cores' reads
  if (warp == 0) {
    umma::tmem_alloc(&s.tmem_base, 512);
    umma::tmem_relinquish();
  }
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = s.tmem_base;

  if (warp == PRODUCER_WARP) {
    // ------------------------------------------------------------ MMA issue
    if (lane == 0) {
      // K-major no-swizzle descriptors: X and W1 with 6 K groups per 8-row group, weight chunks with 8, the ones
      // and bias tiles with 2; per-MMA descriptors add (byte offset >> 4)
      const uint64_t x_desc = umma::sdesc(umma::smem_u32(s.X), 128, 768);
      const uint64_t w1_desc = umma::sdesc(umma::smem_u32(s.W1), 128, 768);
      const uint64_t ring_desc = umma::sdesc(umma::smem_u32(s.ring[0]), 128, 1024);
      const uint64_t ones1_desc = umma::sdesc(umma::smem_u32(s.ONES[0]), 128, 256);
      const uint64_t ones2_desc = umma::sdesc(umma::smem_u32(s.ONES[1]), 128, 256);
      const uint64_t bias_desc = umma::sdesc(umma::smem_u32(s.BIAS), 128, 256);
      const uint32_t idesc1 = umma::idesc_bf16(TM, HID);
      const uint32_t idesc3 = umma::idesc_bf16(TM, NP3);
      uint32_t u_use = 0;
      bool ok = true;
      // MMAs of one 64-wide K chunk: weight chunk u in the ring against the activations of the chunk that
      // starts at tensor-memory address a (K = 16 step ks in columns [a + 16 ks, +8))
      auto chunk_mmas = [&](uint32_t u, uint32_t a, uint32_t d, uint32_t id, bool first) {
        const int b = u % NRING;
        if (!umma::mbar_wait(&s.full[b], (u / NRING) & 1, kWaitNs)) {
          ok = false;
          return;
        }
        umma::fence_after_sync();
        const uint64_t b_c = ring_desc + (uint64_t)(b * (CHUNK_BYTES >> 4));
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) umma::mma_bf16_ta(d, a + 16 * ks, b_c + 16 * ks, id, !(first && ks == 0));
        umma::mma_commit(&s.empty[b]);
      };
      if (my_tiles > 0 && !umma::mbar_wait(&s.w1_full, 0, kWaitNs)) ok = false;
      for (int t = 0; t < my_tiles && ok; ++t) {
        const uint32_t P = tmem + ((t & 1) ? 256u : 0u), Q = tmem + ((t & 1) ? 0u : 256u);
        // layer 1 writes P, where the previous tile's second activations were read by its layer-3 MMAs
        if (t >= 1 && !umma::mbar_wait(&s.l3_done, (t - 1) & 1, kWaitNs)) {
          ok = false;
          break;
        }
        if (!umma::mbar_wait(&s.x_ready, t & 1, kWaitNs)) {
          ok = false;
          break;
        }
        umma::fence_after_sync();
#pragma unroll
        for (int ks = 0; ks < KX / 16; ++ks) umma::mma_bf16(P, x_desc + 16 * ks, w1_desc + 16 * ks, idesc1, ks != 0);
        umma::mma_bf16(P, ones1_desc, bias_desc, idesc1, 1);  // + b1
        umma::mma_commit(&s.l1_done);
        // layer 2 into Q on the first epilogue's chunks (h_ready completion 2t); Q is free once chunk 0 has
        // arrived (the epilogues finished the previous tile's outputs, which sat in Q, before this tile)
        for (int c = 0; c < 4 && ok; ++c) {
          if (!umma::mbar_wait(&s.h_ready[c], 0, kWaitNs)) {
            ok = false;
            break;
          }
          umma::fence_after_sync();
          if (c == 0) umma::mma_bf16(Q, ones2_desc, bias_desc, idesc1, 0);  // accumulator = b2
          chunk_mmas(u_use++, P + 64 * c, Q, idesc1, false);
        }
        if (!ok) break;
        umma::mma_commit(&s.l2_done);
        // layer 3 into P columns [0, NP3) on the second epilogue's chunks (completion 2t + 1); the first
        // activations there were read by the layer-2 MMAs, complete before the second epilogue began
        for (int c = 0; c < 4 && ok; ++c) {
          if (!umma::mbar_wait(&s.h_ready[c], 1, kWaitNs)) {
            ok = false;
            break;
          }
          umma::fence_after_sync();
          chunk_mmas(u_use++, Q + 64 * c, P, idesc3, c == 0);
        }
        if (!ok) break;
        umma::mma_commit(&s.l3_done);
      }
      if (!ok) {
        s.abort = 1;
        atomicExch(err, 2);
      }
      // the MMAs finish before the CTA exits (bounded)
      if (u_use > 0) umma::mbar_wait(&s.empty[(u_use - 1) % NRING], ((u_use - 1) / NRING) & 1, kWaitNs);
    }
  } else if (warp == COPY_WARP) {
    // ------------------------------------------------------------ weight copies
    if (lane == 0 && my_tiles > 0) {
      const uint32_t w3_bytes = (uint32_t)(NP3 * 64 * 2);
      const uint32_t total = (uint32_t)my_tiles * 8;  // 4 chunks of W2 then 4 of W3 per tile
      umma::mbar_arrive_expect_tx(&s.w1_full, HID * KX * 2 + BIAS_BYTES);
      umma::bulk_g2s(s.W1, w1t, HID * KX * 2, &s.w1_full);
      umma::bulk_g2s(s.BIAS, bias, BIAS_BYTES, &s.w1_full);
      uint32_t u = 0;
      for (; u < total; ++u) {
        const int b = u % NRING;
        if (u >= NRING) {
          // the slot is free once the MMAs of chunk u - NRING have completed; stop early if the
          // MMA warp has given up
          const uint64_t t0 = umma::global_ns();
          bool got = false;
          while (!(got = umma::mbar_ready(&s.empty[b], ((u / NRING) - 1) & 1))) {
            if (*reinterpret_cast<volatile int*>(&s.abort)) break;
            if (umma::global_ns() - t0 > kWaitNs) {
              s.abort = 1;
              atomicExch(err, 2);
              break;
            }
          }
          if (!got) break;
        }
        // chunk u: W2 chunk u % 8 for u % 8 < 4, else W3 chunk u % 8 - 4
        const int c = u % 8;
        if (c < 4) {
          umma::mbar_arrive_expect_tx(&s.full[b], CHUNK_BYTES);
          umma::bulk_g2s(s.ring[b], w2c + (size_t)c * (HID * 64), CHUNK_BYTES, &s.full[b]);
        } else {
          umma::mbar_arrive_expect_tx(&s.full[b], w3_bytes);
          umma::bulk_g2s(s.ring[b], w3c + (size_t)(c - 4) * (NP3 * 64), w3_bytes, &s.full[b]);
        }
      }
      // every issued copy lands before the CTA exits (bounded): copies before u - NRING were
      // consumed by the MMA warp before their slots were reissued
      for (uint32_t v = u > NRING ? u - NRING : 0; v < u; ++v)
        umma::mbar_wait(&s.full[v % NRING], (v / NRING) & 1, kWaitNs);
      umma::mbar_wait(&s.w1_full, 0, kWaitNs);
    }
  } else if (warp == LOADER_WARP || warp == LOADER_WARP2) {
    // ------------------------------------------------------------ loaders: fields -> X (bf16, K-major); the
    // two warps take alternate groups of eight fields
    const int l = warp == LOADER_WARP ? 0 : 1;
    for (int t = 0; t < my_tiles; ++t) {
      // X is free once layer 1 of the previous tile has completed
      if (t >= 1 && !umma::mbar_wait(&s.l1_done, (t - 1) & 1, kWaitNs)) s.abort = 1;
      if (s.abort) break;
      const int p0 = (blockIdx.x + t * gridDim.x) * TM;
      // eight fields at a time for this lane's four pixels (32 loads in flight), packed into the
      // 16-byte rows of the K-major core matrices (fields j..j+7 of one pixel)
      for (int jg = l; jg < (J + 7) / 8 && jg < KX / 8; jg += 2) {
        float v[4][8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int j = jg * 8 + e;
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const int pp = r * 32 + lane;
            v[r][e] = (j < J && p0 + pp < npix) ? __ldg(fields + (size_t)j * npix + p0 + pp) : 0.f;
          }
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          uint32_t wd[4];
#pragma unroll
          for (int e2 = 0; e2 < 4; ++e2) {
            const float x0 = SCALED ? v[r][2 * e2] * xscale : v[r][2 * e2];
            const float x1 = SCALED ? v[r][2 * e2 + 1] * xscale : v[r][2 * e2 + 1];
            __nv_bfloat162 h2 = __floats2bfloat162_rn(x0, x1);
            wd[e2] = *reinterpret_cast<uint32_t*>(&h2);
          }
          *reinterpret_cast<uint4*>(s.X + kmajor_off(r * 32 + lane, jg * 8, KX / 8)) = make_uint4(wd[0], wd[1], wd[2], wd[3]);
        }
      }
      umma::fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) umma::mbar_arrive(&s.x_ready);
    }
  } else {
    // ------------------------------------------------------------ epilogue warps
    const int q4 = warp & 3, sl = warp >> 2;
    const int p = q4 * 32 + lane;
    const uint32_t lane_base = (uint32_t)(q4 * 32) << 16;
    float* stage = reinterpret_cast<float*>(s.stage);
    volatile int* abort_flag = &s.abort;
    for (int t = 0; t < my_tiles; ++t) {
      const int tile = blockIdx.x + t * gridDim.x;
      const int p0 = tile * TM;
      const uint32_t P = tmem + ((t & 1) ? 256u : 0u), Q = tmem + ((t & 1) ? 0u : 256u);
      // a failed wait turns the work off (the hand-overs still happen)
      bool skip = *abort_flag != 0;
      if (!skip && !umma::mbar_wait_backoff(&s.l1_done, t & 1, kWaitNs)) skip = true;
      umma::fence_after_sync();
      epilogue_gelu(s, P, warp, lane, skip);
      if (!skip && !umma::mbar_wait_backoff(&s.l2_done, t & 1, kWaitNs)) skip = true;
      umma::fence_after_sync();
      epilogue_gelu(s, Q, warp, lane, skip);
      if (!skip && !umma::mbar_wait_backoff(&s.l3_done, t & 1, kWaitNs)) skip = true;
      umma::fence_after_sync();
      if (skip) *abort_flag = 1;
      // the previous tile's bulk copy has finished reading the staging rows (its issuing thread waits, the
      // barrier passes that on)
      if (vec_out == 2 && tid == 0) bulk_wait_read();
      if (bar_epi_any(skip)) break;
      // outputs: TMEM P [0, NP3) -> y * s3 + c3 in registers (groups q = sl and sl + 4 of 16 columns; NP3 <= 128)
      // with this slice's part of the pixel's flux s^T w (columns past K hold s_k = 0); the four slices of a
      // pixel (the warps sharing its TMEM lane quarter) exchange their parts, then each writes its columns of
      // the unit-flux weights w + (1 - s^T w) s / (s^T s) into FP32 rows of stride KS in the staging area
      const int ngrp = NP3 / 16;
      float o[2][16];
      uint64_t mp2 = 0;  // two lanes of the flux partial sum (even and odd columns)
#pragma unroll
      for (int iq = 0; iq < 2; ++iq) {
        const int q = sl + 4 * iq;
        if (q < ngrp) {
          umma::tmem_ld16(P + lane_base + q * 16, o[iq]);
#pragma unroll
          for (int i = 0; i < 16; i += 2) {  // pairs of columns: two-lane FP32 FMAs, 8-byte broadcast loads
            const int k = q * 16 + i;
            const float2 sc = *reinterpret_cast<const float2*>(&s.s3[k]);
            const float2 cc = *reinterpret_cast<const float2*>(&s.c3[k]);
            const float2 fc = *reinterpret_cast<const float2*>(&s.fs[k]);
            const uint64_t y = fma2(pack2(o[iq][i], o[iq][i + 1]), pack2(sc.x, sc.y), pack2(cc.x, cc.y));
            mp2 = fma2(y, pack2(fc.x, fc.y), mp2);
            const float2 yy = unpack2(y);
            o[iq][i] = yy.x;
            o[iq][i + 1] = yy.y;
          }
        }
      }
      const float2 mpp = unpack2(mp2);
      s.mpart[sl][p] = mpp.x + mpp.y;
      umma::fence_before_sync();
      bar_quarter(q4);
      const float cfl = 1.f - ((s.mpart[0][p] + s.mpart[1][p]) + (s.mpart[2][p] + s.mpart[3][p]));
#pragma unroll
      for (int iq = 0; iq < 2; ++iq) {
        const int q = sl + 4 * iq;
        if (q < ngrp) {
#pragma unroll
          for (int i4 = 0; i4 < 4; ++i4) {
            const int k = q * 16 + 4 * i4;
            if (k < K) {
              const float4 g = *reinterpret_cast<const float4*>(&s.fg[k]);
              const uint64_t c2 = pack2(cfl, cfl);
              const float2 a = unpack2(fma2(c2, pack2(g.x, g.y), pack2(o[iq][4 * i4 + 0], o[iq][4 * i4 + 1])));
              const float2 b = unpack2(fma2(c2, pack2(g.z, g.w), pack2(o[iq][4 * i4 + 2], o[iq][4 * i4 + 3])));
              *reinterpret_cast<float4*>(stage + p * KS + k) = make_float4(a.x, a.y, b.x, b.y);
            }
          }
        }
      }
      if (vec_out == 2) umma::fence_proxy_async_smem();  // staging rows -> the bulk copy below
      bar_epi_any(false);
      const int nlive = min(TM, npix - p0);
      WT* dst = wout + (size_t)p0 * K;
      if (vec_out == 2) {
        // staging rows are contiguous (KS == K): one bulk copy of the tile's outputs, shared -> global; the
        // next tile waits for its reads before writing the staging rows again
        if (tid == 0) bulk_s2g(dst, stage, (uint32_t)(nlive * K * 4));
      } else if (vec_out) {  // FP32 with K % 4 == 0 and 16-byte aligned rows
        const int n4 = nlive * K / 4;
        for (int i = tid; i < n4; i += EPI_THREADS) {
          const int e = 4 * i;
          const int pp = e / K, k = e - pp * K;
          reinterpret_cast<float4*>(dst)[i] = *reinterpret_cast<const float4*>(stage + pp * KS + k);
        }
      } else {
        for (int i = tid; i < nlive * K; i += EPI_THREADS) {
          const int pp = i / K, k = i - pp * K;
          wstore<WT>(dst + i, stage[pp * KS + k]);
        }
      }
    }
    if (*abort_flag && tid == 0) atomicExch(err, 2);
    if (vec_out == 2 && tid == 0) bulk_wait_all();  // the last tile's outputs have reached global memory
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

// scale W[n][k] (given transposed: Wt[k * ncols + n]) -> chunks [kc][n/8][k%64/8][8][8] for n < nrows_pad
__global__ void k_pack_chunks(const float* __restrict__ Wt, int nrows, int nrows_pad, int ncols_t, float scale,
                              __nv_bfloat16* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // over 4 chunks x nrows_pad x 64
  if (i >= 4 * nrows_pad * 64) return;
  const int kc = i / (nrows_pad * 64);
  const int rem = i - kc * nrows_pad * 64;
  const int n = rem / 64, kk = rem - n * 64;
  const int k = kc * 64 + kk;
  const float v = n < nrows ? Wt[(size_t)k * ncols_t + n] * scale : 0.f;
  out[(size_t)kc * nrows_pad * 64 + kmajor_off(n, kk, 8) / 2] = __float2bfloat16_rn(v);
}

// hidden biases -> the 256 x 16 K-major B operand of the bias MMAs: K columns 0, 1 hold
// b1 = hi + lo (hi = bf16(b1), lo = bf16(b1 - hi)), columns 2, 3 the same split of b2
__global__ void k_pack_bias(const float* __restrict__ b1, const float* __restrict__ b2,
                            __nv_bfloat16* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // over 256 x 16
  if (i >= HID * 16) return;
  const int n = i / 16, k = i % 16;
  float v = 0.f;
  if (k < 4) {
    const float b = k < 2 ? b1[n] : b2[n];
    const float hi = __bfloat162float(__float2bfloat16_rn(b));
    v = (k & 1) ? b - hi : hi;
  }
  out[kmajor_off(n, k, 2) / 2] = __float2bfloat16_rn(v);
}

// W1 diag(in_scale) L (L lower triangular, J x J row-major), packed as k_pack_w1: the first layer of the same
// network for the fields before their mixing by L
__global__ void k_pack_w1_mixed(const float* __restrict__ W1t, const float* __restrict__ in_scale,
                                const float* __restrict__ L, int J, __nv_bfloat16* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // over 256 x 48
  if (i >= HID * KX) return;
  const int n = i / KX, j = i - n * KX;
  float v = 0.f;
  for (int r = j; r < J; ++r) v = fmaf(W1t[(size_t)r * HID + n] * in_scale[r], L[r * J + j], v);
  out[kmajor_off(n, j, KX / 8) / 2] = __float2bfloat16_rn(v);
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
  if (!p->tc_w1 && (dfp2s_device_malloc((void**)&p->tc_w1, HID * KX * sizeof(__nv_bfloat16)) != cudaSuccess ||
                    dfp2s_device_malloc((void**)&p->tc_w2, 4 * HID * 64 * sizeof(__nv_bfloat16)) != cudaSuccess ||
                    dfp2s_device_malloc((void**)&p->tc_w3, 4 * 128 * 64 * sizeof(__nv_bfloat16)) != cudaSuccess ||
                    dfp2s_device_malloc((void**)&p->tc_c3, 128 * sizeof(float)) != cudaSuccess ||
                    dfp2s_device_malloc((void**)&p->tc_bias, HID * 16 * sizeof(__nv_bfloat16)) != cudaSuccess))
    return DFP2S_ENOMEM;
  // the SIMT layout keeps W1, W2, W3 transposed: W1t (J x 256), W2t (256 x 256), W3t (256 x K)
  k_pack_w1<<<(HID * KX + 255) / 256, 256, 0, st>>>(p->W1, p->in_scale, p->J, p->tc_w1);
  // the hidden layers store 2 GELU: the weights that read them are halved (exact in bfloat16)
  k_pack_chunks<<<(4 * HID * 64 + 255) / 256, 256, 0, st>>>(p->W2, HID, HID, HID, 0.5f, p->tc_w2);
  k_pack_chunks<<<(4 * NP3 * 64 + 255) / 256, 256, 0, st>>>(p->W3, K, NP3, K, 0.5f, p->tc_w3);
  k_pack_bias<<<HID * 16 / 256, 256, 0, st>>>(p->b1, p->b2, p->tc_bias);
  k_out_affine<<<1, 128, 0, st>>>(p->b3, p->out_scale, p->out_shift, K, p->tc_c3);
  return dfp2s_launch_status();
}

size_t dfp2s_mlp_tc_w1_elems() { return (size_t)HID * KX; }

template <typename WT, bool SCALED>
static void launch_mlp(const float* fields, const dfp2s_p2s_dev* p, int npix, int K, int NP3, const __nv_bfloat16* w1,
                       WT* out, int KS, int vec_out, float xscale, int grid, size_t sm, cudaStream_t st) {
  cudaFuncSetAttribute(k_mlp_tc<WT, SCALED>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_mlp_tc<WT, SCALED><<<grid, THREADS, sm, st>>>(fields, p->J, npix, K, NP3, w1, p->tc_w2, p->tc_w3, p->tc_bias,
                                                  p->tc_c3, p->out_scale, p->flux, out, KS, vec_out, p->err, xscale);
}

int dfp2s_mlp_tc_pack_w1_mixed(const dfp2s_p2s_dev* p, const float* L, __nv_bfloat16* out, cudaStream_t st) {
  if (p->J > KX) return DFP2S_EUNSUPPORTED;
  k_pack_w1_mixed<<<(HID * KX + 255) / 256, 256, 0, st>>>(p->W1, p->in_scale, L, p->J, out);
  return dfp2s_launch_status();
}

int dfp2s_launch_mlp_tc(const dfp2s_p2s_dev* p, const float* fields, int npix, void* w, int w_dtype, cudaStream_t st,
                        const __nv_bfloat16* w1, float xscale) {
  if (!w1) w1 = p->tc_w1;
  const int K = p->K;
  if (p->J > KX) return DFP2S_EUNSUPPORTED;  // the input tile holds at most 48 fields
  const int NP3 = (K + 15) / 16 * 16;
  const int ntiles = (npix + TM - 1) / TM;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = ntiles < sms ? ntiles : sms;
  // staging row stride: a multiple of 4 floats with an odd number of 16-byte units (no bank conflicts)
  int KS = (K + 3) / 4 * 4;
  if ((KS / 4) % 2 == 0) KS += 4;
  // 2: contiguous staging rows (KS == K), one bulk copy per tile; 1: vector copy loop; 0: scalar loop
  int vec_out = (w_dtype == DFP2S_W_F32) && (K % 4) == 0 && ((uintptr_t)w & 15) == 0;
  if (vec_out && KS == K) vec_out = 2;
  const size_t sm = sizeof(Smem) + 1024;
  static_assert(sizeof(Smem) + 1024 <= 227 * 1024, "shared memory layout");
  const bool scaled = xscale != 1.f;
  if (w_dtype == DFP2S_W_BF16) {
    __nv_bfloat16* o = (__nv_bfloat16*)w;
    if (scaled) launch_mlp<__nv_bfloat16, true>(fields, p, npix, K, NP3, w1, o, KS, 0, xscale, grid, sm, st);
    else launch_mlp<__nv_bfloat16, false>(fields, p, npix, K, NP3, w1, o, KS, 0, xscale, grid, sm, st);
  } else {
    float* o = (float*)w;
    if (scaled) launch_mlp<float, true>(fields, p, npix, K, NP3, w1, o, KS, vec_out, xscale, grid, sm, st);
    else launch_mlp<float, false>(fields, p, npix, K, NP3, w1, o, KS, vec_out, xscale, grid, sm, st);
  }
  return dfp2s_launch_status();
}
