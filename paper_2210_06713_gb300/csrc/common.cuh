// Shared device helpers for the DF-P2S kernels (sm_103a).
//
//  * Philox-4x32-10 counter-based generator (Salmon et al., SC 2011) and the
//    FP32 Box-Muller transform with this library's own log and sin/cos, written
//    so that every value is reproducible bit for bit on any IEEE FP32 machine:
//    each step is one correctly rounded operation (__fmul_rn, __fadd_rn, ...),
//    so no multiply-add is ever contracted.
//  * complex helpers and fixed DFTs of length 2, 4 and 8 in registers.
//  * status codes and launch-error checks used by the host code.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/dfp2s.h"

#define DFP2S_DEV __device__ __forceinline__

// ----------------------------------------------------------------- Philox
// The published round: two 32x32->64 multiplies, a Feistel-like permutation,
// and a Weyl-sequence key schedule.
DFP2S_DEV uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    if (r < 9) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
  }
  return c;
}

// Stream layout: key = seed, counter = (q, subsequence), subsequence =
// (tag << 40) | (frame << 8) | mode; counter q covers positions 4q..4q+3.
DFP2S_DEV uint4 philox_at(uint64_t seed, uint64_t sub, uint64_t q) {
  return philox4x32_10(make_uint4((uint32_t)q, (uint32_t)(q >> 32), (uint32_t)sub, (uint32_t)(sub >> 32)),
                       (uint32_t)seed, (uint32_t)(seed >> 32));
}

// (float) v for |v| < 2^22 without an integer-to-float conversion instruction
// (those share the special-function pipe): 1.5 2^23 + v is exact in FP32 and
// has v in its low mantissa bits, and the subtraction is exact.
DFP2S_DEV float dfp2s_small_int_to_float(int v) { return __fsub_rn(__int_as_float(0x4B400000 + v), 12582912.0f); }

// ln(u) for a positive normal FP32 u: u = 2^e m with m in [sqrt(1/2), sqrt(2)),
// ln m = 2 atanh(s) = 2s + s^3 (2/3 + s^2 (2/5 + s^2 (2/7 + s^2 (2/9 + s^2 2/11)))),
// s = (m-1)/(m+1); e ln 2 with ln 2 split into a 12-bit head and an FP32 tail.
// The x y + z steps are fused multiply-adds (one rounding each), the rest one
// IEEE operation each, in this order: the oracle reproduces every bit.
DFP2S_DEV float dfp2s_log(float u) {
  const uint32_t bits = __float_as_uint(u);
  int e = (int)(bits >> 23) - 127;
  float m = __uint_as_float((bits & 0x7FFFFFu) | 0x3F800000u);
  if (m > 0x1.6a09e6p+0f) {  // sqrt(2) rounded to FP32
    m = __fmul_rn(m, 0.5f);
    e += 1;
  }
  const float s = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
  const float s2 = __fmul_rn(s, s);
  float p = 0x1.745d18p-3f;                // 2/11
  p = __fmaf_rn(p, s2, 0x1.c71c72p-3f);  // 2/9
  p = __fmaf_rn(p, s2, 0x1.24924ap-2f);  // 2/7
  p = __fmaf_rn(p, s2, 0x1.99999ap-2f);  // 2/5
  p = __fmaf_rn(p, s2, 0x1.555556p-1f);  // 2/3
  const float logm = __fmaf_rn(__fmul_rn(s, s2), p, __fadd_rn(s, s));
  const float ef = dfp2s_small_int_to_float(e);        // |e| <= 149
  const float lo = __fmaf_rn(ef, 0x1.0bfbe8p-15f, logm);  // ln2 - head
  return __fmaf_rn(ef, 0x1.62ep-1f, lo);                 // head of ln 2 (12 significant bits: e * head exact)
}

// cos and sin of 2 pi u, u = (2k+1) 2^-24.  Quarter turns v = 4u = (2k+1) 2^-22;
// q = round(v) and r = v - q in [-1/2, 1/2] exactly in integers; Taylor series of
// sin((pi/2) r) to r^9 and cos((pi/2) r) to r^10, then the quadrant.
DFP2S_DEV void dfp2s_sincos_2pi(uint32_t k, float* cs, float* sn) {
  // k < 2^23, so num < 2^24 and every step is exact in 32-bit integers
  const int32_t num = 2 * (int32_t)k + 1;
  const int32_t q = (num + (1 << 21)) >> 22;
  const int32_t rnum = num - (q << 22);
  const float r = __fmul_rn(dfp2s_small_int_to_float(rnum), 0x1.0p-22f);  // |rnum| <= 2^21
  const float r2 = __fmul_rn(r, r);
  float sp = 0x1.507834p-13f;
  sp = __fmaf_rn(sp, r2, -0x1.32d2ccp-8f);
  sp = __fmaf_rn(sp, r2, 0x1.466bc6p-4f);
  sp = __fmaf_rn(sp, r2, -0x1.4abbcep-1f);
  sp = __fmaf_rn(sp, r2, 0x1.921fb6p+0f);
  const float s = __fmul_rn(r, sp);
  float cp = -0x1.a6d1f2p-16f;
  cp = __fmaf_rn(cp, r2, 0x1.e1f506p-11f);
  cp = __fmaf_rn(cp, r2, -0x1.55d3c8p-6f);
  cp = __fmaf_rn(cp, r2, 0x1.03c1fp-2f);
  cp = __fmaf_rn(cp, r2, -0x1.3bd3ccp+0f);
  const float c = __fmaf_rn(cp, r2, 1.0f);
  switch ((int)(q & 3)) {
    case 0: *cs = c; *sn = s; break;
    case 1: *cs = -s; *sn = c; break;
    case 2: *cs = -c; *sn = -s; break;
    default: *cs = s; *sn = -c; break;
  }
}

// Two N(0,1) samples from two Philox words: r = sqrt(-2 ln u_a), angle 2 pi u_b.
DFP2S_DEV float2 dfp2s_box_muller(uint32_t wa, uint32_t wb) {
  // u = (2 ka + 1) 2^-24 = (1 + ka 2^-23) - (1 - 2^-24), exact (Sterbenz)
  const uint32_t ka = wa >> 9;
  const float ua = __fsub_rn(__uint_as_float(0x3F800000u | ka), 0x1.fffffep-1f);
  const float t = __fmul_rn(dfp2s_log(ua), -2.0f);
  const float r = __fsqrt_rn(t);
  float c, s;
  dfp2s_sincos_2pi(wb >> 9, &c, &s);
  return make_float2(__fmul_rn(r, c), __fmul_rn(r, s));
}

// ---- the two Box-Muller transforms of a Philox block in lockstep on the two-lane FP32 instructions
// (add/sub/mul/fma .rn.f32x2 round each lane as the scalar __fadd_rn / __fsub_rn / __fmul_rn / __fmaf_rn do, so
// every Gaussian is the same bits as dfp2s_box_muller's; the divisions, square roots, bit manipulations and
// quadrant selections stay per lane).  Every multiply feeds a multiply, a fused multiply-add, a square root or
// a result, never an add: the assembler fuses a two-lane multiply followed by a two-lane add into one fused
// operation, which the unfused steps would not survive.
DFP2S_DEV uint64_t dfp2s_pk(float a, float b) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
DFP2S_DEV float2 dfp2s_upk(uint64_t v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}
DFP2S_DEV uint64_t dfp2s_add2(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
DFP2S_DEV uint64_t dfp2s_sub2(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
DFP2S_DEV uint64_t dfp2s_mul2(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
DFP2S_DEV uint64_t dfp2s_fma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
DFP2S_DEV uint64_t dfp2s_splat(float a) { return dfp2s_pk(a, a); }

// dfp2s_log of two values (the same operations in the same order, lane by lane)
DFP2S_DEV uint64_t dfp2s_log2x(float u0, float u1) {
  float mv[2];
  int ev[2];
  const float uu[2] = {u0, u1};
#pragma unroll
  for (int l = 0; l < 2; ++l) {
    const uint32_t bits = __float_as_uint(uu[l]);
    int e = (int)(bits >> 23) - 127;
    float m = __uint_as_float((bits & 0x7FFFFFu) | 0x3F800000u);
    if (m > 0x1.6a09e6p+0f) {
      m = __fmul_rn(m, 0.5f);  // exact: a fused m 0.5 - 1 below gives the same bits
      e += 1;
    }
    mv[l] = m;
    ev[l] = e;
  }
  const uint64_t m2 = dfp2s_pk(mv[0], mv[1]);
  const float2 num = dfp2s_upk(dfp2s_sub2(m2, dfp2s_splat(1.0f)));
  const float2 den = dfp2s_upk(dfp2s_add2(m2, dfp2s_splat(1.0f)));
  const uint64_t s = dfp2s_pk(__fdiv_rn(num.x, den.x), __fdiv_rn(num.y, den.y));
  const uint64_t s2 = dfp2s_mul2(s, s);
  uint64_t p = dfp2s_splat(0x1.745d18p-3f);
  p = dfp2s_fma2(p, s2, dfp2s_splat(0x1.c71c72p-3f));
  p = dfp2s_fma2(p, s2, dfp2s_splat(0x1.24924ap-2f));
  p = dfp2s_fma2(p, s2, dfp2s_splat(0x1.99999ap-2f));
  p = dfp2s_fma2(p, s2, dfp2s_splat(0x1.555556p-1f));
  const uint64_t logm = dfp2s_fma2(dfp2s_mul2(s, s2), p, dfp2s_add2(s, s));
  const uint64_t ef = dfp2s_pk(dfp2s_small_int_to_float(ev[0]), dfp2s_small_int_to_float(ev[1]));
  const uint64_t lo = dfp2s_fma2(ef, dfp2s_splat(0x1.0bfbe8p-15f), logm);
  return dfp2s_fma2(ef, dfp2s_splat(0x1.62ep-1f), lo);
}

// dfp2s_sincos_2pi of two arguments, lane by lane
DFP2S_DEV void dfp2s_sincos_2pi_2x(uint32_t k0, uint32_t k1, float2* cs, float2* sn) {
  const uint32_t kk[2] = {k0, k1};
  float rv[2];
  int32_t qv[2];
#pragma unroll
  for (int l = 0; l < 2; ++l) {
    const int32_t num = 2 * (int32_t)kk[l] + 1;
    const int32_t q = (num + (1 << 21)) >> 22;
    rv[l] = dfp2s_small_int_to_float(num - (q << 22));
    qv[l] = q;
  }
  const uint64_t r = dfp2s_mul2(dfp2s_pk(rv[0], rv[1]), dfp2s_splat(0x1.0p-22f));
  const uint64_t r2 = dfp2s_mul2(r, r);
  uint64_t sp = dfp2s_splat(0x1.507834p-13f);
  sp = dfp2s_fma2(sp, r2, dfp2s_splat(-0x1.32d2ccp-8f));
  sp = dfp2s_fma2(sp, r2, dfp2s_splat(0x1.466bc6p-4f));
  sp = dfp2s_fma2(sp, r2, dfp2s_splat(-0x1.4abbcep-1f));
  sp = dfp2s_fma2(sp, r2, dfp2s_splat(0x1.921fb6p+0f));
  const float2 s = dfp2s_upk(dfp2s_mul2(r, sp));
  uint64_t cp = dfp2s_splat(-0x1.a6d1f2p-16f);
  cp = dfp2s_fma2(cp, r2, dfp2s_splat(0x1.e1f506p-11f));
  cp = dfp2s_fma2(cp, r2, dfp2s_splat(-0x1.55d3c8p-6f));
  cp = dfp2s_fma2(cp, r2, dfp2s_splat(0x1.03c1fp-2f));
  cp = dfp2s_fma2(cp, r2, dfp2s_splat(-0x1.3bd3ccp+0f));
  const float2 c = dfp2s_upk(dfp2s_fma2(cp, r2, dfp2s_splat(1.0f)));
  const float sv[2] = {s.x, s.y}, cvv[2] = {c.x, c.y};
  float oc[2], os[2];
#pragma unroll
  for (int l = 0; l < 2; ++l) {
    switch ((int)(qv[l] & 3)) {
      case 0: oc[l] = cvv[l]; os[l] = sv[l]; break;
      case 1: oc[l] = -sv[l]; os[l] = cvv[l]; break;
      case 2: oc[l] = -cvv[l]; os[l] = -sv[l]; break;
      default: oc[l] = sv[l]; os[l] = -cvv[l]; break;
    }
  }
  *cs = make_float2(oc[0], oc[1]);
  *sn = make_float2(os[0], os[1]);
}

// Four Gaussians for positions 4q..4q+3 of one (seed, sub) stream: dfp2s_box_muller(w.x, w.y) and
// dfp2s_box_muller(w.z, w.w), evaluated together.
DFP2S_DEV float4 dfp2s_gauss4(uint64_t seed, uint64_t sub, uint64_t q) {
  const uint4 w = philox_at(seed, sub, q);
  const uint32_t ka = w.x >> 9, kb = w.z >> 9;
  const uint64_t ua = dfp2s_sub2(dfp2s_pk(__uint_as_float(0x3F800000u | ka), __uint_as_float(0x3F800000u | kb)),
                                 dfp2s_splat(0x1.fffffep-1f));
  const float2 uv = dfp2s_upk(ua);
  const float2 t = dfp2s_upk(dfp2s_mul2(dfp2s_log2x(uv.x, uv.y), dfp2s_splat(-2.0f)));
  const uint64_t r = dfp2s_pk(__fsqrt_rn(t.x), __fsqrt_rn(t.y));
  float2 c, s;
  dfp2s_sincos_2pi_2x(w.y >> 9, w.w >> 9, &c, &s);
  const float2 zc = dfp2s_upk(dfp2s_mul2(r, dfp2s_pk(c.x, c.y)));
  const float2 zs = dfp2s_upk(dfp2s_mul2(r, dfp2s_pk(s.x, s.y)));
  return make_float4(zc.x, zs.x, zc.y, zs.y);
}

DFP2S_DEV uint64_t dfp2s_subsequence(uint32_t tag, uint32_t frame, uint32_t mode) {
  return ((uint64_t)tag << 40) | ((uint64_t)frame << 8) | (uint64_t)mode;
}

// ---------------------------------------------------------------- complex
DFP2S_DEV float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
DFP2S_DEV float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
DFP2S_DEV float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
DFP2S_DEV float2 cmulc(float2 a, float2 b) {  // a * conj(b)
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
DFP2S_DEV float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
DFP2S_DEV float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <bool INV>
DFP2S_DEV float2 mul_mi(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// ---------------------------------------------------------- FFT building blocks
// In-register DFTs, unnormalised, sign -1 (forward) or +1 (INV) in the exponent.
template <bool INV>
DFP2S_DEV void dft2(float2& a, float2& b) {
  const float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <bool INV>
DFP2S_DEV void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
  const float2 s0 = cadd(a0, a2), d0 = csub(a0, a2);
  const float2 s1 = cadd(a1, a3), d1 = mul_mi<INV>(csub(a1, a3));
  a0 = cadd(s0, s1);
  a2 = csub(s0, s1);
  a1 = cadd(d0, d1);
  a3 = csub(d0, d1);
}

template <bool INV>
DFP2S_DEV void dft8(float2* v) {
  // radix-2 split into even/odd halves, each a DFT-4, then W8 twiddles.
  const float r = 0.70710678118654752f;
  float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<INV>(e0, e1, e2, e3);
  dft4<INV>(o0, o1, o2, o3);
  // o_k *= exp(-+ 2 pi i k / 8)
  o1 = INV ? make_float2(r * (o1.x - o1.y), r * (o1.x + o1.y)) : make_float2(r * (o1.x + o1.y), r * (o1.y - o1.x));
  o2 = mul_mi<INV>(o2);
  o3 = INV ? make_float2(-r * (o3.x + o3.y), r * (o3.x - o3.y)) : make_float2(r * (o3.y - o3.x), -r * (o3.x + o3.y));
  v[0] = cadd(e0, o0);
  v[4] = csub(e0, o0);
  v[1] = cadd(e1, o1);
  v[5] = csub(e1, o1);
  v[2] = cadd(e2, o2);
  v[6] = csub(e2, o2);
  v[3] = cadd(e3, o3);
  v[7] = csub(e3, o3);
}

// ------------------------------------------------------------- host helpers
#define DFP2S_CUDA_TRY(expr)                                      \
  do {                                                           \
    cudaError_t _e = (expr);                                     \
    if (_e != cudaSuccess) return dfp2s_fail_cuda(_e, #expr);    \
  } while (0)

int dfp2s_fail(int code, const char* fmt, ...);
int dfp2s_fail_cuda(cudaError_t e, const char* what);
// Device allocations of the library: cudaMalloc / cudaMallocAsync, unless a test
// has armed a simulated failure (dfp2s_debug_fail_allocation): the armed
// allocation then reports cudaErrorMemoryAllocation without allocating.
cudaError_t dfp2s_device_malloc(void** p, size_t bytes);
cudaError_t dfp2s_device_malloc_async(void** p, size_t bytes, cudaStream_t st);
// Status of the launches a launcher has just enqueued: reads (and so clears) the
// runtime's last error and, when it is one, keeps it for dfp2s_launch_error(),
// so that the entry point reporting the failure names the actual cause.
int dfp2s_launch_status();
// The error the last failing dfp2s_launch_status() of this thread saw (then
// forgotten); cudaGetLastError() when there is none.
cudaError_t dfp2s_launch_error();
