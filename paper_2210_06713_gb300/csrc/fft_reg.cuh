// Register-resident FFTs for the field sampler (sm_103a).
//
// An FFT of length N (power of two, 16 <= N <= 4096) is done by a group of
// T = N / V threads, V = min(N, 32) complex values per thread.  Element index
// n is held by thread n mod T as register n / T ("t + T m" layout) both before
// and after the transform, so a forward FFT's output feeds an inverse FFT
// without any data exchange, and a warp reads or writes a contiguous run of
// memory for each register.
//
// The transform is a Stockham autosort (Govindaraju et al., SC 2008) with a
// radix-V first pass, radix-32 passes while they fit, and one pass of the
// remaining radix: 1024 = 32 x 32, 4096 = 32 x 32 x 4, 512 = 32 x 16.  In the
// pass of radix R on sub-transforms of length Ns, butterfly j (k = j mod Ns)
// reads x[j + r N / R], multiplies by w^(r k) with w = exp(-+2 pi i / (Ns R)),
// does a DFT-R in registers and writes y[(j - k) R + k + r Ns].  Thread t owns
// the butterflies j = t + b T, b < V / R.  Between passes the values go through
// shared memory with one pad slot per 32 entries; within a warp (T <= 32) the
// exchange needs only __syncwarp, across warps __syncthreads, which the whole
// block then executes together.
//
// DFT-R for R in {2, 4, 8, 16, 32} uses fixed-twiddle decompositions
// (32 = 8 x 4, 16 = 4 x 4) whose constants are cos and sin of multiples of
// 2 pi / 32; pass twiddles come from an FP64-rounded table exp(-2 pi i m / N).
#pragma once

#include <utility>

#include "common.cuh"

namespace fftr {

// cos(2 pi m / 32) for m = 0..8
__device__ constexpr float kCos32[9] = {1.0f,
                                        0.980785280403230449126182236134f,
                                        0.923879532511286756128183189397f,
                                        0.831469612302545237078788377618f,
                                        0.707106781186547524400844362105f,
                                        0.555570233019602224742830813949f,
                                        0.382683432365089771728459984030f,
                                        0.195090322016128267848284868477f,
                                        0.0f};

// v *= exp(-+ 2 pi i M / 32) (forward sign -, INV sign +), with the trivial
// multiples of pi / 2 as swaps and the odd multiples of pi / 4 as two adds.
template <int M, bool INV>
DFP2S_DEV float2 twid32(float2 v) {
  constexpr int m = ((M % 32) + 32) % 32;
  if constexpr (m == 0) {
    return v;
  } else if constexpr (m == 8) {
    return mul_mi<INV>(v);
  } else if constexpr (m == 16) {
    return make_float2(-v.x, -v.y);
  } else if constexpr (m == 24) {
    return mul_mi<!INV>(v);
  } else {
    // angle theta = 2 pi m / 32; c = cos theta, s = sin theta from the first-octant table
    constexpr int q = m / 8, rm = m % 8;
    constexpr float c0 = kCos32[rm], s0 = kCos32[8 - rm];
    constexpr float c = q == 0 ? c0 : (q == 1 ? -s0 : (q == 2 ? -c0 : s0));
    constexpr float s = q == 0 ? s0 : (q == 1 ? c0 : (q == 2 ? -s0 : -c0));
    if constexpr (rm == 4) {
      // |c| = |s| = 1/sqrt(2): (x + i y)(c -+ i s) with one multiply per component
      constexpr float h = kCos32[4];
      if constexpr (!INV) {
        // (x c + y s) + i (y c - x s)
        return make_float2(h * ((c > 0 ? v.x : -v.x) + (s > 0 ? v.y : -v.y)),
                           h * ((c > 0 ? v.y : -v.y) - (s > 0 ? v.x : -v.x)));
      } else {
        // (x c - y s) + i (y c + x s)
        return make_float2(h * ((c > 0 ? v.x : -v.x) - (s > 0 ? v.y : -v.y)),
                           h * ((c > 0 ? v.y : -v.y) + (s > 0 ? v.x : -v.x)));
      }
    } else {
      if constexpr (!INV) return make_float2(fmaf(v.x, c, v.y * s), fmaf(v.y, c, -(v.x * s)));
      else return make_float2(fmaf(v.x, c, -(v.y * s)), fmaf(v.y, c, v.x * s));
    }
  }
}

// In-place DFT of R values in registers, natural order in and out.
template <int R, bool INV>
struct Dft;

template <bool INV>
struct Dft<2, INV> {
  static DFP2S_DEV void run(float2* v) { dft2<INV>(v[0], v[1]); }
};
template <bool INV>
struct Dft<4, INV> {
  static DFP2S_DEV void run(float2* v) {
    dft4<INV>(v[0], v[1], v[2], v[3]);
  }
};
template <bool INV>
struct Dft<8, INV> {
  static DFP2S_DEV void run(float2* v) { dft8<INV>(v); }
};

// Cooley-Tukey N = N1 N2 with n = N2 n1 + n2 and k = k1 + N1 k2:
//   X[k1 + N1 k2] = sum_n2 w_N2^(n2 k2) [ w_N^(n2 k1) sum_n1 x[N2 n1 + n2] w_N1^(n1 k1) ].
// Second stage for one k1 (a template argument, so each twiddle is a constant).
template <int N1, int N2, bool INV, int K1>
DFP2S_DEV void ct_column(const float2* y, float2* v) {
  static_assert(N2 <= 4, "second factor of at most 4");
  constexpr int S = 32 / (N1 * N2);  // w_N = w_32^S
  float2 b[N2];
  b[0] = y[K1];
  if constexpr (N2 > 1) b[1] = twid32<1 * K1 * S, INV>(y[1 * N1 + K1]);
  if constexpr (N2 > 2) b[2] = twid32<2 * K1 * S, INV>(y[2 * N1 + K1]);
  if constexpr (N2 > 3) b[3] = twid32<3 * K1 * S, INV>(y[3 * N1 + K1]);
  Dft<N2, INV>::run(b);
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) v[K1 + N1 * k2] = b[k2];
}

template <int N1, int N2, bool INV, int... K1>
DFP2S_DEV void ct_columns(const float2* y, float2* v, std::integer_sequence<int, K1...>) {
  (ct_column<N1, N2, INV, K1>(y, v), ...);
}

template <int N1, int N2, bool INV>
DFP2S_DEV void dft_ct(float2* v) {
  float2 y[N1 * N2];
#pragma unroll
  for (int n2 = 0; n2 < N2; ++n2) {
    float2 a[N1];
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) a[n1] = v[N2 * n1 + n2];
    Dft<N1, INV>::run(a);
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) y[n2 * N1 + k1] = a[k1];
  }
  ct_columns<N1, N2, INV>(y, v, std::make_integer_sequence<int, N1>{});
}

template <bool INV>
struct Dft<16, INV> {
  static DFP2S_DEV void run(float2* v) { dft_ct<4, 4, INV>(v); }
};
template <bool INV>
struct Dft<32, INV> {
  static DFP2S_DEV void run(float2* v) { dft_ct<8, 4, INV>(v); }
};

// ------------------------------------------------------------------ plan
template <int N>
struct Plan {
  static constexpr int V = N < 32 ? N : 32;  // values per thread
  static constexpr int T = N / V;            // threads per FFT
  // radices: V, then 32 while at least 32 remain, then the remainder
  static constexpr int R1 = V;
  static constexpr int REM1 = N / R1;  // = T
  static constexpr int R2 = REM1 >= 32 ? 32 : REM1;
  static constexpr int REM2 = REM1 / (R2 > 0 ? R2 : 1);
  static constexpr int R3 = REM2 >= 32 ? 32 : REM2;
  static constexpr int NPASS = (REM1 == 1) ? 1 : (REM2 == 1 ? 2 : 3);
  static_assert(N >= 16 && N <= 4096 && (N & (N - 1)) == 0, "N a power of two in [16, 4096]");
  static_assert(NPASS < 3 || REM2 / R3 == 1, "at most three passes");
  static constexpr int BUF = N + N / 32;  // padded shared-memory entries per FFT
};

DFP2S_DEV int pad32(int i) { return i + (i >> 5); }

template <int T>
DFP2S_DEV void group_sync() {
  if constexpr (T <= 32) __syncwarp();
  else __syncthreads();
}

// One Stockham pass on the registers (twiddles, DFT-R); the outputs stay in
// registers v[b R + r] = y[(j - k) R + k + r Ns], j = t + b T.
template <int N, int R, int Ns, bool INV>
DFP2S_DEV void pass_compute(float2 (&v)[Plan<N>::V], int t, const float2* __restrict__ tw) {
  constexpr int V = Plan<N>::V, T = Plan<N>::T, B = V / R;
#pragma unroll
  for (int b = 0; b < B; ++b) {
    if constexpr (Ns > 1) {
      const int j = t + b * T;
      const int k = j & (Ns - 1);
      constexpr int step = N / (Ns * R);
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const float2 w = __ldg(tw + r * k * step);
        v[b * R + r] = INV ? cmulc(v[b * R + r], w) : cmul(v[b * R + r], w);
      }
    }
    Dft<R, INV>::run(v + b * R);
  }
}

template <int N, int R, int Ns>
DFP2S_DEV void pass_store(const float2 (&v)[Plan<N>::V], float2* buf, int t) {
  constexpr int V = Plan<N>::V, T = Plan<N>::T, B = V / R;
#pragma unroll
  for (int b = 0; b < B; ++b) {
    const int j = t + b * T;
    const int k = j & (Ns - 1);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) buf[pad32(base + r * Ns)] = v[b * R + r];
  }
}

template <int N, int R>
DFP2S_DEV void pass_load(float2 (&v)[Plan<N>::V], const float2* buf, int t) {
  constexpr int V = Plan<N>::V, T = Plan<N>::T, B = V / R;
#pragma unroll
  for (int b = 0; b < B; ++b)
#pragma unroll
    for (int r = 0; r < R; ++r) v[b * R + r] = buf[pad32(t + b * T + r * (N / R))];
}

// Register index holding output element t + T m after the last pass of radix R:
// the last pass leaves y[j + r N / R] in v[b R + r], j = t + b T, i.e. m = b + (V / R) r.
template <int N>
struct OutIndex {
  static constexpr int V = Plan<N>::V;
  static constexpr int RL = Plan<N>::NPASS == 1 ? Plan<N>::R1 : (Plan<N>::NPASS == 2 ? Plan<N>::R2 : Plan<N>::R3);
  static DFP2S_DEV constexpr int reg(int m) { return (m % (V / RL)) * RL + m / (V / RL); }
};

// FFT of the group's data: in, v[m] = x[t + T m]; out, v[OutIndex<N>::reg(m)] = X[t + T m].
// `buf` is the group's shared-memory buffer (Plan<N>::BUF entries); every thread of the
// block must call this together when T > 32.  On return the buffer may be reused after a
// group_sync.
template <int N, bool INV>
DFP2S_DEV void fft(float2 (&v)[Plan<N>::V], float2* buf, int t, const float2* __restrict__ tw) {
  using P = Plan<N>;
  pass_compute<N, P::R1, 1, INV>(v, t, tw);
  if constexpr (P::NPASS >= 2) {
    pass_store<N, P::R1, 1>(v, buf, t);
    group_sync<P::T>();
    pass_load<N, P::R2>(v, buf, t);
    pass_compute<N, P::R2, P::R1, INV>(v, t, tw);
  }
  if constexpr (P::NPASS >= 3) {
    group_sync<P::T>();  // everyone has read pass 2's input before it is overwritten
    pass_store<N, P::R2, P::R1>(v, buf, t);
    group_sync<P::T>();
    pass_load<N, P::R3>(v, buf, t);
    pass_compute<N, P::R3, P::R1 * P::R2, INV>(v, t, tw);
  }
}

}  // namespace fftr
