// Thread groups of the field sampler's FFT passes (shared by fields.cu and fields_full.cu).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "fft_reg.cuh"

// FFT groups per block: 8 up to N = 1024, then enough for 256 threads.
template <int N>
struct Groups {
  static constexpr int G = N >= 4096 ? 2 : (N >= 2048 ? 4 : 8);
  static constexpr int THREADS = G * fftr::Plan<N>::T;
  static constexpr int BUFE = (fftr::Plan<N>::BUF + 1) / 2 * 2;  // even: 16-byte aligned group buffers
  static constexpr int TS = 2 * G + 1;                     // tile row stride (complex), odd against conflicts
  static constexpr size_t smem_fft = (size_t)G * BUFE * sizeof(float2);
  static constexpr size_t smem_tile = (size_t)(N / 2 + 1) * TS * sizeof(float2);
  static constexpr size_t smem = smem_fft > smem_tile ? smem_fft : smem_tile;
};

