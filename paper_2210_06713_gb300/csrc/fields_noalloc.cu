// Field sampling for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc (or anything that allocates) at the time
// they draw a frame: a render or capture loop that runs under a fixed memory
// plan decided at start-up, a plug-in inside a host framework that owns the
// device allocator, or a loop with hard latency limits, where an allocation
// can synchronise the device or fail under memory pressure.  For them,
// dfp2s_sample_zernike_fields_noalloc runs the same kernels as
// dfp2s_sample_zernike_fields, but the FFT scratch spectrum lives in a
// statically sized device array owned by this library instead of in the
// factor handle.  The caller still provides the (already built) factor and the
// output buffer.
//
// The array below is reserved on every GPU that loads the library and is held
// until the process exits.  Its device address is looked up once per device
// (cudaGetSymbolAddress with that device current) on the first call made on
// that device; make that first call before any stream capture begins.
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace {

// 48 MiB of complex FP32: J (N/2+1) N <= 6,291,456, e.g. N = 512 with J <= 47,
// N = 256 with J <= 64, N = 1024 with J <= 11.
constexpr size_t kNoallocScratchElems = DFP2S_NOALLOC_SCRATCH_BYTES / sizeof(float2);

static __device__ __align__(256) float2 g_noalloc_scratch[kNoallocScratchElems];

constexpr int kMaxDevices = 64;
float2* g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

// Device address of g_noalloc_scratch on the current device (looked up once).
int scratch_for_current_device(float2** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return dfp2s_fail_cuda(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return dfp2s_fail(DFP2S_EUNSUPPORTED, "device ordinal %d too large", dev);
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return dfp2s_fail_cuda(e, "cudaGetSymbolAddress(static scratch)");
    g_scratch_ptr[dev] = static_cast<float2*>(p);
  }
  *out = g_scratch_ptr[dev];
  return DFP2S_OK;
}

}  // namespace

extern "C" int dfp2s_sample_zernike_fields_noalloc(const dfp2s_factor* f, double D_over_r0, uint64_t seed,
                                                   uint32_t frame, int H, int W, float* fields_dev, void* stream) {
  if (!f || !fields_dev) return dfp2s_fail(DFP2S_EINVAL, "null argument");
  if (H < 1 || W < 1 || H > f->d.N || W > f->d.N)
    return dfp2s_fail(DFP2S_EINVAL, "frame %dx%d does not fit the %d grid", H, W, f->d.N);
  if (!(D_over_r0 >= 0 && D_over_r0 <= 1e4)) return dfp2s_fail(DFP2S_EINVAL, "D/r0 = %g out of range", D_over_r0);
  const size_t need = (size_t)f->d.J * (f->d.N / 2 + 1) * f->d.N;
  if (need > kNoallocScratchElems)
    return dfp2s_fail(DFP2S_EINVAL,
                      "J=%d, N=%d needs %zu bytes of scratch; the static scratch holds %zu bytes "
                      "(use dfp2s_sample_zernike_fields)",
                      f->d.J, f->d.N, need * sizeof(float2), (size_t)DFP2S_NOALLOC_SCRATCH_BYTES);
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != f->device)
    return dfp2s_fail(DFP2S_EINVAL, "factor lives on device %d but device %d is current", f->device, dev);
  float2* scratch = nullptr;
  const int rc = scratch_for_current_device(&scratch);
  if (rc != DFP2S_OK) return rc;
  // every scratch entry the passes read is written earlier in the same call, so
  // nothing needs clearing between calls
  const float scale = (float)pow(D_over_r0, 5.0 / 6.0);
  if (dfp2s_launch_sample_fields(scratch, f->d.mult, f->d.tw, f->d.N, f->d.J, H, W, seed, frame, f->d.L32, scale,
                                 fields_dev, reinterpret_cast<cudaStream_t>(stream), nullptr, 0.f, true, -1,
                                 &f->d) != DFP2S_OK)
    return dfp2s_fail_cuda(dfp2s_launch_error(), "sample fields (static scratch)");
  return DFP2S_OK;
}
