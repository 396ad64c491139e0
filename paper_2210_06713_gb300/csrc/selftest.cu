// Verification tap for the failure path of the tensor-core kernels.
//
// Every wait of the tensor-core kernels on an mbarrier is bounded; a wait that
// runs out sets the kernel's error word, and the kernel then still waits
// (bounded by its fixed 2 s limit) for the bulk copies it issued and releases
// its tensor memory before it exits, so the device context stays usable.  This
// kernel takes the same steps on a barrier that nothing ever completes: it
// allocates tensor memory, starts a bulk copy, waits on the dead barrier until
// the given limit runs out, lets the copy land, releases the tensor memory and
// reports the outcome in a status word.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "kernels.h"
#include "umma.cuh"

namespace {

constexpr uint64_t kCleanupNs = 2000000000ull;  // the kernels' fixed bound for their own copies

// status: 1 = the wait ran out (expected), 0 = it did not, 2 = the copy did not land in time
__global__ void k_wait_selftest(const uint4* __restrict__ src, uint64_t limit_ns, int* __restrict__ status) {
  __shared__ __align__(128) uint4 buf[16];
  __shared__ __align__(8) uint64_t never, copied;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x;
  if (tid == 0) {
    umma::mbar_init(&never, 1);
    umma::mbar_init(&copied, 1);
    umma::fence_mbar_init();
  }
  umma::tmem_alloc(&tmem_slot, 32);  // the whole (single) warp
  umma::tmem_relinquish();
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = tmem_slot;
  if (tid == 0) {
    umma::mbar_arrive_expect_tx(&copied, (uint32_t)sizeof(buf));
    umma::bulk_g2s(buf, src, (uint32_t)sizeof(buf), &copied);
    const bool ran_out = !umma::mbar_wait(&never, 0, limit_ns);
    const bool landed = umma::mbar_wait(&copied, 0, kCleanupNs);
    *status = !landed ? 2 : (ran_out ? 1 : 0);
  }
  umma::fence_before_sync();
  __syncthreads();
  umma::tmem_dealloc(tmem, 32);
}

}  // namespace

extern "C" int dfp2s_check_bounded_wait(uint64_t limit_ns, void* stream) {
  if (limit_ns < 1000 || limit_ns > 1000000000ull)
    return dfp2s_fail(DFP2S_EINVAL, "limit %llu ns out of [1 us, 1 s]", (unsigned long long)limit_ns);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  uint8_t* scratch = nullptr;  // 256 bytes copied by the kernel, then its status word
  cudaError_t e = dfp2s_device_malloc((void**)&scratch, 256 + 16);
  if (e != cudaSuccess) return dfp2s_fail_cuda(e, "self-test scratch");
  int h = -1;
  if ((e = cudaMemsetAsync(scratch, 0, 256 + 16, st)) == cudaSuccess) {
    k_wait_selftest<<<1, 32, 0, st>>>(reinterpret_cast<const uint4*>(scratch), limit_ns,
                                     reinterpret_cast<int*>(scratch + 256));
    if ((e = cudaGetLastError()) == cudaSuccess &&
        (e = cudaMemcpyAsync(&h, scratch + 256, sizeof(int), cudaMemcpyDeviceToHost, st)) == cudaSuccess)
      e = cudaStreamSynchronize(st);
  }
  cudaFree(scratch);
  if (e != cudaSuccess) return dfp2s_fail_cuda(e, "bounded-wait self-test");
  if (h == 1)
    return dfp2s_fail(DFP2S_ETIMEOUT, "the wait on a barrier nothing completes ran out after %llu ns (expected)",
                      (unsigned long long)limit_ns);
  if (h == 2) return dfp2s_fail(DFP2S_ECUDA, "self-test: the bulk copy did not land within its bound");
  return dfp2s_fail(DFP2S_ECUDA, "self-test: the wait on a barrier nothing completes did not run out");
}
