// Self-test of the device-side bounded waits (failure detection without a GPU
// fault): one block waits for an mbarrier transaction that is never issued,
// then for a flag that nothing sets.  Both waits use the library's bounded
// wait (the device wait limit of the status block); both give up, record
// their codes (31, 32) in the error word, and the kernel exits normally, so
// the context stays usable and hm_device_status reports HM_ETIMEOUT.  The
// kernel touches only its own shared memory and the status block.
#include "hm_api_internal.h"
#include "k_tc.cuh"

namespace hmi {

__global__ void k_selftest_timeout(DeviceStatusBlock* b) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  const uint32_t a = smem_u32(&bar);
  mbar_init(a, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  mbar_expect_tx(a, 16);          // the phase's only arrival, expecting 16 bytes that never come
  mbar_wait(a, 0, &b->err, 31);   // gives up after the wait limit
  const uint64_t limit = wait_limit_ns(&b->err);
  const uint64_t t0 = gtimer();
  while (atomicAdd(&b->flag, 0) == 0) {
    if (gtimer() - t0 > limit) {
      atomicExch(&b->err, 32);
      break;
    }
    __nanosleep(1000);
  }
}

hm_status launch_selftest_timeout(DeviceStatusBlock* b, cudaStream_t s) {
  k_selftest_timeout<<<1, 32, 0, s>>>(b);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("self-test launch failed: %s", cudaGetErrorString(e));
    return HM_ECUDA;
  }
  return HM_OK;
}

}  // namespace hmi
