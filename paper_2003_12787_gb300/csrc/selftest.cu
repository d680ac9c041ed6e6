// Self-test of the bounded device-side wait (the failure path of the
// tensor-core kernel's completion wait, exercised without any fault).
//
// One CTA initialises an mbarrier that expects one arrival, never arrives,
// and waits on it with the same bounded poll loop the mixed-precision kernel
// uses for its MMA completion. The wait runs out after `limit` polls, the CTA
// sets bit 1 of the handle's status word and returns; the host reads the word
// with stp_device_status (STP_ERR_TIMEOUT) and the context stays usable.
#include "mixed_kernels.cuh"

namespace stp {
namespace {

__global__ void __launch_bounds__(32, 1) wait_timeout_selftest(unsigned int* status, int limit) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mixed::mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const bool arrived = mixed::mbar_wait(&bar, 0u, limit);  // nothing arrives
  if (!arrived && threadIdx.x == 0) atomicOr(status, 2u);
}

}  // namespace

cudaError_t launch_wait_selftest(unsigned int* status, int limit, cudaStream_t stream) {
  wait_timeout_selftest<<<1, 32, 0, stream>>>(status, limit);
  return cudaGetLastError();
}

}  // namespace stp
