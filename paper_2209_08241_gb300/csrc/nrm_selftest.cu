// Self-test of the bounded waits every kernel of this library uses (no
// counterpart in the paper). One CTA waits on a shared-memory barrier that
// nothing ever completes: warp 0 with the warp-level wait (lane 0 polls),
// warp 1 with the per-thread wait. Both give up after timeout_ns of global
// time, record NRM_ERR_TIMEOUT in the status word and return, which is the
// path a kernel takes when a copy it waits for does not land. No copy, no
// fault, and the context stays usable.
#include "nrm_device.cuh"

namespace nrm {

using namespace dev;

namespace {

__global__ void __launch_bounds__(64) wait_expiry_kernel(unsigned long long timeout_ns, int* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);  // one arrival would complete phase 0; none comes
    fence_barrier_init();
  }
  __syncthreads();
  bool ok;
  if (threadIdx.x < 32)
    ok = mbar_wait_warp(smem_u32(&bar), 0, timeout_ns);
  else
    ok = mbar_wait_bounded(smem_u32(&bar), 0, timeout_ns);
  if (!ok && (threadIdx.x & 31) == 0) record_error(status + (threadIdx.x >> 5), NRM_ERR_TIMEOUT);
}

}  // namespace

cudaError_t launch_wait_expiry(unsigned long long timeout_ns, int* status2, cudaStream_t stream) {
  void* args[2] = {&timeout_ns, &status2};
  return cudaLaunchKernel((const void*)wait_expiry_kernel, dim3(1), dim3(64), args, 0, stream);
}

}  // namespace nrm
