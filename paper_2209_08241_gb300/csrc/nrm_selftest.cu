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

#ifdef NRM_DEBUG_CHECKS
namespace {
// The range checks of the checking build, evaluated on addresses inside and
// just outside a block's dynamic shared memory (256 bytes at launch), an
// 8-int global array and a 5-element index range. Only the addresses are
// formed and compared; nothing outside a buffer is read or written.
// results[0..6] = 1, 1, 0, 0, 1, 0, 0 when the checks are right; the failed
// ones also record NRM_ERR_BOUNDS in *status.
__global__ void __launch_bounds__(32) bounds_selftest_kernel(int* results, int* status) {
  extern __shared__ __align__(128) unsigned char dyn[];
  NRM_DEBUG_ENTRY(status);
  if (threadIdx.x != 0) return;
  results[0] = dbg_smem_ok(dyn, 4, "self-test", __LINE__);
  results[1] = dbg_smem_ok(dyn + 252, 4, "self-test", __LINE__);
  results[2] = dbg_smem_ok(dyn + 253, 4, "self-test (expected report)", __LINE__);
  results[3] = dbg_smem_ok(dyn - 4, 4, "self-test (expected report)", __LINE__);
  results[4] = dbg_gmem_ok(results + 7, 4, results, 32, "self-test", __LINE__);
  results[5] = dbg_gmem_ok(results + 8, 4, results, 32, "self-test (expected report)", __LINE__);
  results[6] = dbg_index_ok(5, 5, "self-test (expected report)", __LINE__);
}
}  // namespace
#endif

// results: 8 device ints (results[7] is left alone); status: one device int.
cudaError_t launch_bounds_selftest(int* results, int* status, cudaStream_t stream) {
#ifdef NRM_DEBUG_CHECKS
  void* args[2] = {&results, &status};
  return cudaLaunchKernel((const void*)bounds_selftest_kernel, dim3(1), dim3(32), args, 256, stream);
#else
  (void)results;
  (void)status;
  (void)stream;
  return cudaErrorNotSupported;
#endif
}

cudaError_t launch_wait_expiry(unsigned long long timeout_ns, int* status2, cudaStream_t stream) {
  void* args[2] = {&timeout_ns, &status2};
  return cudaLaunchKernel((const void*)wait_expiry_kernel, dim3(1), dim3(64), args, 0, stream);
}

}  // namespace nrm
