// Forward kernels that also write the organised point cloud (POINTS = true),
// for every compiled tile configuration (kernel templates in
// nrm_forward_kernels.cuh).
#include "nrm_forward_kernels.cuh"

namespace nrm {

const void* fwd_points_kernel(int tile_x, int tile_y, int threads, int out_dtype, bool persistent) {
  if (out_dtype < 0 || out_dtype > 2) return nullptr;
#define NRM_FWD_POINTS(TX, TY, NT)                                                                  \
  if (tile_x == TX && tile_y == TY && threads == NT) {                                              \
    static const void* const plain[3] = {(const void*)fwd_plain_kernel<TX, TY, NT, NRM_OUT_F32X4, true>,  \
                                         (const void*)fwd_plain_kernel<TX, TY, NT, NRM_OUT_F16X4, true>,  \
                                         (const void*)fwd_plain_kernel<TX, TY, NT, NRM_OUT_OCT16, true>}; \
    static const void* const pers[3] = {(const void*)fwd_persistent_kernel<TX, TY, NT, NRM_OUT_F32X4, true>, \
                                        (const void*)fwd_persistent_kernel<TX, TY, NT, NRM_OUT_F16X4, true>, \
                                        (const void*)fwd_persistent_kernel<TX, TY, NT, NRM_OUT_OCT16, true>}; \
    return persistent ? pers[out_dtype] : plain[out_dtype];                                        \
  }
  NRM_FWD_CONFIGS(NRM_FWD_POINTS)
#undef NRM_FWD_POINTS
  return nullptr;
}

}  // namespace nrm
