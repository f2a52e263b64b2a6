// Persistent forward kernels that take the batch's descriptor block as one
// kernel parameter (frame records with their tensor maps in parameter space):
// a launch needs no device descriptor memory, upload or synchronisation, so it
// can be recorded by CUDA stream capture. For every compiled tile
// configuration; normal map and mask only.
#include <cstring>

#include "nrm_forward_kernels.cuh"

namespace nrm {

static_assert(sizeof(ParamBatch) <= 32764, "the descriptor block must fit the kernel parameter limit");

const void* fwd_param_kernel(int tile_x, int tile_y, int threads, int out_dtype) {
  if (out_dtype < 0 || out_dtype > 2) return nullptr;
#define NRM_FWD_PARAM(TX, TY, NT)                                                    \
  if (tile_x == TX && tile_y == TY && threads == NT) {                               \
    static const void* const k[3] = {(const void*)fwd_persistent_param_kernel<TX, TY, NT, NRM_OUT_F32X4>, \
                                     (const void*)fwd_persistent_param_kernel<TX, TY, NT, NRM_OUT_F16X4>, \
                                     (const void*)fwd_persistent_param_kernel<TX, TY, NT, NRM_OUT_OCT16>}; \
    return k[out_dtype];                                                             \
  }
  NRM_FWD_CONFIGS(NRM_FWD_PARAM)
#undef NRM_FWD_PARAM
  return nullptr;
}

size_t param_batch_bytes() { return sizeof(ParamBatch); }

void pack_param_batch(void* dst, const BatchHeader& hdr, const int* tile_begin, const FrameDesc* frames, int n) {
  ParamBatch* pb = static_cast<ParamBatch*>(dst);
  std::memset(pb, 0, sizeof(ParamBatch));
  pb->hdr = hdr;
  std::memcpy(pb->tile_begin, tile_begin, sizeof(int) * (size_t)(n + 1));
  std::memcpy(pb->frames, frames, sizeof(FrameDesc) * (size_t)n);
}

}  // namespace nrm
