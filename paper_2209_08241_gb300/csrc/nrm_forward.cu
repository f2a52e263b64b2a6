// Forward kernels without the point cloud: the registry of compiled tile
// configurations (kernel templates in nrm_forward_kernels.cuh).
#include "nrm_forward_kernels.cuh"

namespace nrm {

#define NRM_FWD_SET(TX, TY, NT)                                                            \
  {TX, TY, NT,                                                                             \
   {(const void*)fwd_plain_kernel<TX, TY, NT, NRM_OUT_F32X4, false>,                       \
    (const void*)fwd_plain_kernel<TX, TY, NT, NRM_OUT_F16X4, false>,                       \
    (const void*)fwd_plain_kernel<TX, TY, NT, NRM_OUT_OCT16, false>},                      \
   {(const void*)fwd_persistent_kernel<TX, TY, NT, NRM_OUT_F32X4, false>,                  \
    (const void*)fwd_persistent_kernel<TX, TY, NT, NRM_OUT_F16X4, false>,                  \
    (const void*)fwd_persistent_kernel<TX, TY, NT, NRM_OUT_OCT16, false>}},

static const FwdKernelSet kFwdSets[] = {NRM_FWD_CONFIGS(NRM_FWD_SET)};

int fwd_kernel_count() { return (int)(sizeof(kFwdSets) / sizeof(kFwdSets[0])); }

const FwdKernelSet* fwd_kernel(int i) {
  return (i >= 0 && i < fwd_kernel_count()) ? &kFwdSets[i] : nullptr;
}

const FwdKernelSet* fwd_kernel_find(int tile_x, int tile_y, int threads) {
  for (int i = 0; i < fwd_kernel_count(); ++i) {
    const FwdKernelSet& k = kFwdSets[i];
    if (k.tile_x == tile_x && k.tile_y == tile_y && k.threads == threads) return &k;
  }
  return nullptr;
}

}  // namespace nrm
