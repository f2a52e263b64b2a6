// Internal declarations shared by the library's translation units (kernels and
// host C ABI). Not part of the public interface (include/nrm.h).
#pragma once

#include <cuda.h>  // CUtensorMap (type only; the driver entry point is looked up at run time)
#include <cuda_runtime.h>
#include <stdint.h>

#include "nrm.h"

#if defined(__CUDACC__)
#define NRM_HD __host__ __device__
#else
#define NRM_HD
#endif

namespace nrm {

// Pixels along x of the halo pad: the TMA box must start on a 16-byte
// boundary, so the left pad alpha is rounded up to 16 bytes of elements.
NRM_HD inline int pad_x(int alpha, int elem_bytes) {
  int q = 16 / elem_bytes;
  return (alpha + q - 1) / q * q;
}

// One frame of a launch. 256 bytes; the tensor map must be 128-byte aligned.
struct alignas(128) FrameDesc {
  CUtensorMap tmap;        // 2-D map of the depth image, box (TX + 2 pad) x (TY + 2 alpha)
  const void* depth;
  void* normals;           // forward: normal map; adjoint: upstream gradient (float4)
  uint8_t* valid;
  float* grad_depth;       // adjoint only: depth gradient (pitch depth_pitch)
  long long depth_pitch;   // elements
  long long out_pitch;     // pixels (normals and mask)
  int H, W;
  int tiles_x;
  int tile_begin;          // first work-list index of this frame
  // Eq. 4-6 constants with the depth unit folded in (u16: times depth_scale^2):
  float a;                 // alpha / (4 fy)
  float b;                 // alpha / (4 fx)
  float c;                 // alpha^2 / (4 fx fy)
  float inv_fx, inv_fy, cx, cy;
  int in_dtype;            // NRM_IN_F32_M or NRM_IN_U16_MM
  int use_tma;             // 1: TMA tile loads; 0: plain loads (unaligned base or pitch)
  int mask_align;          // bytes: largest power of two (<= 16) dividing mask base and pitch
  float point_scale;       // metres per decoded depth unit (u16: depth_scale; f32: 1)
  int out_align;           // bytes: largest power of two (<= 16) dividing normals base and row pitch in bytes
  float* points;           // optional organised point cloud (x, y, z, 0) per pixel, pitch out_pitch; or NULL
};
static_assert(sizeof(FrameDesc) == 256, "FrameDesc layout");

// Header of a batch's device descriptor block, followed by tile_begin[n+1]
// (at kTileBeginOffset) and then the FrameDesc array (at frames_offset()).
struct BatchHeader {
  int n_frames;
  int total_tiles;
  int pad_[14];
};
static_assert(sizeof(BatchHeader) == 64, "BatchHeader layout");
constexpr size_t kTileBeginOffset = 64;
constexpr size_t frames_offset(int capacity) {
  size_t b = kTileBeginOffset + sizeof(int) * (size_t)(capacity + 1);
  return (b + 255) / 256 * 256;
}
constexpr size_t block_bytes(int capacity) { return frames_offset(capacity) + sizeof(FrameDesc) * (size_t)capacity; }

// Launch-wide parameters (by value).
struct Globals {
  int alpha;
  int mask_mode;
  float tau2;              // tau^2 (may be +inf)
  float sign;              // +1 paper orientation, -1 towards the camera
  int* status;             // device status word (first error wins)
  unsigned long long timeout_ns;  // bound of every device-side wait
};

// Frames per capture-safe batched launch, whose descriptor block travels as
// one kernel parameter (under the 32,764-byte parameter limit).
constexpr int kParamMaxFrames = 100;

struct BatchArgs {
  const BatchHeader* hdr;
  const int* tile_begin;
  const FrameDesc* frames;
  int stages;
  unsigned stage_bytes;    // bytes per pipeline stage (multiple of 128)
};

// A compiled forward tile configuration.
struct FwdKernelSet {
  int tile_x, tile_y, threads;
  const void* plain[3];       // [out_dtype] fwd_plain_kernel<...>
  const void* persistent[3];  // [out_dtype] fwd_persistent_kernel<...>
};

// All compiled forward configurations (nrm_forward.cu).
int fwd_kernel_count();
const FwdKernelSet* fwd_kernel(int i);
const FwdKernelSet* fwd_kernel_find(int tile_x, int tile_y, int threads);
// The same configuration's kernel that also writes the point cloud
// (nrm_forward_points.cu), or NULL.
const void* fwd_points_kernel(int tile_x, int tile_y, int threads, int out_dtype, bool persistent);
// The same configuration's persistent kernel taking the descriptor block as a
// kernel parameter (nrm_forward_param.cu; capture-safe launches), its size in
// bytes, and a host routine that packs a batch into that parameter block.
const void* fwd_param_kernel(int tile_x, int tile_y, int threads, int out_dtype);
size_t param_batch_bytes();
void pack_param_batch(void* dst, const BatchHeader& hdr, const int* tile_begin, const FrameDesc* frames, int n);

// Stage buffer bytes for a tile config and alpha: for input elements of eb
// bytes (2: uint16, 4: float32), or the maximum over both (eb = 0).
NRM_HD inline unsigned stage_bytes_for(int tile_x, int tile_y, int alpha, int eb = 0) {
  unsigned f32 = (unsigned)((tile_x + 2 * pad_x(alpha, 4)) * (tile_y + 2 * alpha) * 4);
  unsigned u16 = (unsigned)((tile_x + 2 * pad_x(alpha, 2)) * (tile_y + 2 * alpha) * 2);
  unsigned m = eb == 2 ? u16 : (eb == 4 ? f32 : (f32 > u16 ? f32 : u16));
  return (m + 127) / 128 * 128;
}
// Bytes of the decoded float halo tile: (TX + 2 pad_x(alpha, 4)) x (TY + 2 alpha)
// floats for either input dtype.
NRM_HD inline unsigned ftile_float_bytes(int tile_x, int tile_y, int alpha) {
  unsigned b = (unsigned)((tile_x + 2 * pad_x(alpha, 4)) * (tile_y + 2 * alpha) * 4);
  return (b + 127) / 128 * 128;
}
// Bytes of a decoded tile's buffer: the float tile, then its column and row
// tables (one float4 per column pair and per row).
NRM_HD inline unsigned ftile_bytes_for(int tile_x, int tile_y, int alpha) {
  unsigned t = (unsigned)((tile_x / 2 + tile_y) * 16);
  return ftile_float_bytes(tile_x, tile_y, alpha) + (t + 127) / 128 * 128;
}
// Dynamic shared memory of the plain kernel: staging buffer, decoded tile,
// barrier.
NRM_HD inline unsigned plain_smem_bytes(int tile_x, int tile_y, int alpha) {
  return stage_bytes_for(tile_x, tile_y, alpha) + ftile_bytes_for(tile_x, tile_y, alpha) + 128;
}
// Bytes reserved per pipeline stage for the producer's tile record.
constexpr unsigned kStageInfoBytes = 128;
// Dynamic shared memory of the persistent kernel: `stages` staging buffers
// (sized as stage_bytes_for with eb), two decoded tiles, full/empty barriers
// (128 B) and per-stage tile records.
NRM_HD inline unsigned persistent_smem_bytes(int tile_x, int tile_y, int alpha, int stages, int eb = 0) {
  return stage_bytes_for(tile_x, tile_y, alpha, eb) * stages + 2 * ftile_bytes_for(tile_x, tile_y, alpha) +
         128 + kStageInfoBytes * stages;
}
// Threads of a persistent CTA: the compute threads plus one producer warp.
NRM_HD inline int persistent_threads(int compute_threads) { return compute_threads + 32; }

// Host helpers of the C ABI (nrm_api.cpp) shared with the other entry points:
// validation (sets the thread-local error message) and descriptor filling for
// the forward kernels with tile (tile_x, tile_y).
int host_fail(int code, const char* message);
void host_clear_error();  // clears the thread's last-error message, as every entry point does first
int host_validate_params(const nrm_params& p);
int host_validate_frame(const nrm_frame& f, int index, int out_dtype);
void host_make_forward_desc(FrameDesc* d, const nrm_frame& f, const nrm_params& p, int tile_x, int tile_y);

// Backward (adjoint) kernel for float32 depth: output tile and threads.
constexpr int kBwdTileX = 64;
constexpr int kBwdTileY = 32;
constexpr int kBwdThreads = 256;
// Columns of the mask box to the left of the tile: the TMA box must start on a
// 16-byte boundary, so the mask halo (alpha <= 16 columns) is read from 16.
constexpr int kBwdMaskPad = 16;
constexpr int kBwdMaskBoxW = kBwdTileX + 2 * kBwdMaskPad;

// The adjoint's two further tensor maps per frame: the upstream gradient as a
// 2-D tensor of 8-byte elements (2 W, H), box (2 (TX + 2 alpha), TY + 2 alpha),
// and the mask as a 2-D uint8 tensor, box (kBwdMaskBoxW, TY + 2 alpha).
struct alignas(128) BwdMaps {
  CUtensorMap grad;
  CUtensorMap mask;
};
static_assert(sizeof(BwdMaps) == 256, "BwdMaps layout");
// Descriptor block of a batched adjoint: header, tile offsets, FrameDescs, then BwdMaps.
constexpr size_t bwd_maps_offset(int capacity) { return frames_offset(capacity) + sizeof(FrameDesc) * (size_t)capacity; }
constexpr size_t bwd_block_bytes(int capacity) { return bwd_maps_offset(capacity) + sizeof(BwdMaps) * (size_t)capacity; }

struct BwdBatchArgs {
  const BatchHeader* hdr;
  const int* tile_begin;
  const FrameDesc* frames;
  const BwdMaps* maps;
};

unsigned bwd_smem_bytes(int alpha);
// fd.tmap maps the depth with box (kBwdTileX + 2 pad_x(2 alpha, 4)) x (kBwdTileY + 4 alpha);
// fd.normals holds the upstream gradient, fd.valid the mask, fd.grad_depth the output.
// fd.use_tma = 1 only if all three maps (fd.tmap, maps.grad, maps.mask) are valid.
// scale (optional, device array indexed by frame): the upstream gradient is
// scale[frame] times the float4 buffer (then a target normal map).
cudaError_t launch_backward(const FrameDesc& fd, const BwdMaps& maps, const Globals& g, cudaStream_t stream,
                            const float* scale = nullptr);
// All tiles of a batch in one launch (grid max_tiles x n_frames); the descriptor
// block is in device memory.
cudaError_t launch_backward_batched(const BwdBatchArgs& args, int n_frames, int max_tiles, const Globals& g,
                                    cudaStream_t stream, const float* scale = nullptr);
// One frame's mask for the cosine-loss factor (nrm_cosine_loss_scale).
struct LossCountFrame {
  const uint8_t* valid;
  int H, W;
  long long pitch;
};
constexpr int kLossCountMaxFrames = 128;  // frames per launch (the records travel as the kernel parameter)
// scale[i] = -1 / max(N_valid(i), 1) for frames[0..n) (host array); counts and
// tickets: n zeroed device words each, returned to zero by the kernel.
cudaError_t launch_loss_scale(const LossCountFrame* frames, int n, unsigned* counts, unsigned* tickets, float* scale,
                              cudaStream_t stream);

// The same for at most kBwdParamMaxFrames frames with the records and maps
// (host arrays) passed as one kernel parameter: no upload, no fences.
constexpr int kBwdParamMaxFrames = 60;
cudaError_t launch_backward_batched_param(const FrameDesc* frames, const BwdMaps* maps, int n_frames, int max_tiles,
                                          const Globals& g, cudaStream_t stream, const float* scale = nullptr);

// Evaluation kernels (nrm_eval.cu).
constexpr int kMseBlocks = 2048;  // fixed, so that the reduction order never changes
cudaError_t launch_spherical(const float* normals, const uint8_t* valid, int H, int W, long long pitch, float* phi,
                             float* theta, cudaStream_t stream);
// partials: 3 kMseBlocks doubles of device scratch; out: 3 doubles.
cudaError_t launch_angle_mse(const float* na, const uint8_t* va, const float* nb, const uint8_t* vb, int H, int W,
                             long long pitch, double* partials, double* out, cudaStream_t stream);

// Multi-scale variant (nrm_multiscale.cu): one CTA per kMsTileX x kMsTileY
// tile, halo of the largest scale. Per scale i the constants of its stencil
// (NRM_MS_PAIR: Eq. 1-3; NRM_MS_QUAD: Eq. 4-6), with 1/K, the depth scale^2 and
// the orientation sign folded in: n_x += A_i (...), n_y += B_i (...),
// n . ray += C_i (...).
constexpr int kMsTileX = 128;
constexpr int kMsTileY = 16;
constexpr int kMsThreads = 256;
struct MsConsts {
  int K;
  int alpha_max;
  int alpha[NRM_MAX_SCALES];
  float A[NRM_MAX_SCALES], B[NRM_MAX_SCALES], C[NRM_MAX_SCALES];
};
// fd.tmap must map the depth with box (kMsTileX + 2 pad_x(alpha_max, eb)) x
// (kMsTileY + 2 alpha_max) (or fd.use_tma = 0).
cudaError_t launch_multiscale(const FrameDesc& fd, const MsConsts& ms, const Globals& g, int out_dtype, int form,
                              cudaStream_t stream);
// The batched form: one persistent launch over the batch's work list in a
// device descriptor block (args; stages and stage bytes are set here). Each
// frame's a, b, c hold its bases s^2 / (q fy K), s^2 / (q fx K),
// s^2 / (q fx fy K) (s the depth scale, q = 1 for NRM_MS_PAIR and 4 for
// NRM_MS_QUAD); ms.A, ms.B, ms.C are not used. u16: every frame is uint16.
constexpr int kMsStages = 3;
// param_block: a ParamBatch packed by pack_param_batch (batches of at most
// kParamMaxFrames frames; args' pointers are then unused), or NULL for the
// device descriptor block in args.
cudaError_t launch_multiscale_batched(const BatchArgs& args, const MsConsts& ms, const Globals& g, int out_dtype,
                                      int form, int total_tiles, bool u16, cudaStream_t stream,
                                      const void* param_block = nullptr);

// Bounded-wait self-test (nrm_selftest.cu): status2 = two device ints (zeroed
// by the caller), one per wait flavour.
cudaError_t launch_wait_expiry(unsigned long long timeout_ns, int* status2, cudaStream_t stream);
// Range-check self-test (nrm_selftest.cu): cudaErrorNotSupported unless this is
// the checking build (NRM_DEBUG_CHECKS).
cudaError_t launch_bounds_selftest(int* results, int* status, cudaStream_t stream);

// Plane-fitting ground truth (nrm_planefit.cu): FP32 normals (w = 0) and the
// validity mask of the (2 radius + 1)^2 window fit; fd.depth, fd.normals,
// fd.valid, pitches, H, W, cx, cy, inv_fx, inv_fy and in_dtype are used;
// radius 1..4 (compiled per radius).
cudaError_t launch_plane_fit(const FrameDesc& fd, int radius, float sign, cudaStream_t stream);

}  // namespace nrm
