// Forward kernel templates, instantiated by nrm_forward.cu (normal map and
// mask) and nrm_forward_points.cu (the same plus the organised point cloud,
// POINTS = true; kept apart because that pass needs more registers).
//
// The kernels: fused single-pass normal estimation (arXiv 2209.08241,
// Section 3.1 Eq. 4-6 and the Section 3.2 discontinuity mask) for sm_103a.
//
// Both kernels stage a halo tile of depth, (TX + 2 pad) x (TY + 2 alpha), into
// shared memory with one 2-D TMA load (cp.async.bulk.tensor, mbarrier
// completion; the tensor map's out-of-bounds zero fill doubles as "invalid
// depth" at the image border), decode it once into a float tile (invalid
// depth -> NaN), then every compute thread evaluates its pixels from shared
// memory and streams float4/half4 normals and packed mask bytes out.
//
//  fwd_plain_kernel       one CTA per tile of one frame (the per-frame launch);
//  fwd_persistent_kernel  a persistent grid walks the (frame, tile) work list of
//                         a whole batch. One producer warp walks the list,
//                         stages each tile's frame data in shared memory and
//                         issues the TMA loads into an S-stage ring (full/empty
//                         mbarriers); the NT compute threads decode and compute,
//                         synchronising only among themselves (named barrier 1).
#pragma once

#include "nrm_forward_vec.cuh"

// The compiled tile configurations (tile_x, tile_y, compute threads); the
// first is the default. TX is at most 128 so that the halo box (TX + 2 pad <=
// 256 elements) fits one TMA box.
#define NRM_FWD_CONFIGS(X) \
  X(128, 16, 256) X(128, 8, 256) X(128, 32, 256) X(128, 8, 128) X(128, 16, 128) \
  X(128, 32, 512) X(128, 64, 512) X(64, 16, 128) X(64, 32, 256) X(64, 64, 256)

namespace nrm {

using namespace dev;

// Per-stage tile record written by the producer, read by the compute threads.
struct alignas(16) StageInfo {
  TileFrame f;
  int tx, ty, tma, frame;
};
static_assert(sizeof(StageInfo) <= kStageInfoBytes, "StageInfo must fit its slot");

template <int TX, int TY, int NT, int OUT, bool POINTS>
__global__ void __launch_bounds__(NT)
    fwd_plain_kernel(const __grid_constant__ FrameDesc fd, const Globals g) {
  static_assert(TX / 2 + TY <= NT, "one thread per table entry");
  extern __shared__ __align__(128) unsigned char smem[];
  NRM_DEBUG_ENTRY(g.status);
  const int alpha = g.alpha;
  const bool u16 = fd.in_dtype == NRM_IN_U16_MM;
  const int eb = u16 ? 2 : 4;
  const int padx = pad_x(alpha, eb);  // staging (TMA) box
  const int bw = TX + 2 * padx;
  const int pad4 = pad_x(alpha, 4);   // decoded float tile
  const int fw = TX + 2 * pad4;
  const int bh = TY + 2 * alpha;
  const int gx0 = blockIdx.x * TX;
  const int gy0 = blockIdx.y * TY;
  const unsigned SB = stage_bytes_for(TX, TY, alpha);
  float* F = reinterpret_cast<float*>(smem + SB);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + SB + ftile_bytes_for(TX, TY, alpha));
  const TileFrame tf = tile_frame(fd, g.sign);
  // The column and row tables do not depend on the depth; the barrier at the
  // end of the staging publishes them with the decoded tile.
  fill_tile_tables<TX, TY>(reinterpret_cast<float4*>(smem + SB + ftile_float_bytes(TX, TY, alpha)), tf, gx0, gy0,
                           threadIdx.x);
  if (!stage_plain_tile<NT>(smem, F, bar, fd, tf, alpha, padx, bw, bh, pad4, fw, gx0, gy0, g)) return;
  compute_tile_fwd<TX, TY, NT, OUT, POINTS>(F, fw, pad4, tf, gx0, gy0, g);
}

// A work-list index: through the read-only data path from global memory, or a
// plain load from kernel-parameter space (GLOBAL = false).
template <bool GLOBAL>
__device__ __forceinline__ int load_index(const int* p) {
  if (GLOBAL) return __ldg(p);
  return *p;
}

// The persistent pipeline: block = NT compute threads + one producer warp.
// compute(F, fw, pad4, tf, gx0, gy0) evaluates one decoded tile. FENCE: the
// frame records (and their tensor maps) are in global memory written by the
// host, so each map is fenced before its first use; false for records in
// kernel-parameter space.
template <int TX, int TY, int NT, class Compute, bool FENCE = true>
__device__ __forceinline__ void persistent_pipeline(const BatchArgs& args, const Globals& g, const Compute& compute) {
  static_assert(TX / 2 + TY <= NT, "one thread per table entry");
  extern __shared__ __align__(128) unsigned char smem[];
  const int S = args.stages;
  const unsigned SB = args.stage_bytes;
  const int alpha = g.alpha;
  const unsigned FB = ftile_bytes_for(TX, TY, alpha);
  unsigned char* fbase = smem + (size_t)S * SB;  // two decoded tiles of FB bytes
  uint64_t* full = reinterpret_cast<uint64_t*>(fbase + 2 * FB);
  uint64_t* empty = full + S;
  StageInfo* info = reinterpret_cast<StageInfo*>(fbase + 2 * FB + 128);
  const int total = args.hdr->total_tiles;
  const int nf = args.hdr->n_frames;
  const int G = (int)gridDim.x;
  const int my = (int)blockIdx.x < total ? (total - 1 - (int)blockIdx.x) / G + 1 : 0;
  if (my == 0) return;

  NRM_DEBUG_ENTRY(g.status);
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    fence_barrier_init();
  }
  __syncthreads();

  if (threadIdx.x >= NT) {
    // ------------------------------------------------------------ producer
    if (threadIdx.x != NT) return;
    int cur = 0;      // frame cursor: this CTA's tiles increase monotonically
    int fenced = -1;  // last tensor map fenced
    for (int j = 0; j < my; ++j) {
      const int s = j % S;
      if (j >= S &&
          !mbar_wait_bounded(smem_u32(&empty[s]), (uint32_t)(((j / S) - 1) & 1), g.timeout_ns)) {
        record_error(g.status, NRM_ERR_TIMEOUT);
        // Let every copy this warp issued land before the CTA can exit.
        for (int k = j - S; k < j; ++k)
          mbar_wait_bounded(smem_u32(&full[k % S]), (uint32_t)((k / S) & 1), g.timeout_ns);
        return;
      }
      const int t = (int)blockIdx.x + j * G;
      while (cur + 1 < nf && load_index<FENCE>(args.tile_begin + cur + 1) <= t) ++cur;
      const FrameDesc* fd = args.frames + cur;
      const int local = t - load_index<FENCE>(args.tile_begin + cur);
      const int tiles_x = fd->tiles_x;
      const int ty = local / tiles_x;
      const int tx = local - ty * tiles_x;
      StageInfo& si = info[s];
#ifdef NRM_DEBUG_CHECKS
      if (!dbg_smem_ok(&si, (int)sizeof(StageInfo), "stage record", __LINE__)) return;
#endif
      si.f = tile_frame(*fd, g.sign);
      si.tx = tx;
      si.ty = ty;
      si.tma = fd->use_tma;
      si.frame = cur;
      const uint32_t bar = smem_u32(&full[s]);
      if (si.tma) {
        if (FENCE && cur != fenced) {
          fence_tensormap_acquire(&fd->tmap);
          fenced = cur;
        }
        const int eb = si.f.in_dtype == NRM_IN_U16_MM ? 2 : 4;
        const int padx = pad_x(alpha, eb);
        mbar_arrive_expect_tx(bar, (uint32_t)((TX + 2 * padx) * (TY + 2 * alpha) * eb));
        tma_load_2d(smem_u32(smem + (size_t)s * SB), &fd->tmap, tx * TX - padx, ty * TY - alpha, bar);
      } else {
        mbar_arrive(bar);  // plain-load tile: the compute threads read global memory themselves
      }
    }
    return;
  }

  // -------------------------------------------------------------- compute
  for (int i = 0; i < my; ++i) {
    const int s = i % S;
    const bool ok = mbar_wait_warp(smem_u32(&full[s]), (uint32_t)((i / S) & 1), g.timeout_ns);
    const StageInfo si = NRM_LDS(StageInfo, info + s);
    const bool u16 = si.f.in_dtype == NRM_IN_U16_MM;
    const int padx = pad_x(alpha, u16 ? 2 : 4);  // staging (TMA) box
    const int bw = TX + 2 * padx;
    const int pad4 = pad_x(alpha, 4);             // decoded float tile
    const int fw = TX + 2 * pad4;
    const int bh = TY + 2 * alpha;
    const int gx0 = si.tx * TX;
    const int gy0 = si.ty * TY;
    // Decoded tiles alternate between two buffers: the named barrier below
    // (one per tile) also guarantees that tile i - 2's buffer is no longer read.
    float* F = reinterpret_cast<float*>(fbase + (i & 1) * FB);
    if (ok) {
      if (si.tma) {
        decode_staged<TX, TY, NT>(smem + (size_t)s * SB, F, u16, alpha, fw, bh, bw, padx - pad4);
      } else {
        if (u16)
          load_tile_decoded<uint16_t, NT>(F, fw, bh, si.f, gx0 - pad4, gy0 - alpha);
        else
          load_tile_decoded<float, NT>(F, fw, bh, si.f, gx0 - pad4, gy0 - alpha);
      }
      fill_tile_tables<TX, TY>(reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(F) +
                                                         ftile_float_bytes(TX, TY, alpha)),
                               si.f, gx0, gy0, threadIdx.x);
    }
    if (bar_red_or(1, NT, !ok)) {
      if (threadIdx.x == 0) record_error(g.status, NRM_ERR_TIMEOUT);
      return;
    }
    // Stage s and its record have been consumed by every compute thread.
    if (threadIdx.x == 0) mbar_arrive(smem_u32(&empty[s]));
    compute(F, fw, pad4, si.f, gx0, gy0);
  }
}

// The whole descriptor block of a batch as one kernel parameter (capture-safe
// launches: nothing to upload, tensor maps in parameter space).
struct alignas(128) ParamBatch {
  BatchHeader hdr;
  int tile_begin[kParamMaxFrames + 1];
  FrameDesc frames[kParamMaxFrames];
};

template <int TX, int TY, int NT, int OUT>
__global__ void __launch_bounds__(NT + 32)
    fwd_persistent_param_kernel(const __grid_constant__ ParamBatch pb, const BatchArgs ring, const Globals g) {
  BatchArgs args = ring;
  args.hdr = &pb.hdr;
  args.tile_begin = pb.tile_begin;
  args.frames = pb.frames;
  auto compute = [&](const float* F, int fw, int pad4, const TileFrame& tf, int gx0, int gy0) {
    compute_tile_fwd<TX, TY, NT, OUT, false>(F, fw, pad4, tf, gx0, gy0, g);
  };
  persistent_pipeline<TX, TY, NT, decltype(compute), false>(args, g, compute);
}

template <int TX, int TY, int NT, int OUT, bool POINTS>
__global__ void __launch_bounds__(NT + 32)
    fwd_persistent_kernel(const BatchArgs args, const Globals g) {
  persistent_pipeline<TX, TY, NT>(args, g,
                                  [&](const float* F, int fw, int pad4, const TileFrame& tf, int gx0, int gy0) {
                                    compute_tile_fwd<TX, TY, NT, OUT, POINTS>(F, fw, pad4, tf, gx0, gy0, g);
                                  });
}

}  // namespace nrm
