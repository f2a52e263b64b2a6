// Multi-scale variant (arXiv 2209.08241, Section 2: the authors' previous
// method averages its closed-form normal over pixel distances alpha_1..alpha_K;
// every neighbour depth is sampled at its own scale's distance). Two per-scale
// stencils:
//   PAIR  Eq. 1-3, one tangent pair (neighbours (col + a, row), (col, row + a)):
//           n_x = -(a/fy) d3 (d2 - d1),  n_y = -(a/fx) d2 (d3 - d1),
//           n . (u1, v1, 1) = a^2/(fx fy) d2 d3;
//   QUAD  Eq. 4-6, the four-direction form of Section 3.1 at distance a.
// The unnormalised per-scale vectors are averaged (the 1/K, the depth scale^2
// and the orientation sign are folded into per-scale constants), then the
// Section 3.2 statistic, mask and stores are those of the single-scale kernel
// (compute_tile_with). Both stencils give n_z = -u1 n_x - v1 n_y + n . ray, so
// only n_x, n_y and n . ray are accumulated.
//
// fwd_ms_kernel: one CTA per 128 x 16 tile of one frame, with a halo of the
// largest scale, staged by TMA (or plain loads) and decoded once; the
// per-pixel work is K stencil evaluations from shared memory.
// fwd_ms_persistent_kernel: the batched form, on the persistent pipeline of
// the single-scale batched kernel (producer warp, TMA stage ring); each
// frame's descriptor carries its base constants a, b, c (see
// launch_multiscale_batched), scaled per scale by alpha_i and alpha_i^2.
#include <algorithm>
#include <atomic>

#include "nrm_forward_kernels.cuh"

namespace nrm {

using namespace dev;

namespace {

constexpr int TX = kMsTileX, TY = kMsTileY, NT = kMsThreads;

template <int FORM>
struct MultiStencil {
  const MsConsts* ms;
  int bw;
  __device__ __forceinline__ void operator()(const float* pa, const float* pb, float2 d1, float2& nx, float2& ny,
                                             float2& P) const {
    const float2 M1 = f2(-1.0f, -1.0f);
    // -0 is the identity of addition for every operand, +0 included, so the
    // first scale's fused multiply-add returns its product exactly, signed zero
    // included (one four-direction scale then equals the single-scale kernel).
    float2 ax = f2(-0.f, -0.f), ay = f2(-0.f, -0.f), ap = f2(-0.f, -0.f);
#pragma unroll 1
    for (int i = 0; i < ms->K; ++i) {
      const int a = ms->alpha[i];
      const int dv = a * bw;
      const float2 A = f2(ms->A[i], ms->A[i]), B = f2(ms->B[i], ms->B[i]), C = f2(ms->C[i], ms->C[i]);
      const float2 d2 = f2(pa[a], pb[a]);
      const float2 d3 = f2(pa[dv], pb[dv]);
      if (FORM == NRM_MS_PAIR) {
        // Eq. 1-3: A = -sign a/(K fy) s^2, B = -sign a/(K fx) s^2, C = sign a^2/(K fx fy) s^2.
        const float2 D21 = __ffma2_rn(M1, d1, d2), D31 = __ffma2_rn(M1, d1, d3);
        ax = __ffma2_rn(__fmul2_rn(A, d3), D21, ax);
        ay = __ffma2_rn(__fmul2_rn(B, d2), D31, ay);
        ap = __ffma2_rn(__fmul2_rn(C, d2), d3, ap);
      } else {
        // Eq. 4-6: A = -sign a/(4 K fy) s^2, B = -sign a/(4 K fx) s^2, C = sign a^2/(4 K fx fy) s^2.
        const float2 d4 = f2(pa[-a], pb[-a]);
        const float2 d5 = f2(pa[-dv], pb[-dv]);
        const float2 S24 = __fadd2_rn(d2, d4), D24 = __ffma2_rn(M1, d4, d2);
        const float2 S35 = __fadd2_rn(d3, d5), D35 = __ffma2_rn(M1, d5, d3);
        ax = __ffma2_rn(__fmul2_rn(A, S35), D24, ax);
        ay = __ffma2_rn(__fmul2_rn(B, S24), D35, ay);
        ap = __ffma2_rn(__fmul2_rn(C, S24), S35, ap);
      }
    }
    nx = ax;
    ny = ay;
    P = ap;
  }
};

template <int OUT, int FORM>
__global__ void __launch_bounds__(NT)
    fwd_ms_kernel(const __grid_constant__ FrameDesc fd, const __grid_constant__ MsConsts ms, const Globals g) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int alpha = ms.alpha_max;
  const int eb = fd.in_dtype == NRM_IN_U16_MM ? 2 : 4;
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
  if (!stage_plain_tile<NT>(smem, F, bar, fd, tf, alpha, padx, bw, bh, pad4, fw, gx0, gy0, g)) return;
  const MultiStencil<FORM> st{&ms, fw};
  const bool full = gx0 + TX <= tf.W;
  if (g.mask_mode == NRM_MASK_SECANT) {
    if (full)
      compute_tile_with<TX, TY, NT, OUT, true, true>(F, fw, pad4, tf, gx0, gy0, alpha, g.tau2, st);
    else
      compute_tile_with<TX, TY, NT, OUT, true, false>(F, fw, pad4, tf, gx0, gy0, alpha, g.tau2, st);
  } else {
    if (full)
      compute_tile_with<TX, TY, NT, OUT, false, true>(F, fw, pad4, tf, gx0, gy0, alpha, g.tau2, st);
    else
      compute_tile_with<TX, TY, NT, OUT, false, false>(F, fw, pad4, tf, gx0, gy0, alpha, g.tau2, st);
  }
}

// Per-frame form of MultiStencil: the constants of scale i are alpha_i a,
// alpha_i b, alpha_i^2 c from the frame's (sign-folded) bases.
template <int FORM>
struct FrameMultiStencil {
  const MsConsts* ms;
  float a, b, c;
  int bw;
  __device__ __forceinline__ void operator()(const float* pa, const float* pb, float2 d1, float2& nx, float2& ny,
                                             float2& P) const {
    const float2 M1 = f2(-1.0f, -1.0f);
    float2 ax = f2(-0.f, -0.f), ay = f2(-0.f, -0.f), ap = f2(-0.f, -0.f);
#pragma unroll 1
    for (int i = 0; i < ms->K; ++i) {
      const int al = ms->alpha[i];
      const int dv = al * bw;
      const float fa = (float)al;
      const float sa = fa * a, sb = fa * b, sc = fa * fa * c;
      const float2 A = f2(sa, sa), B = f2(sb, sb), C = f2(sc, sc);
      const float2 d2 = f2(pa[al], pb[al]);
      const float2 d3 = f2(pa[dv], pb[dv]);
      if (FORM == NRM_MS_PAIR) {
        const float2 D21 = __ffma2_rn(M1, d1, d2), D31 = __ffma2_rn(M1, d1, d3);
        ax = __ffma2_rn(__fmul2_rn(A, d3), D21, ax);
        ay = __ffma2_rn(__fmul2_rn(B, d2), D31, ay);
        ap = __ffma2_rn(__fmul2_rn(C, d2), d3, ap);
      } else {
        const float2 d4 = f2(pa[-al], pb[-al]);
        const float2 d5 = f2(pa[-dv], pb[-dv]);
        const float2 S24 = __fadd2_rn(d2, d4), D24 = __ffma2_rn(M1, d4, d2);
        const float2 S35 = __fadd2_rn(d3, d5), D35 = __ffma2_rn(M1, d5, d3);
        ax = __ffma2_rn(__fmul2_rn(A, S35), D24, ax);
        ay = __ffma2_rn(__fmul2_rn(B, S24), D35, ay);
        ap = __ffma2_rn(__fmul2_rn(C, S24), S35, ap);
      }
    }
    nx = ax;
    ny = ay;
    P = ap;
  }
};

// The multi-scale tile: the frame's stencil constants, then the shared epilogue.
template <int OUT, int FORM>
__device__ __forceinline__ void ms_tile(const MsConsts& ms, const Globals& g, const float* F, int fw, int pad4,
                                        const TileFrame& tf, int gx0, int gy0) {
  const FrameMultiStencil<FORM> st{&ms, tf.a, tf.b, tf.c, fw};
  const bool full = gx0 + TX <= tf.W;
  if (g.mask_mode == NRM_MASK_SECANT) {
    if (full)
      compute_tile_with<TX, TY, NT, OUT, true, true>(F, fw, pad4, tf, gx0, gy0, g.alpha, g.tau2, st);
    else
      compute_tile_with<TX, TY, NT, OUT, true, false>(F, fw, pad4, tf, gx0, gy0, g.alpha, g.tau2, st);
  } else {
    if (full)
      compute_tile_with<TX, TY, NT, OUT, false, true>(F, fw, pad4, tf, gx0, gy0, g.alpha, g.tau2, st);
    else
      compute_tile_with<TX, TY, NT, OUT, false, false>(F, fw, pad4, tf, gx0, gy0, g.alpha, g.tau2, st);
  }
}

// The batch's descriptor block as a kernel parameter (no upload, no fences).
template <int OUT, int FORM>
__global__ void __launch_bounds__(NT + 32)
    fwd_ms_persistent_param_kernel(const __grid_constant__ ParamBatch pb, const BatchArgs ring,
                                   const __grid_constant__ MsConsts ms, const Globals g) {
  BatchArgs args = ring;
  args.hdr = &pb.hdr;
  args.tile_begin = pb.tile_begin;
  args.frames = pb.frames;
  auto compute = [&](const float* F, int fw, int pad4, const TileFrame& tf, int gx0, int gy0) {
    ms_tile<OUT, FORM>(ms, g, F, fw, pad4, tf, gx0, gy0);
  };
  persistent_pipeline<TX, TY, NT, decltype(compute), false>(args, g, compute);
}

template <int OUT, int FORM>
__global__ void __launch_bounds__(NT + 32)
    fwd_ms_persistent_kernel(const BatchArgs args, const __grid_constant__ MsConsts ms, const Globals g) {
  persistent_pipeline<TX, TY, NT>(
      args, g, [&](const float* F, int fw, int pad4, const TileFrame& tf, int gx0, int gy0) {
        const FrameMultiStencil<FORM> st{&ms, tf.a, tf.b, tf.c, fw};
        const bool full = gx0 + TX <= tf.W;
        if (g.mask_mode == NRM_MASK_SECANT) {
          if (full)
            compute_tile_with<TX, TY, NT, OUT, true, true>(F, fw, pad4, tf, gx0, gy0, g.alpha, g.tau2, st);
          else
            compute_tile_with<TX, TY, NT, OUT, true, false>(F, fw, pad4, tf, gx0, gy0, g.alpha, g.tau2, st);
        } else {
          if (full)
            compute_tile_with<TX, TY, NT, OUT, false, true>(F, fw, pad4, tf, gx0, gy0, g.alpha, g.tau2, st);
          else
            compute_tile_with<TX, TY, NT, OUT, false, false>(F, fw, pad4, tf, gx0, gy0, g.alpha, g.tau2, st);
        }
      });
}

const void* ms_persistent_param_kernel(int out_dtype, int form) {
  static const void* k[3][2] = {
      {(const void*)fwd_ms_persistent_param_kernel<NRM_OUT_F32X4, NRM_MS_PAIR>,
       (const void*)fwd_ms_persistent_param_kernel<NRM_OUT_F32X4, NRM_MS_QUAD>},
      {(const void*)fwd_ms_persistent_param_kernel<NRM_OUT_F16X4, NRM_MS_PAIR>,
       (const void*)fwd_ms_persistent_param_kernel<NRM_OUT_F16X4, NRM_MS_QUAD>},
      {(const void*)fwd_ms_persistent_param_kernel<NRM_OUT_OCT16, NRM_MS_PAIR>,
       (const void*)fwd_ms_persistent_param_kernel<NRM_OUT_OCT16, NRM_MS_QUAD>}};
  return k[out_dtype][form];
}

const void* ms_persistent_kernel(int out_dtype, int form) {
  static const void* k[3][2] = {
      {(const void*)fwd_ms_persistent_kernel<NRM_OUT_F32X4, NRM_MS_PAIR>,
       (const void*)fwd_ms_persistent_kernel<NRM_OUT_F32X4, NRM_MS_QUAD>},
      {(const void*)fwd_ms_persistent_kernel<NRM_OUT_F16X4, NRM_MS_PAIR>,
       (const void*)fwd_ms_persistent_kernel<NRM_OUT_F16X4, NRM_MS_QUAD>},
      {(const void*)fwd_ms_persistent_kernel<NRM_OUT_OCT16, NRM_MS_PAIR>,
       (const void*)fwd_ms_persistent_kernel<NRM_OUT_OCT16, NRM_MS_QUAD>}};
  return k[out_dtype][form];
}

const void* ms_kernel(int out_dtype, int form) {
  static const void* k[3][2] = {
      {(const void*)fwd_ms_kernel<NRM_OUT_F32X4, NRM_MS_PAIR>, (const void*)fwd_ms_kernel<NRM_OUT_F32X4, NRM_MS_QUAD>},
      {(const void*)fwd_ms_kernel<NRM_OUT_F16X4, NRM_MS_PAIR>, (const void*)fwd_ms_kernel<NRM_OUT_F16X4, NRM_MS_QUAD>},
      {(const void*)fwd_ms_kernel<NRM_OUT_OCT16, NRM_MS_PAIR>, (const void*)fwd_ms_kernel<NRM_OUT_OCT16, NRM_MS_QUAD>}};
  return k[out_dtype][form];
}

}  // namespace

cudaError_t launch_multiscale(const FrameDesc& fd, const MsConsts& ms, const Globals& g, int out_dtype, int form,
                              cudaStream_t stream) {
  if (out_dtype < 0 || out_dtype > 2 || form < 0 || form > 1) return cudaErrorInvalidValue;
  const void* fn = ms_kernel(out_dtype, form);
  const unsigned smem = plain_smem_bytes(TX, TY, ms.alpha_max);
  // Grant, once per (kernel, device), the dynamic shared memory of the largest
  // scale any call may use (concurrent first calls set the same value).
  static std::atomic<bool> granted[3][2][64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 63;
  if (!granted[out_dtype][form][dev].load()) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)plain_smem_bytes(TX, TY, NRM_MAX_ALPHA));
    if (e != cudaSuccess) return e;
    granted[out_dtype][form][dev].store(true);
  }
  dim3 grid((fd.W + TX - 1) / TX, (fd.H + TY - 1) / TY);
  FrameDesc d = fd;
  MsConsts m = ms;
  Globals gg = g;
  void* args[3] = {&d, &m, &gg};
  cudaError_t e = cudaLaunchKernel(fn, grid, dim3(NT), args, smem, stream);
  return e;
}

cudaError_t launch_multiscale_batched(const BatchArgs& args, const MsConsts& ms, const Globals& g, int out_dtype,
                                      int form, int total_tiles, bool u16, cudaStream_t stream,
                                      const void* param_block) {
  if (out_dtype < 0 || out_dtype > 2 || form < 0 || form > 1) return cudaErrorInvalidValue;
  const bool param = param_block != nullptr;
  const void* fn = param ? ms_persistent_param_kernel(out_dtype, form) : ms_persistent_kernel(out_dtype, form);
  static std::atomic<bool> granted[2][3][2][64];
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 63;
  if (!granted[param][out_dtype][form][dev].load()) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)persistent_smem_bytes(TX, TY, NRM_MAX_ALPHA, kMsStages));
    if (e != cudaSuccess) return e;
    granted[param][out_dtype][form][dev].store(true);
  }
  const unsigned smem = persistent_smem_bytes(TX, TY, ms.alpha_max, kMsStages, u16 ? 2 : 0);
  int occ = 0;
  cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, persistent_threads(NT), smem);
  if (e != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  // Two CTAs of 256 compute threads per SM: 16 compute warps, the count at
  // which the single-scale batched kernel writes to HBM fastest.
  const int grid = std::min(total_tiles, std::min(occ, 2) * sms);
  BatchArgs a = args;
  a.stages = kMsStages;
  a.stage_bytes = stage_bytes_for(TX, TY, ms.alpha_max, u16 ? 2 : 0);
  MsConsts m = ms;
  Globals gg = g;
  gg.alpha = ms.alpha_max;
  if (param) {
    void* pargs[4] = {const_cast<void*>(param_block), &a, &m, &gg};
    return cudaLaunchKernel(fn, dim3(grid), dim3(persistent_threads(NT)), pargs, smem, stream);
  }
  void* kargs[3] = {&a, &m, &gg};
  return cudaLaunchKernel(fn, dim3(grid), dim3(persistent_threads(NT)), kargs, smem, stream);
}

}  // namespace nrm
