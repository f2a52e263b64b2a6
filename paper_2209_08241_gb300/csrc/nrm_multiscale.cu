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
// (emit_pair, emit_mask_row). Both stencils give n_z = -u1 n_x - v1 n_y +
// n . ray, so only n_x, n_y and n . ray are accumulated.
//
// fwd_ms_kernel: one CTA per 128 x 16 tile of one frame, with a halo of the
// largest scale, staged by TMA (or plain loads) and decoded once; the
// per-pixel work is K stencil evaluations from shared memory.
// fwd_ms_persistent_kernel / fwd_ms_persistent_param_kernel: the batched
// form, on the persistent pipeline of the single-scale batched kernel
// (producer warp, TMA stage ring), with the descriptor block in global memory
// or as the kernel parameter; each frame's descriptor carries its base
// constants a, b, c (see launch_multiscale_batched), scaled per scale by
// alpha_i and alpha_i^2.
#include <algorithm>
#include <atomic>

#include "nrm_forward_kernels.cuh"

namespace nrm {

using namespace dev;

namespace {

constexpr int TX = kMsTileX, TY = kMsTileY, NT = kMsThreads;

constexpr int kMsCtasPerSm = 3;
constexpr int NW = NT / 32;
constexpr int NP = TX / 64;  // pixel pairs per lane and row
static_assert(TY % NW == 0 && TX % 64 == 0, "tile shape");

// One tile. Warp w handles rows w, w + NW, ... and lane l the pixel pairs
// (64 p + l, 64 p + 32 + l), as in the single-scale tile; per row the lane
// keeps the running sums of n_x, n_y and P of its NP pairs and walks the
// scales once, so each scale's constants and shared-memory offsets are formed
// once per row rather than once per pixel pair. Consts(i, A, B, C) gives scale
// i's constants (sign, 1/K and depth scale folded in). -0 is the identity of
// addition for every operand, +0 included, so the first scale's fused
// multiply-add returns its product exactly, signed zero included (one
// four-direction scale then equals the single-scale kernel). The epilogue
// (statistic, mask, stores) is the single-scale one.
template <int OUT, int FORM, bool SECANT, bool FULL, class Consts>
__device__ __forceinline__ void ms_compute(const float* __restrict__ F, int fw, int pad4, const TileFrame& f,
                                           int gx0, int gy0, int halo, float tau2, int n_scales,
                                           const int* alphas, const Consts& consts) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const float2 M1 = f2(-1.0f, -1.0f);
  float2 nu1[NP], ku[NP];
  bool colok[2 * NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const int gxa = gx0 + 64 * p + lane, gxb = gxa + 32;
    const float ua = ((float)gxa - f.cx) * f.inv_fx;
    const float ub = ((float)gxb - f.cx) * f.inv_fx;
    nu1[p] = f2(-ua, -ub);
    ku[p] = f2(fmaf(ua, ua, 1.0f), fmaf(ub, ub, 1.0f));
    colok[2 * p] = FULL || gxa < f.W;
    colok[2 * p + 1] = FULL || gxb < f.W;
  }
  const float2 T = f2(tau2, tau2);

#pragma unroll 1
  for (int ly = warp; ly < TY; ly += NW) {
    const int gy = gy0 + ly;
    if (gy >= f.H) break;
    const float* row = F + (ly + halo) * fw + pad4 + lane;
    float2 d1[NP], ax[NP], ay[NP], ap[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      d1[p] = f2(NRM_LDS(float, row + 64 * p), NRM_LDS(float, row + 64 * p + 32));
      ax[p] = ay[p] = ap[p] = f2(-0.f, -0.f);
    }
#pragma unroll 1
    for (int i = 0; i < n_scales; ++i) {
      const int al = alphas[i];
      const int dv = al * fw;
      float sa, sb, sc;
      consts(i, sa, sb, sc);
      const float2 A = f2(sa, sa), B = f2(sb, sb), C = f2(sc, sc);
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        const float* pa = row + 64 * p;
        const float* pb = pa + 32;
        const float2 d2 = f2(NRM_LDS(float, pa + al), NRM_LDS(float, pb + al));
        const float2 d3 = f2(NRM_LDS(float, pa + dv), NRM_LDS(float, pb + dv));
        if (FORM == NRM_MS_PAIR) {
          // Eq. 1-3: A = -sign a/(K fy) s^2, B = -sign a/(K fx) s^2, C = sign a^2/(K fx fy) s^2.
          const float2 D21 = __ffma2_rn(M1, d1[p], d2), D31 = __ffma2_rn(M1, d1[p], d3);
          ax[p] = __ffma2_rn(__fmul2_rn(A, d3), D21, ax[p]);
          ay[p] = __ffma2_rn(__fmul2_rn(B, d2), D31, ay[p]);
          ap[p] = __ffma2_rn(__fmul2_rn(C, d2), d3, ap[p]);
        } else {
          // Eq. 4-6: A = -sign a/(4 K fy) s^2, B = -sign a/(4 K fx) s^2, C = sign a^2/(4 K fx fy) s^2.
          const float2 d4 = f2(NRM_LDS(float, pa - al), NRM_LDS(float, pb - al));
          const float2 d5 = f2(NRM_LDS(float, pa - dv), NRM_LDS(float, pb - dv));
          const float2 S24 = __fadd2_rn(d2, d4), D24 = __ffma2_rn(M1, d4, d2);
          const float2 S35 = __fadd2_rn(d3, d5), D35 = __ffma2_rn(M1, d5, d3);
          ax[p] = __ffma2_rn(__fmul2_rn(A, S35), D24, ax[p]);
          ay[p] = __ffma2_rn(__fmul2_rn(B, S24), D35, ay[p]);
          ap[p] = __ffma2_rn(__fmul2_rn(C, S24), S35, ap[p]);
        }
      }
    }
    const float v1 = ((float)gy - f.cy) * f.inv_fy;
    const float2 nv1 = f2(-v1, -v1);
    const float2 kv = f2(v1 * v1, v1 * v1);
    const long long out_row = (long long)gy * f.out_pitch + gx0 + lane;
    uint32_t ballots[2 * NP];
#pragma unroll
    for (int p = 0; p < NP; ++p)
      emit_pair<OUT, SECANT, FULL>(f, out_row, p, d1[p], ax[p], ay[p], ap[p], nu1[p], ku[p], nv1, kv, T, tau2,
                                   colok[2 * p], colok[2 * p + 1], ballots[2 * p], ballots[2 * p + 1]);
    emit_mask_row<2 * NP, FULL>(f, gx0, gy, lane, ballots);
  }
}

template <int OUT, int FORM, class Consts>
__device__ __forceinline__ void ms_tile_any(const MsConsts& ms, const Globals& g, const float* F, int fw, int pad4,
                                            const TileFrame& tf, int gx0, int gy0, int halo, const Consts& c) {
  const bool full = gx0 + TX <= tf.W;
  if (g.mask_mode == NRM_MASK_SECANT) {
    if (full)
      ms_compute<OUT, FORM, true, true>(F, fw, pad4, tf, gx0, gy0, halo, g.tau2, ms.K, ms.alpha, c);
    else
      ms_compute<OUT, FORM, true, false>(F, fw, pad4, tf, gx0, gy0, halo, g.tau2, ms.K, ms.alpha, c);
  } else {
    if (full)
      ms_compute<OUT, FORM, false, true>(F, fw, pad4, tf, gx0, gy0, halo, g.tau2, ms.K, ms.alpha, c);
    else
      ms_compute<OUT, FORM, false, false>(F, fw, pad4, tf, gx0, gy0, halo, g.tau2, ms.K, ms.alpha, c);
  }
}

// Single-frame constants: precomputed per scale on the host.
struct HostScaleConsts {
  const MsConsts* ms;
  __device__ __forceinline__ void operator()(int i, float& A, float& B, float& C) const {
    A = ms->A[i];
    B = ms->B[i];
    C = ms->C[i];
  }
};

// Per-frame constants of a batch: alpha_i a, alpha_i b, alpha_i^2 c from the
// frame's (sign-folded) bases.
struct FrameScaleConsts {
  const MsConsts* ms;
  float a, b, c;
  __device__ __forceinline__ void operator()(int i, float& A, float& B, float& C) const {
    const float fa = (float)ms->alpha[i];
    A = fa * a;
    B = fa * b;
    C = fa * fa * c;
  }
};

template <int OUT, int FORM>
__global__ void __launch_bounds__(NT)
    fwd_ms_kernel(const __grid_constant__ FrameDesc fd, const __grid_constant__ MsConsts ms, const Globals g) {
  extern __shared__ __align__(128) unsigned char smem[];
  NRM_DEBUG_ENTRY(g.status);
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
  ms_tile_any<OUT, FORM>(ms, g, F, fw, pad4, tf, gx0, gy0, alpha, HostScaleConsts{&ms});
}

// The multi-scale tile of a batch frame.
template <int OUT, int FORM>
__device__ __forceinline__ void ms_tile(const MsConsts& ms, const Globals& g, const float* F, int fw, int pad4,
                                        const TileFrame& tf, int gx0, int gy0) {
  ms_tile_any<OUT, FORM>(ms, g, F, fw, pad4, tf, gx0, gy0, g.alpha, FrameScaleConsts{&ms, tf.a, tf.b, tf.c});
}

// The batch's descriptor block as a kernel parameter (no upload, no fences).
template <int OUT, int FORM>
__global__ void __launch_bounds__(NT + 32, kMsCtasPerSm)
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
__global__ void __launch_bounds__(NT + 32, kMsCtasPerSm)
    fwd_ms_persistent_kernel(const BatchArgs args, const __grid_constant__ MsConsts ms, const Globals g) {
  persistent_pipeline<TX, TY, NT>(args, g,
                                  [&](const float* F, int fw, int pad4, const TileFrame& tf, int gx0, int gy0) {
                                    ms_tile<OUT, FORM>(ms, g, F, fw, pad4, tf, gx0, gy0);
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
  // Three CTAs of 256 compute threads per SM (24 compute warps): the K
  // stencils per pixel make this kernel issue-bound rather than HBM-bound, and
  // the extra warps hide the shared-memory and arithmetic latencies.
  const int grid = std::min(total_tiles, std::min(occ, kMsCtasPerSm) * sms);
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
