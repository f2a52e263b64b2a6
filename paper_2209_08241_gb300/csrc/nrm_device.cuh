// Device building blocks of the sm_103a normal-estimation kernels:
// inline-PTX wrappers for mbarrier and TMA (cp.async.bulk.tensor), bounded
// waits, the per-pixel closed form (Eq. 4-6 of arXiv 2209.08241) with the
// Section 3.2 mask, and the tile loop shared by the plain and persistent
// forward kernels.
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

#include "nrm_internal.h"

namespace nrm {
namespace dev {

// ------------------------------------------------------------------ PTX

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long global_timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// Makes barrier initialisation visible to the async (TMA) proxy.
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (TMA) accesses.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Acquire fence for a tensor map that the host wrote to global memory.
__device__ __forceinline__ void fence_tensormap_acquire(const void* tmap) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(tmap) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for phase `parity` of the barrier to complete, for at most timeout_ns
// of global time and at most 2^30 polls. Returns false if the bound ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity,
                                                  unsigned long long timeout_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_timer_ns();
  for (uint32_t i = 0; i < (1u << 30); ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_timer_ns() - t0 > timeout_ns) return false;
  }
  return false;
}

// 2-D tiled TMA load of box (x, y) into shared memory; completion is signalled
// as transaction bytes on `bar`. x * element size must be a multiple of 16.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void* tmap, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(tmap), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void record_error(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// ------------------------------------------------------ per-pixel method

// Depth element decoding. f32: metres, valid iff positive and finite.
// u16: raw units (the frame constants carry depth_scale^2), valid iff != 0.
// Sums and differences of u16 are formed exactly in integers (|.| < 2^17).
struct StencilSums {
  float S24, D24, S35, D35;
  bool ok;
};

__device__ __forceinline__ bool depth_ok(float d) { return d > 0.0f && d <= 3.402823466e38f; }

__device__ __forceinline__ StencilSums stencil_sums(const float* p, int alpha, int bw) {
  const float d1 = p[0], d2 = p[alpha], d4 = p[-alpha];
  const float d3 = p[alpha * bw], d5 = p[-alpha * bw];
  StencilSums s;
  s.ok = depth_ok(d1) & depth_ok(d2) & depth_ok(d3) & depth_ok(d4) & depth_ok(d5);
  s.S24 = d2 + d4;
  s.D24 = d2 - d4;
  s.S35 = d3 + d5;
  s.D35 = d3 - d5;
  return s;
}

__device__ __forceinline__ StencilSums stencil_sums(const uint16_t* p, int alpha, int bw) {
  const int d1 = p[0], d2 = p[alpha], d4 = p[-alpha];
  const int d3 = p[alpha * bw], d5 = p[-alpha * bw];
  StencilSums s;
  s.ok = (d1 != 0) & (d2 != 0) & (d3 != 0) & (d4 != 0) & (d5 != 0);
  s.S24 = (float)(d2 + d4);
  s.D24 = (float)(d2 - d4);
  s.S35 = (float)(d3 + d5);
  s.D35 = (float)(d3 - d5);
  return s;
}

struct FrameConsts {
  float a, b, c, inv_fx, inv_fy, cx, cy;
};

// Eq. 4-6 (Section 3.1): the reformulated multi-direction normal
// n = 1/4 s24 x s35 in closed form; returns n and P = n . (u1, v1, 1).
__device__ __forceinline__ void closed_form_normal(const StencilSums& s, const FrameConsts& k,
                                                   float u1, float v1, float& nx, float& ny,
                                                   float& nz, float& P) {
  nx = -k.a * s.S35 * s.D24;
  ny = -k.b * s.S24 * s.D35;
  P = k.c * s.S24 * s.S35;
  nz = fmaf(-u1, nx, fmaf(-v1, ny, P));
}

// Section 3.2 mask, compared in squared form (no square root):
//   RAW:    ||n|| <= tau                  <=>  q <= tau^2
//   SECANT: ||n|| ||ray|| / P <= tau      <=>  q ray2 <= tau^2 P^2   (P > 0)
__device__ __forceinline__ bool keep_pixel(bool ok, float q, float P, float ray2, int mode,
                                           float tau2) {
  if (mode == NRM_MASK_RAW) return ok && q > 0.0f && q <= tau2;
  return ok && P > 0.0f && q * ray2 <= tau2 * (P * P);
}

// Expands the low `n` bits of b into n bytes of value 0/1 (n = 2 or 4).
__device__ __forceinline__ uint32_t bits_to_bytes4(uint32_t b) {
  return (b * 0x00204081u) & 0x01010101u;
}

// --------------------------------------------------------- tile compute

// The frame fields the tile loop needs, read once per tile into registers.
// The orientation sign is folded into the Eq. 4-6 constants: the normal is
// linear in (a, b, c), so scaling them by -1 negates n and leaves q = n . n
// and P^2 unchanged.
struct TileFrame {
  float a, b, c, inv_fx, inv_fy, cx, cy;
  int H, W;
  long long out_pitch;
  void* normals;
  uint8_t* valid;
  int mask_align;
};

__device__ __forceinline__ TileFrame tile_frame(const FrameDesc& fd, float sign) {
  TileFrame f;
  f.a = -sign * fd.a;  // n_x = -a S35 D24  ->  (A S35) D24 with A = -sign a
  f.b = -sign * fd.b;
  f.c = sign * fd.c;
  f.inv_fx = fd.inv_fx;
  f.inv_fy = fd.inv_fy;
  f.cx = fd.cx;
  f.cy = fd.cy;
  f.H = fd.H;
  f.W = fd.W;
  f.out_pitch = fd.out_pitch;
  f.normals = fd.normals;
  f.valid = fd.valid;
  f.mask_align = fd.mask_align;
  return f;
}

// Decodes one staged depth element to float; an invalid depth becomes NaN so
// that every quantity computed from it is NaN and fails the mask comparison.
// float32: valid iff 0 < d <= FLT_MAX, i.e. bits - 1 < 0x7F7FFFFF (unsigned).
__device__ __forceinline__ float decode_depth(float d) {
  return (__float_as_uint(d) - 1u) < 0x7F7FFFFFu ? d : __int_as_float(0x7fc00000);
}
// uint16: exact conversion (2^23 + u is representable; subtracting 2^23 is
// exact); raw 0 is invalid. The depth scale is folded into a, b, c.
__device__ __forceinline__ float decode_depth_u16(uint32_t u) {
  const float f = __uint_as_float(0x4B000000u | u) - 8388608.0f;
  return u != 0u ? f : __int_as_float(0x7fc00000);
}

// Staged tile (TMA box, native dtype) -> decoded float tile, n elements
// (a multiple of 4; both buffers 16-byte aligned).
template <int NT>
__device__ __forceinline__ void decode_tile(const float* __restrict__ src, float* __restrict__ dst, int n) {
  for (int i = threadIdx.x * 4; i < n; i += NT * 4) {
    float4 v = *reinterpret_cast<const float4*>(src + i);
    v.x = decode_depth(v.x);
    v.y = decode_depth(v.y);
    v.z = decode_depth(v.z);
    v.w = decode_depth(v.w);
    *reinterpret_cast<float4*>(dst + i) = v;
  }
}

template <int NT>
__device__ __forceinline__ void decode_tile(const uint16_t* __restrict__ src, float* __restrict__ dst, int n) {
  for (int i = threadIdx.x * 4; i < n; i += NT * 4) {
    const uint2 r = *reinterpret_cast<const uint2*>(src + i);
    float4 v;
    v.x = decode_depth_u16(r.x & 0xFFFFu);
    v.y = decode_depth_u16(r.x >> 16);
    v.z = decode_depth_u16(r.y & 0xFFFFu);
    v.w = decode_depth_u16(r.y >> 16);
    *reinterpret_cast<float4*>(dst + i) = v;
  }
}

// Plain-load path (frames whose base or pitch rules out TMA): reads the halo
// box straight from global memory into the decoded float tile; outside the
// image counts as invalid, exactly like the TMA zero fill.
template <typename InT>
__device__ __forceinline__ void load_tile_decoded(float* dst, int bw, int bh, const FrameDesc& fd, int x0,
                                                  int y0) {
  const InT* src = reinterpret_cast<const InT*>(fd.depth);
  const int n = bw * bh;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int ly = i / bw, lx = i - ly * bw;
    const int x = x0 + lx, y = y0 + ly;
    float v = __int_as_float(0x7fc00000);
    if (x >= 0 && y >= 0 && x < fd.W && y < fd.H) {
      const InT raw = __ldg(src + (long long)y * fd.depth_pitch + x);
      if constexpr (sizeof(InT) == 2)
        v = decode_depth_u16(raw);
      else
        v = decode_depth(raw);
    }
    dst[i] = v;
  }
}

// Computes one TX x TY output tile from the decoded float halo tile F
// (origin global (gx0 - padx, gy0 - alpha), row pitch bw).
// Warp w handles rows w, w + NW, ...; lane l handles columns 32 k + l, so each
// store instruction of a warp covers 32 consecutive pixels (512 B of float4).
// Per-column terms (u1, 1 + u1^2) are computed once per tile. Mask bytes are
// gathered with one ballot per 32 pixels and written as TX/32 consecutive bytes
// per lane.
template <int TX, int TY, int NT, bool HALF, bool SECANT>
__device__ __forceinline__ void compute_tile(const float* __restrict__ F, int bw, int padx,
                                             const TileFrame& f, int gx0, int gy0, int alpha,
                                             float tau2) {
  constexpr int NW = NT / 32;
  constexpr int CH = TX / 32;
  static_assert(TY % NW == 0, "rows must divide among warps");
  static_assert(CH == 2 || CH == 4, "TX must be 64 or 128");
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;

  float u1[CH], ku[CH];
  bool colok[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) {
    const int gx = gx0 + 32 * c + lane;
    u1[c] = ((float)gx - f.cx) * f.inv_fx;
    ku[c] = fmaf(u1[c], u1[c], 1.0f);
    colok[c] = gx < f.W;
  }
  const int dv = alpha * bw;

#pragma unroll 1
  for (int ly = warp; ly < TY; ly += NW) {
    const int gy = gy0 + ly;
    if (gy >= f.H) break;
    const float v1 = ((float)gy - f.cy) * f.inv_fy;
    const float kv = v1 * v1;
    const float* row = F + (ly + alpha) * bw + padx + lane;
    const long long out_row = (long long)gy * f.out_pitch + gx0 + lane;
    uint32_t ballots[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const float* p = row + 32 * c;
      const float d1 = p[0];
      const float d2 = p[alpha], d4 = p[-alpha];
      const float d3 = p[dv], d5 = p[-dv];
      // Eq. 4-6 (Section 3.1).
      const float S24 = d2 + d4, D24 = d2 - d4;
      const float S35 = d3 + d5, D35 = d3 - d5;
      const float nx = (f.a * S35) * D24;
      const float ny = (f.b * S24) * D35;
      const float P = (f.c * S24) * S35;  // n . (u1, v1, 1) (times the sign)
      const float nz = fmaf(-u1[c], nx, fmaf(-v1, ny, P));
      const float q = fmaf(nx, nx, fmaf(ny, ny, nz * nz));
      // Section 3.2 mask in squared form; NaN (invalid depth) fails every test.
      bool keep = colok[c] && (d1 == d1) && (q > 0.0f);
      if (SECANT)
        keep = keep && (q * (ku[c] + kv) <= tau2 * (P * P));
      else
        keep = keep && (q <= tau2);
      // Select, not multiply: n is NaN next to invalid depths.
      const float inv = rsqrtf(q);
      const float ox = keep ? nx * inv : 0.0f;
      const float oy = keep ? ny * inv : 0.0f;
      const float oz = keep ? nz * inv : 0.0f;
      ballots[c] = __ballot_sync(0xffffffffu, keep);
      if (colok[c]) {
        if (HALF) {
          __half2 xy = __floats2half2_rn(ox, oy);
          __half2 zw = __floats2half2_rn(oz, 0.0f);
          uint2 v;
          v.x = *reinterpret_cast<uint32_t*>(&xy);
          v.y = *reinterpret_cast<uint32_t*>(&zw);
          __stcs(reinterpret_cast<uint2*>(f.normals) + out_row + 32 * c, v);
        } else {
          __stcs(reinterpret_cast<float4*>(f.normals) + out_row + 32 * c, make_float4(ox, oy, oz, 0.0f));
        }
      }
    }
    // Mask: lane l owns tile columns [CH l, CH l + CH).
    const int first = CH * lane;
    const int cidx = first >> 5;
    uint32_t word = 0;
#pragma unroll
    for (int c = 0; c < CH; ++c) word = (c == cidx) ? ballots[c] : word;
    const uint32_t bits = (word >> (first & 31)) & ((1u << CH) - 1u);
    const int gx = gx0 + first;
    uint8_t* mrow = f.valid + (long long)gy * f.out_pitch;
    if (gx + CH <= f.W && f.mask_align >= CH) {
      if (CH == 2) {
        const uint32_t v = bits_to_bytes4(bits);
        __stcs(reinterpret_cast<unsigned short*>(mrow + gx), (unsigned short)v);
      } else {
        __stcs(reinterpret_cast<unsigned int*>(mrow + gx), bits_to_bytes4(bits));
      }
    } else {
#pragma unroll
      for (int j = 0; j < CH; ++j) {
        if (gx + j < f.W) mrow[gx + j] = (uint8_t)((bits >> j) & 1u);
      }
    }
  }
}

// Both mask modes of compute_tile, chosen once per tile.
template <int TX, int TY, int NT, bool HALF>
__device__ __forceinline__ void compute_tile_any(const float* __restrict__ F, int bw, int padx,
                                                 const TileFrame& f, int gx0, int gy0, const Globals& g) {
  if (g.mask_mode == NRM_MASK_SECANT)
    compute_tile<TX, TY, NT, HALF, true>(F, bw, padx, f, gx0, gy0, g.alpha, g.tau2);
  else
    compute_tile<TX, TY, NT, HALF, false>(F, bw, padx, f, gx0, gy0, g.alpha, g.tau2);
}

// Loads the halo tile with plain loads (frames whose base or pitch rules out
// TMA), zero-filling outside the image exactly as the TMA out-of-bounds fill.
template <typename InT>
__device__ __forceinline__ void load_tile_plain(InT* sm, int bw, int bh, const FrameDesc& fd,
                                                int x0, int y0) {
  const InT* src = reinterpret_cast<const InT*>(fd.depth);
  const int n = bw * bh;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int ly = i / bw, lx = i - ly * bw;
    const int x = x0 + lx, y = y0 + ly;
    InT v = InT(0);
    if (x >= 0 && y >= 0 && x < fd.W && y < fd.H) v = __ldg(src + (long long)y * fd.depth_pitch + x);
    sm[i] = v;
  }
}

// Geometry of a frame's halo box for the forward kernels.
__device__ __forceinline__ int elem_bytes(int in_dtype) { return in_dtype == NRM_IN_U16_MM ? 2 : 4; }

}  // namespace dev
}  // namespace nrm
