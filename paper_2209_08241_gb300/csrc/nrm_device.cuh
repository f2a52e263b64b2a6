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

// Computes one TX x TY output tile from a shared-memory halo tile.
//   sm:    tile origin = global (gx0 - padx, gy0 - alpha), row pitch bw elements
//   Normals: float4 (HALF = false) or 4 x half (HALF = true) per pixel.
// Warp w handles rows w, w + NW, ...; lane l handles columns 32 k + l, so each
// store instruction of a warp covers 32 consecutive pixels (512 B of float4).
// Mask bytes are gathered with one ballot per 32 pixels and written as
// TX/32 consecutive bytes per lane.
template <int TX, int TY, int NT, bool HALF, typename InT>
__device__ __forceinline__ void compute_tile(const InT* __restrict__ sm, int bw, int padx,
                                             const FrameDesc& fd, int gx0, int gy0,
                                             const Globals& g) {
  constexpr int NW = NT / 32;
  constexpr int CH = TX / 32;
  static_assert(TY % NW == 0, "rows must divide among warps");
  static_assert(CH == 2 || CH == 4, "TX must be 64 or 128");
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int alpha = g.alpha;
  const int H = fd.H, W = fd.W;
  const FrameConsts k = {fd.a, fd.b, fd.c, fd.inv_fx, fd.inv_fy, fd.cx, fd.cy};
  const float sign = g.sign;

#pragma unroll 1
  for (int ly = warp; ly < TY; ly += NW) {
    const int gy = gy0 + ly;
    if (gy >= H) break;
    const float v1 = ((float)gy - k.cy) * k.inv_fy;
    const InT* row = sm + (ly + alpha) * bw + padx;
    uint32_t ballots[CH];
    const long long out_row = (long long)gy * fd.out_pitch;
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const int lx = 32 * c + lane;
      const int gx = gx0 + lx;
      const StencilSums s = stencil_sums(row + lx, alpha, bw);
      const float u1 = ((float)gx - k.cx) * k.inv_fx;
      float nx, ny, nz, P;
      closed_form_normal(s, k, u1, v1, nx, ny, nz, P);
      const float q = fmaf(nx, nx, fmaf(ny, ny, nz * nz));
      const float ray2 = fmaf(u1, u1, fmaf(v1, v1, 1.0f));
      const bool keep = keep_pixel(s.ok && gx < W, q, P, ray2, g.mask_mode, g.tau2);
      // Select, not multiply: n may be NaN or infinite next to invalid depths.
      const float inv = sign * rsqrtf(q);
      const float ox = keep ? nx * inv : 0.0f;
      const float oy = keep ? ny * inv : 0.0f;
      const float oz = keep ? nz * inv : 0.0f;
      ballots[c] = __ballot_sync(0xffffffffu, keep);
      if (gx < W) {
        if (HALF) {
          __half2 xy = __floats2half2_rn(ox, oy);
          __half2 zw = __floats2half2_rn(oz, 0.0f);
          uint2 v;
          v.x = *reinterpret_cast<uint32_t*>(&xy);
          v.y = *reinterpret_cast<uint32_t*>(&zw);
          __stcs(reinterpret_cast<uint2*>(fd.normals) + out_row + gx, v);
        } else {
          __stcs(reinterpret_cast<float4*>(fd.normals) + out_row + gx, make_float4(ox, oy, oz, 0.0f));
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
    uint8_t* mrow = fd.valid + out_row;
    if (gx + CH <= W && fd.mask_align >= CH) {
      if (CH == 2) {
        const uint32_t v = bits_to_bytes4(bits);
        __stcs(reinterpret_cast<unsigned short*>(mrow + gx), (unsigned short)v);
      } else {
        __stcs(reinterpret_cast<unsigned int*>(mrow + gx), bits_to_bytes4(bits));
      }
    } else {
#pragma unroll
      for (int j = 0; j < CH; ++j) {
        if (gx + j < W) mrow[gx + j] = (uint8_t)((bits >> j) & 1u);
      }
    }
  }
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
