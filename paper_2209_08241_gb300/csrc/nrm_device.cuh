// Device building blocks of the sm_103a normal-estimation kernels:
// inline-PTX wrappers for mbarrier, named barriers and TMA
// (cp.async.bulk.tensor), bounded waits, depth decoding, the per-pixel closed
// form (Eq. 4-6 of arXiv 2209.08241) with the Section 3.2 mask, and the tile
// loop shared by the plain and persistent forward kernels.
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

#include <cstdio>

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

// Tests phase `parity` for completion. A thread whose phase is not complete
// is suspended by the hardware until the phase completes or about
// kSuspendHintNs elapse, so a waiting warp does not spin on issue slots.
constexpr uint32_t kSuspendHintNs = 1000000;
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(kSuspendHintNs)
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

// The same wait for a whole (converged) warp: lane 0 polls, with a short sleep
// between polls, and broadcasts the outcome; on success every lane then tests
// the completed phase once itself, which returns at once and gives each lane
// the acquire ordering of the barrier. A warp of waiting threads therefore
// costs one polling thread's instructions instead of 32.
__device__ __forceinline__ bool mbar_wait_warp(uint32_t bar, uint32_t parity, unsigned long long timeout_ns) {
  const int lane = threadIdx.x & 31;
  uint32_t ok = 0;
  if (lane == 0) {
    ok = mbar_try_wait(bar, parity);
    if (!ok) {
      const unsigned long long t0 = global_timer_ns();
      for (uint32_t i = 0; i < (1u << 30); ++i) {
        __nanosleep(64);
        if (mbar_try_wait(bar, parity)) {
          ok = 1;
          break;
        }
        if (global_timer_ns() - t0 > timeout_ns) break;
      }
    }
  }
  ok = __shfl_sync(0xffffffffu, ok, 0);
  if (ok) ok = mbar_try_wait(bar, parity);
  return ok != 0;
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

// Named barrier over `count` threads (a multiple of 32) that also ORs a
// predicate across them.
__device__ __forceinline__ bool bar_red_or(uint32_t id, uint32_t count, bool pred) {
  uint32_t out;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(out)
      : "r"((uint32_t)pred), "r"(id), "r"(count)
      : "memory");
  return out != 0;
}

// Hardware reciprocal square root, flush-to-zero (inputs here are >= FLT_MIN).
__device__ __forceinline__ float rsqrt_ftz(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ void record_error(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// ------------------------------------------------------- checking build
//
// Built with NRM_DEBUG_CHECKS (build.py --debug), every shared-memory access of
// the kernels and every global access that depends on frame geometry goes
// through the macros below: an index outside its buffer skips the access,
// prints the site and records NRM_ERR_BOUNDS in the launch's status word (its
// address is kept per block by NRM_DEBUG_ENTRY). Nothing traps. In ordinary
// builds the macros are the plain accesses.

// Bytes spanned by an H x W buffer of esz-byte elements with row pitch `pitch`
// (the extent the checks allow for an output or input buffer).
__host__ __device__ __forceinline__ long long dbg_span(int H, int W, long long pitch, int esz) {
  return H > 0 && W > 0 ? ((long long)(H - 1) * pitch + W) * esz : 0;
}

#ifdef NRM_DEBUG_CHECKS
__device__ __forceinline__ int*& dbg_status_slot() {
  __shared__ int* slot;
  return slot;
}
static __device__ __noinline__ void dbg_fail(const char* what, int line, long long off, long long len) {
  printf("NRM_BOUNDS %s (line %d): byte offset %lld outside [0, %lld), block %d, thread %d\n", what, line, off,
         len, (int)blockIdx.x, (int)threadIdx.x);
  record_error(dbg_status_slot(), NRM_ERR_BOUNDS);
}
// p lies, with `bytes` bytes, inside the block's dynamic shared memory.
__device__ __forceinline__ bool dbg_smem_ok(const void* p, int bytes, const char* what, int line) {
  extern __shared__ __align__(128) unsigned char dbg_dyn_smem[];  // the alignment of every kernel's own declaration, so both name the same address
  uint32_t size;
  asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(size));
  const long long off = (long long)smem_u32(p) - (long long)smem_u32(dbg_dyn_smem);
  if (off < 0 || off + bytes > (long long)size) {
    dbg_fail(what, line, off, size);
    return false;
  }
  return true;
}
// p lies, with `bytes` bytes, inside [lo, lo + len).
__device__ __forceinline__ bool dbg_gmem_ok(const void* p, int bytes, const void* lo, long long len, const char* what,
                                            int line) {
  const long long off = (const char*)p - (const char*)lo;
  if (off < 0 || off + bytes > len) {
    dbg_fail(what, line, off, len);
    return false;
  }
  return true;
}
// Index i of a fixed-size (static shared or local) array of n elements.
__device__ __forceinline__ bool dbg_index_ok(long long i, long long n, const char* what, int line) {
  if (i < 0 || i >= n) {
    dbg_fail(what, line, i, n);
    return false;
  }
  return true;
}
// At kernel entry: the status word the checks report to (all threads).
#define NRM_DEBUG_ENTRY(status)                            \
  do {                                                     \
    if (threadIdx.x == 0) nrm::dev::dbg_status_slot() = (status); \
    __syncthreads();                                       \
  } while (0)
#define NRM_LDS(T, p) (nrm::dev::dbg_smem_ok((p), (int)sizeof(T), "shared load", __LINE__) ? *(p) : T())
#define NRM_STS(p, v)                                                              \
  do {                                                                             \
    if (nrm::dev::dbg_smem_ok((p), (int)sizeof(*(p)), "shared store", __LINE__)) *(p) = (v); \
  } while (0)
#define NRM_GOK(p, lo, len) nrm::dev::dbg_gmem_ok((p), (int)sizeof(*(p)), (lo), (len), "global access", __LINE__)
#define NRM_IOK(i, n) nrm::dev::dbg_index_ok((i), (n), "array index", __LINE__)
#else
#define NRM_DEBUG_ENTRY(status) \
  do {                          \
  } while (0)
#define NRM_LDS(T, p) (*(p))
#define NRM_STS(p, v) (*(p) = (v))
#define NRM_GOK(p, lo, len) true
#define NRM_IOK(i, n) true
#endif

// -------------------------------------------------- per-pixel (adjoint path)

// Stencil sums and differences of Eq. 4-6 (adjoint kernel).
struct StencilSums {
  float S24, D24, S35, D35;
};

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

// Loads a halo box with plain loads, zero-filling outside the image.
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
    NRM_STS(sm + i, v);
  }
}

// ------------------------------------------------------------ forward tiles

// Everything the forward tile loop needs about a frame, in registers. The
// orientation sign is folded into the Eq. 4-6 constants: the normal is linear
// in (a, b, c), so scaling them by -1 negates n and leaves q = n . n and P^2
// unchanged.
struct TileFrame {
  float a, b, c;           // n_x = (a S35) D24, n_y = (b S24) D35, P = (c S24) S35
  float inv_fx, inv_fy, cx, cy;
  int H, W;
  int mask_align;
  int out_align;
  int in_dtype;
  long long out_pitch;
  void* normals;
  uint8_t* valid;
  const void* depth;
  long long depth_pitch;
  float* points;       // optional point cloud output, or NULL
  float point_scale;   // metres per decoded depth unit
};

__device__ __forceinline__ TileFrame tile_frame(const FrameDesc& fd, float sign) {
  TileFrame f;
  f.a = -sign * fd.a;
  f.b = -sign * fd.b;
  f.c = sign * fd.c;
  f.inv_fx = fd.inv_fx;
  f.inv_fy = fd.inv_fy;
  f.cx = fd.cx;
  f.cy = fd.cy;
  f.H = fd.H;
  f.W = fd.W;
  f.mask_align = fd.mask_align;
  f.out_align = fd.out_align;
  f.in_dtype = fd.in_dtype;
  f.out_pitch = fd.out_pitch;
  f.normals = fd.normals;
  f.valid = fd.valid;
  f.depth = fd.depth;
  f.depth_pitch = fd.depth_pitch;
  f.points = fd.points;
  f.point_scale = fd.point_scale;
  return f;
}

// Decodes one staged depth element to float; an invalid depth becomes NaN so
// that every quantity computed from it is NaN and fails the mask comparison.
// float32: valid iff 0 < d <= FLT_MAX, i.e. bits - 1 < 0x7F7FFFFF (unsigned).
__device__ __forceinline__ float decode_depth(float d) {
  return (__float_as_uint(d) - 1u) < 0x7F7FFFFFu ? d : __int_as_float(0x7fc00000);
}
// uint16 (u < 2^16): for u >= 1 the bits (u - 1) | 0x4B000000 encode the float
// 2^23 + u - 1 exactly, and subtracting 2^23 - 1 gives u exactly; for the
// invalid raw value 0 they are 0xFFFFFFFF, a NaN, which the subtraction
// keeps. The depth scale is folded into a, b, c.
__device__ __forceinline__ float decode_depth_u16(uint32_t u) {
  return __uint_as_float((u - 1u) | 0x4B000000u) - 8388607.0f;
}

// Staged tile (TMA box, native dtype) -> decoded float tile, by threads
// 0..NT-1. The float tile always has the float32 geometry: pitch
// fw = TX + 2 pad_x(alpha, 4) (a multiple of 4), origin gx0 - pad_x(alpha, 4);
// a uint16 box is wider (pad_x(alpha, 2) >= pad_x(alpha, 4)), so its columns
// are read from offset `skip` = pad_x(alpha, 2) - pad_x(alpha, 4) (a multiple
// of 4). Work is in groups of 4 consecutive elements of one row.
template <int NT>
__device__ __forceinline__ void decode_tile(const float* __restrict__ src, float* __restrict__ dst, int fw,
                                            int rows, int /*src_pitch*/, int /*skip*/) {
  const int n = fw * rows;  // same geometry: a flat copy
  for (int i = threadIdx.x * 4; i < n; i += NT * 4) {
    float4 v = NRM_LDS(float4, reinterpret_cast<const float4*>(src + i));
    v.x = decode_depth(v.x);
    v.y = decode_depth(v.y);
    v.z = decode_depth(v.z);
    v.w = decode_depth(v.w);
    NRM_STS(reinterpret_cast<float4*>(dst + i), v);
  }
}

template <int NT>
__device__ __forceinline__ void decode_tile(const uint16_t* __restrict__ src, float* __restrict__ dst, int fw,
                                            int rows, int src_pitch, int skip) {
  const int gpr = fw >> 2;  // 4-element groups per row
  const int n = gpr * rows;
  for (int gi = threadIdx.x; gi < n; gi += NT) {
    const int r = gi / gpr;
    const int c = (gi - r * gpr) << 2;
    const uint2 raw = NRM_LDS(uint2, reinterpret_cast<const uint2*>(src + r * src_pitch + skip + c));
    float4 v;
    v.x = decode_depth_u16(raw.x & 0xFFFFu);
    v.y = decode_depth_u16(raw.x >> 16);
    v.z = decode_depth_u16(raw.y & 0xFFFFu);
    v.w = decode_depth_u16(raw.y >> 16);
    NRM_STS(reinterpret_cast<float4*>(dst + r * fw + c), v);
  }
}

// Plain-load path (frames whose base or pitch rules out TMA): reads the halo
// box straight from global memory into the decoded float tile, by threads
// 0..NT-1; outside the image counts as invalid, exactly like the TMA zero fill.
template <typename InT, int NT>
__device__ __forceinline__ void load_tile_decoded(float* dst, int bw, int bh, const TileFrame& f, int x0,
                                                  int y0) {
  const InT* src = reinterpret_cast<const InT*>(f.depth);
  const int n = bw * bh;
  for (int i = threadIdx.x; i < n; i += NT) {
    const int ly = i / bw, lx = i - ly * bw;
    const int x = x0 + lx, y = y0 + ly;
    float v = __int_as_float(0x7fc00000);
    if (x >= 0 && y >= 0 && x < f.W && y < f.H) {
      const InT raw = __ldg(src + (long long)y * f.depth_pitch + x);
      if constexpr (sizeof(InT) == 2)
        v = decode_depth_u16(raw);
      else
        v = decode_depth(raw);
    }
    NRM_STS(dst + i, v);
  }
}

__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }

// Hardware reciprocal, flush-to-zero (the octahedral code's quantisation step,
// 1/32767, dwarfs its error).
__device__ __forceinline__ float rcp_ftz(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Octahedral code of the direction of a normal (Meyer et al. 2010; Cigolle et
// al. 2014): p = (n_x, n_y) / (|n_x| + |n_y| + |n_z|); where n_z < 0 the lower
// half is folded over the diagonals, p <- (1 - |p_y|, 1 - |p_x|) with the signs of
// p. Since 1 - |p_y| = (|n_x| + |n_z|) / l1, both cases are
// p = (n_x + sgn(n_x) m, n_y + sgn(n_y) m) / l1 with m = max(-n_z, 0). Each
// coordinate becomes the signed 16-bit integer round(32767 p) (|32767 p| <=
// 32767 up to rounding, far below 32767.5, so it fits): one fused multiply-add
// with 1.5 * 2^23 rounds to the nearest integer, which then sits in the low
// mantissa bits (two's complement modulo 2^16). x in the low half of the
// word, y in the high half. The code does not depend on the length of n.
__device__ __forceinline__ uint32_t oct16_code(float nx, float ny, float nz) {
  const float s = 32767.0f * rcp_ftz(fabsf(nx) + fabsf(ny) + fabsf(nz));
  const float m = fmaxf(-nz, 0.0f);
  const float tx = nx + copysignf(m, nx);
  const float ty = ny + copysignf(m, ny);
  const float kRound = 12582912.0f;  // 1.5 * 2^23
  return __byte_perm(__float_as_uint(fmaf(tx, s, kRound)), __float_as_uint(fmaf(ty, s, kRound)), 0x5410);
}

__device__ __forceinline__ void oct16_encode2(float2 nx, float2 ny, float2 nz, uint32_t& ca, uint32_t& cb) {
  ca = oct16_code(nx.x, ny.x, nz.x);
  cb = oct16_code(nx.y, ny.y, nz.y);
}

// Expands the low 2 or 4 bits of b into bytes of value 0/1.
__device__ __forceinline__ uint32_t bits_to_bytes4(uint32_t b) {
  return (b * 0x00204081u) & 0x01010101u;
}

// Stages the halo tile of a plain launch (one CTA per tile) and decodes it into
// the float tile F (fw x bh, invalid depth -> NaN): one TMA box of bw x bh
// elements at (gx0 - padx, gy0 - alpha) into smem (out-of-bounds zero fill =
// invalid), or plain loads when the frame has no tensor map. Returns false on
// every thread if the TMA wait expired, after thread 0 has recorded
// NRM_ERR_TIMEOUT and waited (bounded) for the copy to land.
template <int NT>
__device__ __forceinline__ bool stage_plain_tile(unsigned char* smem, float* F, uint64_t* bar, const FrameDesc& fd,
                                                 const TileFrame& tf, int alpha, int padx, int bw, int bh, int pad4,
                                                 int fw, int gx0, int gy0, const Globals& g) {
  const bool u16 = fd.in_dtype == NRM_IN_U16_MM;
  const int eb = u16 ? 2 : 4;
  bool ok = true;
  if (fd.use_tma) {
    const uint32_t b = smem_u32(bar);
    if (threadIdx.x == 0) {
      mbar_init(b, 1);
      fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      mbar_arrive_expect_tx(b, (uint32_t)(bw * bh * eb));
      tma_load_2d(smem_u32(smem), &fd.tmap, gx0 - padx, gy0 - alpha, b);
    }
    ok = mbar_wait_warp(b, 0, g.timeout_ns);
    if (ok) {
      if (u16)
        decode_tile<NT>(reinterpret_cast<const uint16_t*>(smem), F, fw, bh, bw, padx - pad4);
      else
        decode_tile<NT>(reinterpret_cast<const float*>(smem), F, fw, bh, bw, 0);
    }
  } else {
    if (u16)
      load_tile_decoded<uint16_t, NT>(F, fw, bh, tf, gx0 - pad4, gy0 - alpha);
    else
      load_tile_decoded<float, NT>(F, fw, bh, tf, gx0 - pad4, gy0 - alpha);
  }
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) {
      record_error(g.status, NRM_ERR_TIMEOUT);
      mbar_wait_bounded(smem_u32(bar), 0, g.timeout_ns);  // let the copy land before exiting
    }
    return false;
  }
  return true;
}

// The Eq. 4-6 stencil of one pixel pair at distance alpha (Section 3.1): the
// unnormalised n_x, n_y and P = n . (u1, v1, 1), all times the orientation
// sign folded into A, B, C. pa, pb point at the pair's centre depths in the
// decoded tile; dv = alpha rows.
struct QuadStencil {
  float2 A, B, C;
  int alpha, dv;
  __device__ __forceinline__ void operator()(const float* pa, const float* pb, float2 d1, float2& nx, float2& ny,
                                             float2& P) const {
    const float2 M1 = f2(-1.0f, -1.0f);
    const float2 d2 = f2(NRM_LDS(float, pa + alpha), NRM_LDS(float, pb + alpha));
    const float2 d4 = f2(NRM_LDS(float, pa - alpha), NRM_LDS(float, pb - alpha));
    const float2 d3 = f2(NRM_LDS(float, pa + dv), NRM_LDS(float, pb + dv));
    const float2 d5 = f2(NRM_LDS(float, pa - dv), NRM_LDS(float, pb - dv));
    (void)d1;
    // d2 - d4 as one fused (-1) d4 + d2: a single rounding, like a subtraction.
    const float2 S24 = __fadd2_rn(d2, d4), D24 = __ffma2_rn(M1, d4, d2);
    const float2 S35 = __fadd2_rn(d3, d5), D35 = __ffma2_rn(M1, d5, d3);
    nx = __fmul2_rn(__fmul2_rn(A, S35), D24);
    ny = __fmul2_rn(__fmul2_rn(B, S24), D35);
    P = __fmul2_rn(__fmul2_rn(C, S24), S35);  // n . (u1, v1, 1), times the sign
  }
};

// Section 3.2 for one pixel pair (tile columns 64 p + lane and 64 p + 32 + lane
// of the row whose first output element is out_row): from the unnormalised
// n_x, n_y and P = n . (u1, v1, 1), the statistic in squared form, the mask
// ballots and the normal (or octahedral code) stores. nu1 = -(u1 of both
// columns), ku = 1 + u1^2, nv1 = -v1, kv = v1^2, T = tau^2 in both lanes.
template <int OUT, bool SECANT, bool FULL>
__device__ __forceinline__ void emit_pair(const TileFrame& f, long long out_row, int p, float2 d1, float2 nx,
                                          float2 ny, float2 P, float2 nu1, float2 ku, float2 nv1, float2 kv,
                                          float2 T, float tau2, bool cola, bool colb, uint32_t& ballot_a,
                                          uint32_t& ballot_b) {
  const float kFltMin = 1.17549435e-38f;
  const float2 nz = __ffma2_rn(nu1, nx, __ffma2_rn(nv1, ny, P));
  const float2 q = __ffma2_rn(nx, nx, __ffma2_rn(ny, ny, __fmul2_rn(nz, nz)));
  // Section 3.2 mask in squared form; NaN (invalid depth) fails every test.
  // (Bitwise &: every operand is side-effect free, and no branches.)
  bool ka = cola & (d1.x == d1.x) & (q.x >= kFltMin);
  bool kb = colb & (d1.y == d1.y) & (q.y >= kFltMin);
  if (SECANT) {
    const float2 lhs = __fmul2_rn(q, __fadd2_rn(ku, kv));
    const float2 rhs = __fmul2_rn(T, __fmul2_rn(P, P));
    ka = ka & (lhs.x <= rhs.x);
    kb = kb & (lhs.y <= rhs.y);
  } else {
    ka = ka & (q.x <= tau2);
    kb = kb & (q.y <= tau2);
  }
  ballot_a = __ballot_sync(0xffffffffu, ka);
  ballot_b = __ballot_sync(0xffffffffu, kb);
  if (OUT == NRM_OUT_OCT16) {
    // Octahedral code of n (scale-invariant: n need not be normalised).
    uint32_t ca, cb;
    oct16_encode2(nx, ny, nz, ca, cb);
    ca = ka ? ca : 0u;
    cb = kb ? cb : 0u;
    uint32_t* dst = reinterpret_cast<uint32_t*>(f.normals) + out_row + 64 * p;
    [[maybe_unused]] const long long nlen = dbg_span(f.H, f.W, f.out_pitch, 4);
    if ((FULL || cola) && NRM_GOK(dst, f.normals, nlen)) __stcs(dst, ca);
    if ((FULL || colb) && NRM_GOK(dst + 32, f.normals, nlen)) __stcs(dst + 32, cb);
    return;
  }
  const float2 inv = f2(rsqrt_ftz(q.x), rsqrt_ftz(q.y));
  const float2 ox = __fmul2_rn(nx, inv), oy = __fmul2_rn(ny, inv), oz = __fmul2_rn(nz, inv);
  // Select, not multiply: n is NaN next to invalid depths.
  const float4 va = ka ? make_float4(ox.x, oy.x, oz.x, 0.0f) : make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 vb = kb ? make_float4(ox.y, oy.y, oz.y, 0.0f) : make_float4(0.f, 0.f, 0.f, 0.f);
  if (OUT == NRM_OUT_F16X4) {
    const __half2 xya = __floats2half2_rn(va.x, va.y), zwa = __floats2half2_rn(va.z, 0.0f);
    const __half2 xyb = __floats2half2_rn(vb.x, vb.y), zwb = __floats2half2_rn(vb.z, 0.0f);
    uint2* dst = reinterpret_cast<uint2*>(f.normals) + out_row + 64 * p;
    [[maybe_unused]] const long long nlen = dbg_span(f.H, f.W, f.out_pitch, 8);
    if ((FULL || cola) && NRM_GOK(dst, f.normals, nlen))
      __stcs(dst, make_uint2(*reinterpret_cast<const uint32_t*>(&xya), *reinterpret_cast<const uint32_t*>(&zwa)));
    if ((FULL || colb) && NRM_GOK(dst + 32, f.normals, nlen))
      __stcs(dst + 32, make_uint2(*reinterpret_cast<const uint32_t*>(&xyb), *reinterpret_cast<const uint32_t*>(&zwb)));
  } else {
    float4* dst = reinterpret_cast<float4*>(f.normals) + out_row + 64 * p;
    [[maybe_unused]] const long long nlen = dbg_span(f.H, f.W, f.out_pitch, 16);
    if ((FULL || cola) && NRM_GOK(dst, f.normals, nlen)) __stcs(dst, va);
    if ((FULL || colb) && NRM_GOK(dst + 32, f.normals, nlen)) __stcs(dst + 32, vb);
  }
}

// The mask bytes of one tile row from its CH ballots (ballot c covers tile
// columns 32 c .. 32 c + 31): lane l writes columns [CH l, CH l + CH).
template <int CH, bool FULL>
__device__ __forceinline__ void emit_mask_row(const TileFrame& f, int gx0, int gy, int lane,
                                              const uint32_t (&ballots)[CH]) {
  const int first = CH * lane;
  const int cidx = first >> 5;
  uint32_t word = 0;
#pragma unroll
  for (int c = 0; c < CH; ++c) word = (c == cidx) ? ballots[c] : word;
  const uint32_t bits = (word >> (first & 31)) & ((1u << CH) - 1u);
  const int gx = gx0 + first;
  uint8_t* mrow = f.valid + (long long)gy * f.out_pitch;
  if ((FULL || gx + CH <= f.W) && f.mask_align >= CH) {
    [[maybe_unused]] const long long mlen = dbg_span(f.H, f.W, f.out_pitch, 1);
    if (CH == 2) {
      unsigned short* mp = reinterpret_cast<unsigned short*>(mrow + gx);
      if (NRM_GOK(mp, f.valid, mlen)) __stcs(mp, (unsigned short)bits_to_bytes4(bits));
    } else {
      unsigned int* mp = reinterpret_cast<unsigned int*>(mrow + gx);
      if (NRM_GOK(mp, f.valid, mlen)) __stcs(mp, bits_to_bytes4(bits));
    }
  } else {
#pragma unroll
    for (int j = 0; j < CH; ++j) {
      if (gx + j < f.W && NRM_GOK(mrow + gx + j, f.valid, dbg_span(f.H, f.W, f.out_pitch, 1)))
        mrow[gx + j] = (uint8_t)((bits >> j) & 1u);
    }
  }
}

// Computes one TX x TY output tile from the decoded float halo tile F
// (origin global (gx0 - padx, gy0 - halo), row pitch bw), threads 0..NT-1,
// with the stencil st giving each pixel pair's unnormalised normal.
// Warp w handles rows w, w + NW, ...; lane l handles columns 32 k + l, so each
// store instruction of a warp covers 32 consecutive pixels (512 B of float4).
// Pixels 32 k + l and 32 (k+1) + l are evaluated as a pair with the paired
// FP32 instructions (FADD2 / FMUL2 / FFMA2), whose per-lane results are those
// of the scalar operations. Per-column terms are computed once per tile. Mask
// bytes are gathered with one ballot per 32 pixels and written as TX/32
// consecutive bytes per lane.
template <int TX, int TY, int NT, int OUT, bool SECANT, bool FULL, class Stencil, bool POINTS = false>
__device__ __forceinline__ void compute_tile_with(const float* __restrict__ F, int bw, int padx,
                                                  const TileFrame& f, int gx0, int gy0, int halo, float tau2,
                                                  const Stencil& st) {
  constexpr int NW = NT / 32;
  constexpr int CH = TX / 32;
  constexpr int NP = CH / 2;
  static_assert(TY % NW == 0, "rows must divide among warps");
  static_assert(CH == 2 || CH == 4, "TX must be 64 or 128");
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;

  float2 nu1[NP], ku[NP];
  bool colok[CH];
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
    const float v1 = ((float)gy - f.cy) * f.inv_fy;
    const float2 nv1 = f2(-v1, -v1);
    const float2 kv = f2(v1 * v1, v1 * v1);
    const float* row = F + (ly + halo) * bw + padx + lane;
    const long long out_row = (long long)gy * f.out_pitch + gx0 + lane;
    uint32_t ballots[CH];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const float* pa = row + 64 * p;
      const float* pb = pa + 32;
      const float2 d1 = f2(NRM_LDS(float, pa), NRM_LDS(float, pb));
      float2 nx, ny, P;
      st(pa, pb, d1, nx, ny, P);
      emit_pair<OUT, SECANT, FULL>(f, out_row, p, d1, nx, ny, P, nu1[p], ku[p], nv1, kv, T, tau2, colok[2 * p],
                                   colok[2 * p + 1], ballots[2 * p], ballots[2 * p + 1]);
    }
    emit_mask_row<CH, FULL>(f, gx0, gy, lane, ballots);
  }
  if (POINTS && f.points) {
    // Organised point cloud P = d1 (u1, v1, 1) in metres (Section 2), the
    // origin where d1 is invalid (independent of the normal mask): a second
    // pass over the decoded tile, compiled only into the kernels instantiated
    // with POINTS (they need more registers than the normal-only kernels).
#pragma unroll 1
    for (int ly = warp; ly < TY; ly += NW) {
      const int gy = gy0 + ly;
      if (gy >= f.H) break;
      const float v1 = ((float)gy - f.cy) * f.inv_fy;
      const float* row = F + (ly + halo) * bw + padx + lane;
      float4* prow = reinterpret_cast<float4*>(f.points) + (long long)gy * f.out_pitch + gx0 + lane;
#pragma unroll
      for (int c = 0; c < CH; ++c) {
        const float d = NRM_LDS(float, row + 32 * c);
        const float z = d * f.point_scale;
        const float u1 = (c & 1) ? -nu1[c >> 1].y : -nu1[c >> 1].x;
        const float4 q = d == d ? make_float4(z * u1, z * v1, z, 0.0f) : make_float4(0.f, 0.f, 0.f, 0.f);
        if ((FULL || colok[c]) && NRM_GOK(prow + 32 * c, f.points, dbg_span(f.H, f.W, f.out_pitch, 16)))
          __stcs(prow + 32 * c, q);
      }
    }
  }
}

template <int TX, int TY, int NT, int OUT, bool SECANT, bool FULL, bool POINTS>
__device__ __forceinline__ void compute_tile(const float* __restrict__ F, int bw, int padx,
                                             const TileFrame& f, int gx0, int gy0, int alpha,
                                             float tau2) {
  const QuadStencil st{f2(f.a, f.a), f2(f.b, f.b), f2(f.c, f.c), alpha, alpha * bw};
  compute_tile_with<TX, TY, NT, OUT, SECANT, FULL, QuadStencil, POINTS>(F, bw, padx, f, gx0, gy0, alpha, tau2, st);
}

// compute_tile for the tile's mask mode, with the column checks compiled out
// for tiles that lie entirely inside the image width (all but the last tile
// column of a frame whose width is not a multiple of TX).
template <int TX, int TY, int NT, int OUT, bool POINTS>
__device__ __forceinline__ void compute_tile_any(const float* __restrict__ F, int bw, int padx,
                                                 const TileFrame& f, int gx0, int gy0, const Globals& g) {
  const bool full = gx0 + TX <= f.W;
  if (g.mask_mode == NRM_MASK_SECANT) {
    if (full)
      compute_tile<TX, TY, NT, OUT, true, true, POINTS>(F, bw, padx, f, gx0, gy0, g.alpha, g.tau2);
    else
      compute_tile<TX, TY, NT, OUT, true, false, POINTS>(F, bw, padx, f, gx0, gy0, g.alpha, g.tau2);
  } else {
    if (full)
      compute_tile<TX, TY, NT, OUT, false, true, POINTS>(F, bw, padx, f, gx0, gy0, g.alpha, g.tau2);
    else
      compute_tile<TX, TY, NT, OUT, false, false, POINTS>(F, bw, padx, f, gx0, gy0, g.alpha, g.tau2);
  }
}

}  // namespace dev
}  // namespace nrm
