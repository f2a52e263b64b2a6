// The vector tile loop of the forward kernels for half4 and octahedral
// outputs (arXiv 2209.08241, Section 3.1 Eq. 4-6 and the Section 3.2 mask),
// for pixel distance ALPHA = 1 or 2 known at compile time.
//
// Each lane evaluates V consecutive pixels of one row per step, as many as one
// 16-byte store of its output holds (half4: 2, octahedral: 4), so that:
//  - the five depths of the stencil come from five vector loads of the decoded
//    float tile per V pixels (the centre run and the runs ALPHA rows above and
//    below it, plus two 2-element runs left and right of it), at offsets
//    fixed at compile time;
//  - the output of V pixels is one 16-byte streaming store (a warp writes 512
//    contiguous bytes) and their mask bytes one 2- or 4-byte store;
//  - consecutive pixels form the operand pairs of the paired FP32
//    instructions (FADD2 / FMUL2 / FFMA2) without register moves (ALPHA = 2).
// The per-column terms (-u1, 1 + u1^2) and per-row terms (-v1, v1^2) come
// from tables that the compute threads write next to the decoded tile while
// they decode it. The arithmetic of each pixel is that of emit_pair, operation
// for operation, so both loops give the same bits; tiles that reach past the
// frame's right edge, unaligned outputs and other distances take the scalar
// loop (compute_tile_any).
#pragma once

#include "nrm_device.cuh"

namespace nrm {
namespace dev {

// Column and row tables of a decoded tile (after the float tile in its
// buffer), written by compute thread t < TX / 2 + TY: column pair j (tile
// columns 2j, 2j + 1) -> (-u1, -u1', 1 + u1^2, 1 + u1'^2); row r ->
// (-v1, -v1, v1^2, v1^2). u1 = (col - cx) / fx and v1 = (row - cy) / fy are
// formed as in compute_tile_with.
template <int TX, int TY>
__device__ __forceinline__ void fill_tile_tables(float4* tab, const TileFrame& f, int gx0, int gy0, int t) {
  if (t < TX / 2) {
    const float ua = ((float)(gx0 + 2 * t) - f.cx) * f.inv_fx;
    const float ub = ((float)(gx0 + 2 * t + 1) - f.cx) * f.inv_fx;
    NRM_STS(tab + t, make_float4(-ua, -ub, fmaf(ua, ua, 1.0f), fmaf(ub, ub, 1.0f)));
  } else if (t < TX / 2 + TY) {
    const int r = t - TX / 2;
    const float v1 = ((float)(gy0 + r) - f.cy) * f.inv_fy;
    NRM_STS(tab + t, make_float4(-v1, -v1, v1 * v1, v1 * v1));
  }
}

template <int TX, int TY, int ALPHA>
__device__ __forceinline__ const float4* tile_tables(const float* F) {
  return reinterpret_cast<const float4*>(reinterpret_cast<const unsigned char*>(F) +
                                         ftile_float_bytes(TX, TY, ALPHA));
}

// Decodes a TMA-staged uint16 halo tile into the float tile for ALPHA <= 2
// (geometry fixed at compile time: staging pitch TX + 16 elements, float tile
// pitch TX + 8, float column c <- staged column c + 4, TY + 2 ALPHA rows), with
// no division: each warp pass converts M = TX / 4 groups of four elements of
// 32 / M rows (lane l: row l / M, group l % M, the tile's own columns), and one
// more set of passes converts the two 4-column halo groups of each row (16
// rows per pass). Same values as decode_tile.
template <int TX, int TY, int NT, int ALPHA>
__device__ __forceinline__ void decode_tile_u16_fixed(const uint16_t* __restrict__ src, float* __restrict__ dst) {
  constexpr int SP = TX + 16;  // staged row pitch: pad_x(alpha, 2) = 8 for alpha <= 8
  constexpr int FW = TX + 8;   // float tile pitch: pad_x(alpha, 4) = 4 for alpha <= 4
  constexpr int ROWS = TY + 2 * ALPHA;
  constexpr int M = TX / 4;
  constexpr int RP = 32 / M;
  constexpr int NW = NT / 32;
  static_assert(M * RP == 32, "TX must be 64 or 128");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane % M;
  const float2 kb = f2(-8388607.0f, -8388607.0f);
  auto cvt4 = [&](const uint16_t* s, float* d) {
    const uint2 raw = NRM_LDS(uint2, reinterpret_cast<const uint2*>(s));
    // (u - 1) | 0x4B000000 is the float 2^23 + u - 1 for u >= 1 and a NaN for
    // u = 0; subtracting 2^23 - 1 gives u exactly and keeps the NaN.
    const float2 lo = __fadd2_rn(f2(__uint_as_float(((raw.x & 0xFFFFu) - 1u) | 0x4B000000u),
                                    __uint_as_float(((raw.x >> 16) - 1u) | 0x4B000000u)), kb);
    const float2 hi = __fadd2_rn(f2(__uint_as_float(((raw.y & 0xFFFFu) - 1u) | 0x4B000000u),
                                    __uint_as_float(((raw.y >> 16) - 1u) | 0x4B000000u)), kb);
    NRM_STS(reinterpret_cast<float4*>(d), make_float4(lo.x, lo.y, hi.x, hi.y));
  };
#pragma unroll 1
  for (int r = warp * RP + lane / M; r < ROWS; r += NW * RP) cvt4(src + r * SP + 8 + 4 * g, dst + r * FW + 4 + 4 * g);
  for (int h = threadIdx.x; h < 2 * ROWS; h += NT) {
    const int r = h >> 1;
    const int c = (h & 1) ? TX + 4 : 0;  // float column of the halo group
    cvt4(src + r * SP + 4 + c, dst + r * FW + c);
  }
}

// The staged tile of a persistent or plain launch decoded into the float tile.
template <int TX, int TY, int NT>
__device__ __forceinline__ void decode_staged(const unsigned char* stage, float* F, bool u16, int alpha, int fw,
                                              int bh, int bw, int skip) {
  if (u16) {
    if (alpha == 2)
      decode_tile_u16_fixed<TX, TY, NT, 2>(reinterpret_cast<const uint16_t*>(stage), F);
    else if (alpha == 1)
      decode_tile_u16_fixed<TX, TY, NT, 1>(reinterpret_cast<const uint16_t*>(stage), F);
    else
      decode_tile<NT>(reinterpret_cast<const uint16_t*>(stage), F, fw, bh, bw, skip);
  } else {
    decode_tile<NT>(reinterpret_cast<const float*>(stage), F, fw, bh, bw, 0);
  }
}

// Pixels per lane and step of the vector loop.
template <int TX, int OUT>
struct VecShape {
  static constexpr int BPP = OUT == NRM_OUT_F16X4 ? 8 : 4;  // output bytes per pixel
  static constexpr int V = (16 / BPP) < (TX / 32) ? (16 / BPP) : (TX / 32);
};

// True if frame f's outputs allow the vector stores: normals base and row
// pitch aligned to V pixels of output, mask base and pitch to V bytes.
template <int TX, int OUT>
__device__ __forceinline__ bool vec_aligned(const TileFrame& f) {
  using S = VecShape<TX, OUT>;
  return f.out_align >= S::V * S::BPP && f.mask_align >= S::V;
}

// Section 3.2 for one pixel pair: n_z, q = n . n and the mask decisions, in
// the operation order of emit_pair.
template <bool SECANT>
__device__ __forceinline__ void pair_decide(float2 d1, float2 nx, float2 ny, float2 P, float2 nu1, float2 ku,
                                            float2 nv1, float2 kv, float2 T, float tau2, float2& nz, float2& q,
                                            bool& ka, bool& kb) {
  const float kFltMin = 1.17549435e-38f;
  nz = __ffma2_rn(nu1, nx, __ffma2_rn(nv1, ny, P));
  q = __ffma2_rn(nx, nx, __ffma2_rn(ny, ny, __fmul2_rn(nz, nz)));
  ka = (d1.x == d1.x) & (q.x >= kFltMin);
  kb = (d1.y == d1.y) & (q.y >= kFltMin);
  if (SECANT) {
    const float2 lhs = __fmul2_rn(q, __fadd2_rn(ku, kv));
    const float2 rhs = __fmul2_rn(T, __fmul2_rn(P, P));
    ka = ka & (lhs.x <= rhs.x);
    kb = kb & (lhs.y <= rhs.y);
  } else {
    ka = ka & (q.x <= tau2);
    kb = kb & (q.y <= tau2);
  }
}

__device__ __forceinline__ uint32_t h2_bits(__half2 h) { return *reinterpret_cast<const uint32_t*>(&h); }

// One FULL tile (gx0 + TX <= W) with aligned outputs. Warp w takes column
// segment w % SEGX (32 V columns) and rows w / SEGX, w / SEGX + NW / SEGX, ...
template <int TX, int TY, int NT, int OUT, bool SECANT, int ALPHA>
__device__ __forceinline__ void compute_tile_vec(const float* __restrict__ F, const TileFrame& f, int gx0, int gy0,
                                                 float tau2) {
  using S = VecShape<TX, OUT>;
  constexpr int V = S::V;
  constexpr int BPP = S::BPP;
  constexpr int SEGX = TX / (32 * V);
  constexpr int NW = NT / 32;
  static_assert(V == 2 || V == 4, "two or four pixels per lane");
  static_assert(ALPHA == 1 || ALPHA == 2, "compiled distances");
  static_assert(NW % SEGX == 0, "each warp keeps one column segment");
  constexpr int RSTEP = NW / SEGX;
  static_assert(TY % RSTEP == 0, "rows must divide among warps");
  constexpr int NR = TY / RSTEP;
  constexpr int FW = TX + 8;  // decoded tile pitch: pad_x(alpha, 4) = 4 for alpha <= 4
  constexpr int NP = V / 2;   // pixel pairs per lane and step
  const float4* tab = tile_tables<TX, TY, ALPHA>(F);
  const float4* rtab = tab + TX / 2;

  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int cs = warp % SEGX;
  const int r0 = warp / SEGX;
  const int xl = cs * 32 * V + lane * V;  // tile column of the lane's first pixel

  float2 nu1[NP], ku[NP];
#pragma unroll
  for (int j = 0; j < NP; ++j) {
    const float4 c = NRM_LDS(float4, tab + xl / 2 + j);
    nu1[j] = f2(c.x, c.y);
    ku[j] = f2(c.z, c.w);
  }
  const float2 A = f2(f.a, f.a), B = f2(f.b, f.b), C = f2(f.c, f.c);
  const float2 T = f2(tau2, tau2);
  const float2 M1 = f2(-1.0f, -1.0f);

  const float* Fc = F + (ALPHA + r0) * FW + 4 + xl;
  unsigned char* nptr = reinterpret_cast<unsigned char*>(f.normals) +
                        ((long long)(gy0 + r0) * f.out_pitch + gx0 + xl) * BPP;
  uint8_t* mptr = f.valid + (long long)(gy0 + r0) * f.out_pitch + gx0 + xl;
  const long long nstep = (long long)RSTEP * f.out_pitch * BPP;
  const long long mstep = (long long)RSTEP * f.out_pitch;
  const int rows = f.H - gy0 - r0;  // this warp's rows k RSTEP < rows lie in the frame

#pragma unroll
  for (int k = 0; k < NR; ++k) {
    if (k * RSTEP >= rows) break;
    const float* p = Fc + k * RSTEP * FW;
    // rowv[i + 2] = depth of pixel i of this step (i = -2 .. V + 1).
    float rowv[V + 4];
    float up[V], dn[V];
    if (V == 4) {
      const float4 c = NRM_LDS(float4, reinterpret_cast<const float4*>(p));
      const float4 u = NRM_LDS(float4, reinterpret_cast<const float4*>(p - ALPHA * FW));
      const float4 d = NRM_LDS(float4, reinterpret_cast<const float4*>(p + ALPHA * FW));
      rowv[2] = c.x, rowv[3] = c.y, rowv[4] = c.z, rowv[5] = c.w;
      up[0] = u.x, up[1] = u.y, up[2] = u.z, up[3] = u.w;
      dn[0] = d.x, dn[1] = d.y, dn[2] = d.z, dn[3] = d.w;
    } else {
      const float2 c = NRM_LDS(float2, reinterpret_cast<const float2*>(p));
      const float2 u = NRM_LDS(float2, reinterpret_cast<const float2*>(p - ALPHA * FW));
      const float2 d = NRM_LDS(float2, reinterpret_cast<const float2*>(p + ALPHA * FW));
      rowv[2] = c.x, rowv[3] = c.y;
      up[0] = u.x, up[1] = u.y;
      dn[0] = d.x, dn[1] = d.y;
    }
    if (ALPHA == 2) {
      const float2 l = NRM_LDS(float2, reinterpret_cast<const float2*>(p - 2));
      const float2 r = NRM_LDS(float2, reinterpret_cast<const float2*>(p + V));
      rowv[0] = l.x, rowv[1] = l.y;
      rowv[V + 2] = r.x, rowv[V + 3] = r.y;
    } else {
      rowv[0] = 0.0f, rowv[1] = NRM_LDS(float, p - 1);
      rowv[V + 2] = NRM_LDS(float, p + V), rowv[V + 3] = 0.0f;
    }
    const float4 rr = NRM_LDS(float4, rtab + r0 + k * RSTEP);
    const float2 nv1 = f2(rr.x, rr.y), kv = f2(rr.z, rr.w);

    uint32_t w[V * BPP / 4];
    uint32_t mbits = 0;
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      const int i = 2 * j;  // pixels i, i + 1
      const float2 d1 = f2(rowv[i + 2], rowv[i + 3]);
      const float2 d2 = f2(rowv[i + 2 + ALPHA], rowv[i + 3 + ALPHA]);
      const float2 d4 = f2(rowv[i + 2 - ALPHA], rowv[i + 3 - ALPHA]);
      const float2 d3 = f2(dn[i], dn[i + 1]);
      const float2 d5 = f2(up[i], up[i + 1]);
      // The QuadStencil arithmetic.
      const float2 S24 = __fadd2_rn(d2, d4), D24 = __ffma2_rn(M1, d4, d2);
      const float2 S35 = __fadd2_rn(d3, d5), D35 = __ffma2_rn(M1, d5, d3);
      const float2 nx = __fmul2_rn(__fmul2_rn(A, S35), D24);
      const float2 ny = __fmul2_rn(__fmul2_rn(B, S24), D35);
      const float2 P = __fmul2_rn(__fmul2_rn(C, S24), S35);
      float2 nz, q;
      bool ka, kb;
      pair_decide<SECANT>(d1, nx, ny, P, nu1[j], ku[j], nv1, kv, T, tau2, nz, q, ka, kb);
      mbits |= (ka ? 1u : 0u) << (8 * i);
      mbits |= (kb ? 1u : 0u) << (8 * i + 8);
      if (OUT == NRM_OUT_OCT16) {
        uint32_t ca, cb;
        oct16_encode2(nx, ny, nz, ca, cb);
        w[i] = ka ? ca : 0u;
        w[i + 1] = kb ? cb : 0u;
      } else {
        const float2 inv = f2(rsqrt_ftz(q.x), rsqrt_ftz(q.y));
        const float2 ox = __fmul2_rn(nx, inv), oy = __fmul2_rn(ny, inv), oz = __fmul2_rn(nz, inv);
        const uint32_t xya = h2_bits(__floats2half2_rn(ox.x, oy.x)), zwa = h2_bits(__floats2half2_rn(oz.x, 0.0f));
        const uint32_t xyb = h2_bits(__floats2half2_rn(ox.y, oy.y)), zwb = h2_bits(__floats2half2_rn(oz.y, 0.0f));
        w[2 * i] = ka ? xya : 0u;
        w[2 * i + 1] = ka ? zwa : 0u;
        w[2 * i + 2] = kb ? xyb : 0u;
        w[2 * i + 3] = kb ? zwb : 0u;
      }
    }
    unsigned char* np_ = nptr + k * nstep;
    uint8_t* mp = mptr + k * mstep;
    [[maybe_unused]] const long long nlen = dbg_span(f.H, f.W, f.out_pitch, BPP);
    [[maybe_unused]] const long long mlen = dbg_span(f.H, f.W, f.out_pitch, 1);
    if (V * BPP == 16) {
      uint4* q = reinterpret_cast<uint4*>(np_);
      if (NRM_GOK(q, f.normals, nlen)) __stcs(q, make_uint4(w[0], w[1], w[2], w[3]));
    } else {
      uint2* q = reinterpret_cast<uint2*>(np_);
      if (NRM_GOK(q, f.normals, nlen)) __stcs(q, make_uint2(w[0], w[1]));
    }
    if (V == 4) {
      unsigned int* q = reinterpret_cast<unsigned int*>(mp);
      if (NRM_GOK(q, f.valid, mlen)) __stcs(q, mbits);
    } else {
      unsigned short* q = reinterpret_cast<unsigned short*>(mp);
      if (NRM_GOK(q, f.valid, mlen)) __stcs(q, (unsigned short)mbits);
    }
  }
}

// The forward tile: the vector loop where it applies (see the file comment),
// else the scalar loop.
template <int TX, int TY, int NT, int OUT, bool POINTS>
__device__ __forceinline__ void compute_tile_fwd(const float* __restrict__ F, int bw, int padx, const TileFrame& f,
                                                 int gx0, int gy0, const Globals& g) {
  if constexpr (OUT != NRM_OUT_F32X4 && !POINTS) {
    if (gx0 + TX <= f.W && (g.alpha == 1 || g.alpha == 2) && vec_aligned<TX, OUT>(f)) {
      if (g.alpha == 2) {
        if (g.mask_mode == NRM_MASK_SECANT)
          compute_tile_vec<TX, TY, NT, OUT, true, 2>(F, f, gx0, gy0, g.tau2);
        else
          compute_tile_vec<TX, TY, NT, OUT, false, 2>(F, f, gx0, gy0, g.tau2);
      } else {
        if (g.mask_mode == NRM_MASK_SECANT)
          compute_tile_vec<TX, TY, NT, OUT, true, 1>(F, f, gx0, gy0, g.tau2);
        else
          compute_tile_vec<TX, TY, NT, OUT, false, 1>(F, f, gx0, gy0, g.tau2);
      }
      return;
    }
  }
  compute_tile_any<TX, TY, NT, OUT, POINTS>(F, bw, padx, f, gx0, gy0, g);
}

}  // namespace dev
}  // namespace nrm
