// Adjoint of the forward normal map with respect to float32 depth, mask held
// fixed (arXiv 2209.08241: derivatives of Eq. 4-6 and of the normalisation).
//
// For a valid pixel p with unit normal n_hat = s n / ||n|| (s = +-1) and upstream
// gradient g_p = dL/d(n_hat_p):
//   h_p = s (g_p - (g_p . n_hat) n_hat) / ||n||            (d n_hat / d n)^T g_p
// and, with e_x = h_x - u1 h_z, e_y = h_y - v1 h_z (the n_z row of Eq. 6 folded in),
// the four depth weights w_k(p) = h_p . dn/dd_k are
//   w2 = -e_x a S35 - e_y b D35 + h_z c S35
//   w4 = +e_x a S35 - e_y b D35 + h_z c S35
//   w3 = -e_x a D24 - e_y b S24 + h_z c S24
//   w5 = -e_x a D24 + e_y b S24 + h_z c S24
// (a, b, c the Eq. 4-6 constants). dn/dd1 = 0. Each depth pixel q then gathers
//   dL/dd_q = w2(q - alpha x) + w4(q + alpha x) + w3(q - alpha y) + w5(q + alpha y),
// a deterministic gather with no atomics.
//
// One CTA per 64 x 32 output tile. Three TMA loads on one mbarrier stage the
// tile's inputs in shared memory: the depth halo of radius 2 alpha, the upstream
// gradient of the tile extended by alpha (a 2-D box of 8-byte elements, two per
// pixel, i.e. float4 per pixel) and the mask of the same region (a
// uint8 box starting 16 columns left of the tile, the alignment TMA needs).
// Phase 1 turns each staged gradient into the four weights in place; phase 2
// gathers. Frames whose buffers cannot be TMA-mapped use plain loads into the
// same shared-memory layout. bwd_kernel covers one frame (grid = its tiles);
// bwd_batched_kernel covers a batch (grid = max tiles of a frame x frames).
// Both are compiled for alpha = 1..4 as constants (shared-memory offsets and
// loop steps become immediates) and once for any alpha.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "nrm_device.cuh"

namespace nrm {

using namespace dev;

namespace {

constexpr int TX = kBwdTileX;
constexpr int TY = kBwdTileY;
constexpr int NT = kBwdThreads;
constexpr int NW = NT / 32;
constexpr int MW = kBwdMaskBoxW;   // mask tile pitch (bytes)
constexpr int MP = kBwdMaskPad;    // mask tile column of global x = gx0 - MP

__host__ __device__ inline unsigned round128(unsigned b) { return (b + 127) / 128 * 128; }
__host__ __device__ inline unsigned depth_tile_bytes(int alpha) {
  return round128((unsigned)((TX + 2 * pad_x(2 * alpha, 4)) * (TY + 4 * alpha) * 4));
}
__host__ __device__ inline unsigned weight_tile_bytes(int alpha) {
  return round128((unsigned)((TX + 2 * alpha) * (TY + 2 * alpha) * 16));
}
__host__ __device__ inline unsigned mask_tile_bytes(int alpha) {
  return round128((unsigned)(MW * (TY + 2 * alpha)));
}
// u1 of each column and v1 of each row of the extended region.
__host__ __device__ inline unsigned coord_table_bytes(int alpha) {
  return round128((unsigned)((TX + TY + 4 * alpha) * 4));
}

// One output tile (gx0, gy0) of frame fd. tmap_d/tmap_g/tmap_m: its depth,
// gradient and mask tensor maps (param or global memory; used only when
// fd.use_tma). If the bounded wait for the copies runs out, the tile records
// NRM_ERR_TIMEOUT in the status word and writes nothing.
// ALPHA > 0 compiles the tile for that pixel distance (offsets and loop steps
// become constants); ALPHA = 0 takes g.alpha at run time.
template <int ALPHA>
__device__ __forceinline__ void bwd_tile(const FrameDesc& fd, const void* tmap_d, const void* tmap_g,
                                         const void* tmap_m, int gx0, int gy0, const Globals& g,
                                         unsigned char* smem, const float* __restrict__ scale, int frame) {
  // Upstream gradient = scale[frame] x the staged float4 when scale is given
  // (the fused loss entry: the staged values are then target normals).
  const float sc = scale ? __ldg(scale + frame) : 1.0f;
  const int alpha = ALPHA > 0 ? ALPHA : g.alpha;
  const int p2 = pad_x(2 * alpha, 4);
  const int bw = TX + 2 * p2;       // depth tile pitch
  const int bh = TY + 4 * alpha;
  const int ex_w = TX + 2 * alpha;  // extended region (gradient / weight / mask)
  const int ex_h = TY + 2 * alpha;
  float* dep = reinterpret_cast<float*>(smem);
  float4* gw = reinterpret_cast<float4*>(smem + depth_tile_bytes(alpha));
  uint8_t* msk = smem + depth_tile_bytes(alpha) + weight_tile_bytes(alpha);
  float* ucol = reinterpret_cast<float*>(msk + mask_tile_bytes(alpha));  // u1 of extended column ex
  float* vrow = ucol + ex_w;                                              // v1 of extended row ey
  uint64_t* bar = reinterpret_cast<uint64_t*>(reinterpret_cast<unsigned char*>(ucol) + coord_table_bytes(alpha));
  const int H = fd.H, W = fd.W;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // The ray coordinates of the extended region, formed while the copies are
  // in flight (the barrier that follows them publishes these too).
  for (int t = threadIdx.x; t < ex_w + ex_h; t += NT) {
    if (t < ex_w)
      NRM_STS(ucol + t, ((float)(gx0 - alpha + t) - fd.cx) * fd.inv_fx);
    else
      NRM_STS(vrow + t - ex_w, ((float)(gy0 - alpha + t - ex_w) - fd.cy) * fd.inv_fy);
  }

  if (fd.use_tma) {
    const uint32_t b = smem_u32(bar);
    if (threadIdx.x == 0) {
      mbar_init(b, 1);
      fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      mbar_arrive_expect_tx(b, (uint32_t)(bw * bh * 4 + ex_w * ex_h * 16 + MW * ex_h));
      tma_load_2d(smem_u32(dep), tmap_d, gx0 - p2, gy0 - 2 * alpha, b);
      tma_load_2d(smem_u32(gw), tmap_g, 2 * (gx0 - alpha), gy0 - alpha, b);  // x in 8-byte units: even
      tma_load_2d(smem_u32(msk), tmap_m, gx0 - MP, gy0 - alpha, b);
    }
    const bool ok = mbar_wait_warp(b, 0, g.timeout_ns);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {
        record_error(g.status, NRM_ERR_TIMEOUT);
        mbar_wait_bounded(b, 0, g.timeout_ns);
      }
      return;
    }
  } else {
    load_tile_plain(dep, bw, bh, fd, gx0 - p2, gy0 - 2 * alpha);
    const float4* gn = reinterpret_cast<const float4*>(fd.normals);
    for (int ey = warp; ey < ex_h; ey += NW) {
      const int py = gy0 - alpha + ey;
      for (int ex = lane; ex < ex_w; ex += 32) {
        const int px = gx0 - alpha + ex;
        const bool in = px >= 0 && py >= 0 && px < W && py < H;
        const long long o = (long long)py * fd.out_pitch + px;
        NRM_STS(gw + ey * ex_w + ex, in ? __ldg(gn + o) : make_float4(0.f, 0.f, 0.f, 0.f));
        NRM_STS(msk + ey * MW + ex + MP - alpha, in ? __ldg(fd.valid + o) : (uint8_t)0);
      }
    }
    __syncthreads();
  }

  // Phase 1: the weights of every pixel p of the extended tile, in place of
  // its staged gradient. Threads walk the ex_w x ex_h elements in row-major
  // order with stride NT, advancing (ey, ex) by increments (no division).
  // A pixel the forward marked valid has a positive finite five-point stencil
  // (that is what made it valid), so only the mask is consulted here.
  // With A35 = a S35, B35 = b D35, C35 = c S35 and A24 = a D24, B24 = b S24,
  // C24 = c S24, Eq. 4-6 read n_x = -A35 D24, n_y = -B24 D35, P = C24 S35, and
  // the weights (e_x = h_x - u1 h_z, e_y = h_y - v1 h_z) are
  //   w2 = -e_x A35 - e_y B35 + h_z C35,  w4 = e_x A35 - e_y B35 + h_z C35,
  //   w3 = -e_x A24 - e_y B24 + h_z C24,  w5 = -e_x A24 + e_y B24 + h_z C24.
  const float ka = fd.a, kb = fd.b, kc = fd.c;
  const int n_ext = ex_w * ex_h;
  const int step_rows = NT / ex_w, step_cols = NT - step_rows * ex_w;
  int ey = threadIdx.x / ex_w;
  int ex = threadIdx.x - ey * ex_w;
  const float* dep_c = dep + alpha * bw + p2 - alpha;  // depth-tile position of (ey, ex) = (0, 0)
  const uint8_t* msk_c = msk + MP - alpha;
  for (int i = threadIdx.x; i < n_ext; i += NT) {
    float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
    if (NRM_LDS(uint8_t, msk_c + ey * MW + ex)) {
      const float* pc = dep_c + ey * bw + ex;
      const float d2 = NRM_LDS(float, pc + alpha), d4 = NRM_LDS(float, pc - alpha);
      const float d3 = NRM_LDS(float, pc + alpha * bw), d5 = NRM_LDS(float, pc - alpha * bw);
      const float S24 = d2 + d4, D24 = d2 - d4, S35 = d3 + d5, D35 = d3 - d5;
      const float u1 = NRM_LDS(float, ucol + ex), v1 = NRM_LDS(float, vrow + ey);
      const float A35 = ka * S35, B35 = kb * D35, C35 = kc * S35;
      const float A24 = ka * D24, B24 = kb * S24, C24 = kc * S24;
      const float nx = -A35 * D24, ny = -B24 * D35, P = C24 * S35;
      const float nz = fmaf(-u1, nx, fmaf(-v1, ny, P));
      const float q = fmaf(nx, nx, fmaf(ny, ny, nz * nz));
      const float inv = rsqrt_ftz(fmaxf(q, 1.17549435e-38f));
      const float hx0 = nx * inv, hy0 = ny * inv, hz0 = nz * inv;
      float4 gv = NRM_LDS(float4, gw + i);
      if (scale) {
        gv.x *= sc;
        gv.y *= sc;
        gv.z *= sc;
      }
      const float gd = fmaf(gv.x, hx0, fmaf(gv.y, hy0, gv.z * hz0));
      const float si = g.sign * inv;
      const float hx = fmaf(-gd, hx0, gv.x) * si;
      const float hy = fmaf(-gd, hy0, gv.y) * si;
      const float hz = fmaf(-gd, hz0, gv.z) * si;
      const float e_x = fmaf(-u1, hz, hx);
      const float e_y = fmaf(-v1, hz, hy);
      const float c35 = fmaf(hz, C35, -e_y * B35);
      const float c24 = fmaf(hz, C24, -e_x * A24);
      w.x = fmaf(-e_x, A35, c35);  // w2
      w.y = fmaf(-e_y, B24, c24);  // w3
      w.z = fmaf(e_x, A35, c35);   // w4
      w.w = fmaf(e_y, B24, c24);   // w5
    }
    NRM_STS(gw + i, w);
    ey += step_rows;
    ex += step_cols;
    if (ex >= ex_w) {
      ex -= ex_w;
      ++ey;
    }
  }
  __syncthreads();
  // Phase 2: gather.
  float* __restrict__ grad = fd.grad_depth;
  for (int ly = warp; ly < TY; ly += NW) {
    const int qy = gy0 + ly;
    if (qy >= H) break;
    for (int lx = lane; lx < TX; lx += 32) {
      const int qx = gx0 + lx;
      if (qx >= W) break;
      const int c = (ly + alpha) * ex_w + (lx + alpha);
      const float v = NRM_LDS(float4, gw + c - alpha).x + NRM_LDS(float4, gw + c + alpha).z +
                      NRM_LDS(float4, gw + c - alpha * ex_w).y + NRM_LDS(float4, gw + c + alpha * ex_w).w;
      float* q = grad + (long long)qy * fd.depth_pitch + qx;
      if (NRM_GOK(q, grad, dbg_span(H, W, fd.depth_pitch, 4))) *q = v;
    }
  }
}

template <int ALPHA>
__global__ void __launch_bounds__(NT)
    bwd_kernel(const __grid_constant__ FrameDesc fd, const __grid_constant__ BwdMaps maps, const Globals g,
               const float* scale) {
  extern __shared__ __align__(128) unsigned char smem[];
  NRM_DEBUG_ENTRY(g.status);
  bwd_tile<ALPHA>(fd, &fd.tmap, &maps.grad, &maps.mask, blockIdx.x * TX, blockIdx.y * TY, g, smem, scale, 0);
}

// Grid (max tiles of a frame, frames): block (x, f) is tile x of frame f; frames
// with fewer tiles leave their extra blocks idle.
template <int ALPHA>
__global__ void __launch_bounds__(NT) bwd_batched_kernel(const BwdBatchArgs args, const Globals g, const float* scale) {
  extern __shared__ __align__(128) unsigned char smem[];
  NRM_DEBUG_ENTRY(g.status);
  const int f = (int)blockIdx.y;
  const FrameDesc& fd = args.frames[f];
  const int tiles_x = fd.tiles_x;
  const int local = (int)blockIdx.x;
  if (tiles_x == 0 || local >= tiles_x * ((fd.H + TY - 1) / TY)) return;
  if (threadIdx.x == 0 && fd.use_tma) {
    fence_tensormap_acquire(&fd.tmap);
    fence_tensormap_acquire(&args.maps[f].grad);
    fence_tensormap_acquire(&args.maps[f].mask);
  }
  const int ty = local / tiles_x;
  const int tx = local - ty * tiles_x;
  bwd_tile<ALPHA>(fd, &fd.tmap, &args.maps[f].grad, &args.maps[f].mask, tx * TX, ty * TY, g, smem, scale, f);
}

// A batch of at most kBwdParamMaxFrames frames with its records and tensor
// maps in kernel-parameter space: no descriptor upload and no tensor-map fence
// (each CTA of the global-memory form fences three maps for its one tile).
struct alignas(128) BwdParamBatch {
  FrameDesc frames[kBwdParamMaxFrames];
  BwdMaps maps[kBwdParamMaxFrames];
};
static_assert(sizeof(BwdParamBatch) <= 32764, "the descriptor block must fit the kernel parameter limit");

// Grid (max tiles of a frame, frames), as bwd_batched_kernel.
template <int ALPHA>
__global__ void __launch_bounds__(NT)
    bwd_batched_param_kernel(const __grid_constant__ BwdParamBatch pb, const Globals g, const float* scale) {
  extern __shared__ __align__(128) unsigned char smem[];
  NRM_DEBUG_ENTRY(g.status);
  const int f = (int)blockIdx.y;
  const FrameDesc& fd = pb.frames[f];
  const int tiles_x = fd.tiles_x;
  const int local = (int)blockIdx.x;
  if (tiles_x == 0 || local >= tiles_x * ((fd.H + TY - 1) / TY)) return;
  const int ty = local / tiles_x;
  const int tx = local - ty * tiles_x;
  bwd_tile<ALPHA>(fd, &fd.tmap, &pb.maps[f].grad, &pb.maps[f].mask, tx * TX, ty * TY, g, smem, scale, f);
}

const void* bwd_param_kernel_for(int alpha) {
  switch (alpha) {
    case 1: return (const void*)bwd_batched_param_kernel<1>;
    case 2: return (const void*)bwd_batched_param_kernel<2>;
    case 3: return (const void*)bwd_batched_param_kernel<3>;
    case 4: return (const void*)bwd_batched_param_kernel<4>;
    default: return (const void*)bwd_batched_param_kernel<0>;
  }
}

// The kernel for alpha: compiled for alpha = 1..4 (constant offsets and loop
// steps), generic above.
const void* bwd_kernel_for(int alpha, bool batched) {
  switch (alpha) {
    case 1: return batched ? (const void*)bwd_batched_kernel<1> : (const void*)bwd_kernel<1>;
    case 2: return batched ? (const void*)bwd_batched_kernel<2> : (const void*)bwd_kernel<2>;
    case 3: return batched ? (const void*)bwd_batched_kernel<3> : (const void*)bwd_kernel<3>;
    case 4: return batched ? (const void*)bwd_batched_kernel<4> : (const void*)bwd_kernel<4>;
    default: return batched ? (const void*)bwd_batched_kernel<0> : (const void*)bwd_kernel<0>;
  }
}

// Grants the dynamic shared memory a kernel needs, once per (kernel, device)
// and size.
cudaError_t set_smem(const void* fn, unsigned bytes) {
  static std::map<std::pair<const void*, int>, unsigned> granted;
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  int dev = 0;
  cudaGetDevice(&dev);
  auto key = std::make_pair(fn, dev);
  auto it = granted.find(key);
  if (it != granted.end() && it->second >= bytes) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) granted[key] = bytes;
  return e;
}

// The per-frame factor of the cosine loss, scale = -1 / max(N_valid, 1), with
// N_valid the number of nonzero mask bytes of the frame: kCountBlocks blocks
// per frame count rows y = blockIdx.x, blockIdx.x + kCountBlocks, ...; each
// block adds its count to the frame's counter, and the last block of the frame
// to finish (the ordering of a fence and an atomic ticket) writes the scale
// and returns both counters to zero for the next call. Integer sums: the
// result does not depend on the order.
constexpr int kCountBlocks = 32;
constexpr int kCountThreads = 256;

struct CountArgs {
  LossCountFrame f[kLossCountMaxFrames];
};

__global__ void __launch_bounds__(kCountThreads)
    loss_scale_kernel(const __grid_constant__ CountArgs a, unsigned* __restrict__ counts,
                      unsigned* __restrict__ tickets, float* __restrict__ scale) {
  NRM_DEBUG_ENTRY(nullptr);
  const int f = (int)blockIdx.y;
  const LossCountFrame fr = a.f[f];
  unsigned c = 0;
  for (int y = blockIdx.x; y < fr.H; y += gridDim.x) {
    const uint8_t* row = fr.valid + (long long)y * fr.pitch;
    for (int x = threadIdx.x; x < fr.W; x += kCountThreads) c += __ldg(row + x) != 0 ? 1u : 0u;
  }
  c = __reduce_add_sync(0xffffffffu, c);
  __shared__ unsigned part[kCountThreads / 32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = 0;
    for (int w = 0; w < kCountThreads / 32; ++w) t += part[w];
    atomicAdd(counts + f, t);
    __threadfence();
    if (atomicAdd(tickets + f, 1u) == gridDim.x - 1) {
      const unsigned total = atomicExch(counts + f, 0u);
      atomicExch(tickets + f, 0u);
      scale[f] = -1.0f / (float)(total > 0 ? total : 1u);
    }
  }
}

}  // namespace

cudaError_t launch_loss_scale(const LossCountFrame* frames, int n, unsigned* counts, unsigned* tickets, float* scale,
                              cudaStream_t stream) {
  for (int first = 0; first < n; first += kLossCountMaxFrames) {
    const int m = std::min(kLossCountMaxFrames, n - first);
    CountArgs a;
    std::memset(&a, 0, sizeof(a));
    std::memcpy(a.f, frames + first, sizeof(LossCountFrame) * (size_t)m);
    unsigned* c = counts + first;
    unsigned* t = tickets + first;
    float* sc = scale + first;
    void* args[4] = {&a, &c, &t, &sc};
    cudaError_t e = cudaLaunchKernel((const void*)loss_scale_kernel, dim3(kCountBlocks, m), dim3(kCountThreads), args,
                                     0, stream);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

unsigned bwd_smem_bytes(int alpha) {
  return depth_tile_bytes(alpha) + weight_tile_bytes(alpha) + mask_tile_bytes(alpha) + coord_table_bytes(alpha) + 16;
}

cudaError_t launch_backward(const FrameDesc& fd, const BwdMaps& maps, const Globals& g, cudaStream_t stream,
                            const float* scale) {
  const unsigned smem = bwd_smem_bytes(g.alpha);
  const void* fn = bwd_kernel_for(g.alpha, false);
  cudaError_t e = set_smem(fn, smem);
  if (e != cudaSuccess) return e;
  dim3 grid((fd.W + TX - 1) / TX, (fd.H + TY - 1) / TY);
  FrameDesc d = fd;
  BwdMaps m = maps;
  Globals gg = g;
  const float* sc = scale;
  void* args[4] = {&d, &m, &gg, &sc};
  e = cudaLaunchKernel(fn, grid, dim3(NT), args, smem, stream);
  return e;
}

cudaError_t launch_backward_batched(const BwdBatchArgs& args, int n_frames, int max_tiles, const Globals& g,
                                    cudaStream_t stream, const float* scale) {
  const unsigned smem = bwd_smem_bytes(g.alpha);
  const void* fn = bwd_kernel_for(g.alpha, true);
  cudaError_t e = set_smem(fn, smem);
  if (e != cudaSuccess) return e;
  BwdBatchArgs a = args;
  Globals gg = g;
  const float* sc = scale;
  void* kargs[3] = {&a, &gg, &sc};
  e = cudaLaunchKernel(fn, dim3(max_tiles, n_frames), dim3(NT), kargs, smem, stream);
  return e;
}

cudaError_t launch_backward_batched_param(const FrameDesc* frames, const BwdMaps* maps, int n_frames, int max_tiles,
                                          const Globals& g, cudaStream_t stream, const float* scale) {
  if (n_frames < 1 || n_frames > kBwdParamMaxFrames) return cudaErrorInvalidValue;
  const unsigned smem = bwd_smem_bytes(g.alpha);
  const void* fn = bwd_param_kernel_for(g.alpha);
  cudaError_t e = set_smem(fn, smem);
  if (e != cudaSuccess) return e;
  std::vector<unsigned char> raw(sizeof(BwdParamBatch) + 128);
  void* aligned = raw.data() + (128 - reinterpret_cast<uintptr_t>(raw.data()) % 128) % 128;
  BwdParamBatch* pb = static_cast<BwdParamBatch*>(aligned);
  std::memset(pb, 0, sizeof(BwdParamBatch));
  std::memcpy(pb->frames, frames, sizeof(FrameDesc) * (size_t)n_frames);
  std::memcpy(pb->maps, maps, sizeof(BwdMaps) * (size_t)n_frames);
  Globals gg = g;
  const float* sc = scale;
  void* kargs[3] = {pb, &gg, &sc};
  return cudaLaunchKernel(fn, dim3(max_tiles, n_frames), dim3(NT), kargs, smem, stream);
}

}  // namespace nrm
