// Host side of the C ABI declared in include/nrm.h.
//
// Responsibilities: argument validation (nothing is launched on bad input),
// per-frame descriptors with the Eq. 4-6 constants and TMA tensor maps, the
// plain per-frame launch, the batched persistent launch replayed from a CUDA
// graph (descriptor upload node -> [event] -> kernel node -> [event]) over a
// ring of descriptor slots, the adjoint launch, kernel timing, the device
// status word and the autotuner with its JSON cache.
#include <cuda.h>
#include <cuda_runtime.h>
#include <unistd.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "nrm.h"
#include "nrm_internal.h"

using nrm::FrameDesc;
using nrm::FwdKernelSet;

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation)
    return fail(NRM_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
  if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver)
    return fail(NRM_ERR_NO_DEVICE, "%s: %s", what, cudaGetErrorString(e));
  return fail(NRM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define NRM_CUDA(call, what)                 \
  do {                                       \
    cudaError_t e_ = (call);                 \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

// Returns a nonzero status from a library routine.
#define NRM_CHECK(call)       \
  do {                        \
    int rc_ = (call);         \
    if (rc_) return rc_;      \
  } while (0)

// ------------------------------------------------ driver entry point (TMA)

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  // Looked up once (thread-safe static initialisation).
  static const EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<EncodeTiledFn>(p);
    return static_cast<EncodeTiledFn>(nullptr);
  }();
  return fn;
}

// cuTensorMapEncodeTiled for a rank-2 or rank-3 map with unit element
// strides, no interleave or swizzle, 256-byte L2 promotion and zero fill.
bool encode_tiled(CUtensorMap* m, CUtensorMapDataType dtype, int rank, const void* base, const cuuint64_t* dims,
                  const cuuint64_t* strides, const cuuint32_t* box) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint32_t es[3] = {1, 1, 1};
  return fn(m, dtype, (cuuint32_t)rank, const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

// Encodes a 2-D tiled map of a depth image with box (box_w x box_h) elements,
// zero fill outside the image. Returns false if the map cannot be made.
bool encode_depth_map(CUtensorMap* m, const void* base, int in_dtype, int W, int H, long long pitch,
                      int box_w, int box_h) {
  const int eb = in_dtype == NRM_IN_U16_MM ? 2 : 4;
  const cuuint64_t dims[2] = {(cuuint64_t)W, (cuuint64_t)H};
  const cuuint64_t strides[1] = {(cuuint64_t)pitch * (cuuint64_t)eb};
  const cuuint32_t box[2] = {(cuuint32_t)box_w, (cuuint32_t)box_h};
  return encode_tiled(m, in_dtype == NRM_IN_U16_MM ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                      2, base, dims, strides, box);
}

// Upstream gradient of the adjoint (float4 per pixel) as a 2-D tensor of
// 8-byte elements (two per pixel): box (2 box_w, box_h) lands in shared memory
// as float4 per pixel, each box row one contiguous run of 16 box_w bytes (a
// 3-D float32 view with the 4 components innermost would move 16-byte rows).
bool encode_grad_map(CUtensorMap* m, const void* base, int W, int H, long long out_pitch, int box_w,
                     int box_h) {
  if ((uintptr_t)base % 16) return false;
  const cuuint64_t dims[2] = {2 * (cuuint64_t)W, (cuuint64_t)H};
  const cuuint64_t strides[1] = {(cuuint64_t)out_pitch * 16};
  const cuuint32_t box[2] = {2 * (cuuint32_t)box_w, (cuuint32_t)box_h};
  return encode_tiled(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, base, dims, strides, box);
}

// The mask (one byte per pixel, pitch out_pitch) as a 2-D uint8 tensor.
bool encode_mask_map(CUtensorMap* m, const void* base, int W, int H, long long out_pitch, int box_w, int box_h) {
  if ((uintptr_t)base % 16 || out_pitch % 16) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)W, (cuuint64_t)H};
  const cuuint64_t strides[1] = {(cuuint64_t)out_pitch};
  const cuuint32_t box[2] = {(cuuint32_t)box_w, (cuuint32_t)box_h};
  return encode_tiled(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, base, dims, strides, box);
}

bool finite_positive(double v) { return std::isfinite(v) && v > 0.0; }

int pow2_align(uintptr_t v, int cap) {
  int a = 1;
  while (a < cap && (v % (uintptr_t)(2 * a)) == 0) a *= 2;
  return a;
}

// Fills everything of a FrameDesc except tile_begin. box_* are the halo box
// for the kernel that will read it. Returns NRM_OK or an error (message set).
int make_desc(FrameDesc* d, const void* depth, void* normals, uint8_t* valid, int H, int W,
              long long depth_pitch, long long out_pitch, const nrm_intrinsics& K, int in_dtype,
              const nrm_params& p, int tile_x, int tile_y, int box_w, int box_h, float* points = nullptr) {
  std::memset(d, 0, sizeof(*d));
  d->depth = depth;
  d->normals = normals;
  d->valid = valid;
  d->H = H;
  d->W = W;
  d->depth_pitch = depth_pitch;
  d->out_pitch = out_pitch;
  d->tiles_x = W > 0 ? (W + tile_x - 1) / tile_x : 0;
  const double s = in_dtype == NRM_IN_U16_MM ? (double)p.depth_scale : 1.0;
  const double al = (double)p.alpha;
  d->a = (float)(al / (4.0 * K.fy) * s * s);
  d->b = (float)(al / (4.0 * K.fx) * s * s);
  d->c = (float)(al * al / (4.0 * K.fx * K.fy) * s * s);
  d->inv_fx = (float)(1.0 / K.fx);
  d->inv_fy = (float)(1.0 / K.fy);
  d->cx = (float)K.cx;
  d->cy = (float)K.cy;
  d->in_dtype = in_dtype;
  d->points = points;
  d->point_scale = (float)s;
  d->mask_align = valid ? std::min(pow2_align((uintptr_t)valid, 16), pow2_align((uintptr_t)out_pitch, 16)) : 1;
  const long long bpp = p.out_dtype == NRM_OUT_F32X4 ? 16 : (p.out_dtype == NRM_OUT_F16X4 ? 8 : 4);
  d->out_align = normals ? std::min(pow2_align((uintptr_t)normals, 16), pow2_align((uintptr_t)(out_pitch * bpp), 16)) : 1;
  const int eb = in_dtype == NRM_IN_U16_MM ? 2 : 4;
  const bool aligned = ((uintptr_t)depth % 16 == 0) && ((depth_pitch * eb) % 16 == 0) &&
                       (depth_pitch * eb) < (1LL << 40) && H > 0 && W > 0;
  d->use_tma = 0;
  if (aligned && encode_depth_map(&d->tmap, depth, in_dtype, W, H, depth_pitch, box_w, box_h)) d->use_tma = 1;
  (void)tile_y;
  return NRM_OK;
}

// Descriptor and tensor maps of one adjoint frame (float32 depth). use_tma is
// set only when the depth, gradient and mask maps can all be made.
void make_bwd_desc(FrameDesc* d, nrm::BwdMaps* maps, const float* depth, const float* grad_normals,
                   const uint8_t* valid, float* grad_depth, int H, int W, long long depth_pitch,
                   long long out_pitch, const nrm_intrinsics& K, const nrm_params& p) {
  const int TX = nrm::kBwdTileX, TY = nrm::kBwdTileY, a = p.alpha;
  make_desc(d, depth, const_cast<float*>(grad_normals), const_cast<uint8_t*>(valid), H, W, depth_pitch, out_pitch,
            K, NRM_IN_F32_M, p, TX, TY, TX + 2 * nrm::pad_x(2 * a, 4), TY + 4 * a);
  d->grad_depth = grad_depth;
  std::memset(maps, 0, sizeof(*maps));
  if (d->use_tma) {
    const bool ok = encode_grad_map(&maps->grad, grad_normals, W, H, out_pitch, TX + 2 * a, TY + 2 * a) &&
                    encode_mask_map(&maps->mask, valid, W, H, out_pitch, nrm::kBwdMaskBoxW, TY + 2 * a);
    if (!ok) d->use_tma = 0;
  }
}

int validate_params(const nrm_params& p) {
  if (p.alpha < 1 || p.alpha > NRM_MAX_ALPHA)
    return fail(NRM_ERR_UNSUPPORTED, "alpha %d outside 1..%d", p.alpha, NRM_MAX_ALPHA);
  if (p.mask_mode != NRM_MASK_RAW && p.mask_mode != NRM_MASK_SECANT)
    return fail(NRM_ERR_INVALID_ARG, "mask_mode %d", p.mask_mode);
  if (!(p.tau >= 0.0f)) return fail(NRM_ERR_INVALID_ARG, "tau must be >= 0 (got %g)", (double)p.tau);
  if (!(p.depth_scale > 0.0f) || !std::isfinite(p.depth_scale))
    return fail(NRM_ERR_INVALID_ARG, "depth_scale must be positive and finite");
  if (p.in_dtype != NRM_IN_F32_M && p.in_dtype != NRM_IN_U16_MM)
    return fail(NRM_ERR_INVALID_ARG, "in_dtype %d", p.in_dtype);
  if (p.out_dtype != NRM_OUT_F32X4 && p.out_dtype != NRM_OUT_F16X4 && p.out_dtype != NRM_OUT_OCT16)
    return fail(NRM_ERR_INVALID_ARG, "out_dtype %d", p.out_dtype);
  if (p.orient_to_camera != 0 && p.orient_to_camera != 1)
    return fail(NRM_ERR_INVALID_ARG, "orient_to_camera must be 0 or 1");
  return NRM_OK;
}

int validate_intrinsics(const nrm_intrinsics& K) {
  if (!finite_positive(K.fx) || !finite_positive(K.fy) || !std::isfinite(K.cx) || !std::isfinite(K.cy))
    return fail(NRM_ERR_INVALID_ARG, "intrinsics must be finite with positive fx, fy");
  return NRM_OK;
}

constexpr int kSlots = 3;
constexpr unsigned long long kDefaultTimeoutNs = 2000000000ull;  // 2 s

struct Slot {
  void* host = nullptr;       // pinned staging of the descriptor block
  void* dev = nullptr;        // device descriptor block
  int capacity = 0;           // frames
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t copy_node = nullptr;
  cudaEvent_t ev_start = nullptr, ev_end = nullptr, done = nullptr;
  bool graph_timed = false;
  bool graph_points = false;  // the graph's kernel also writes point clouds
  bool graph_u16 = false;     // the graph's staging buffers are sized for uint16 frames only
  bool in_flight = false;
  bool timed_launch = false;
  int tiles = 0;
};

// Descriptor ring slot of the batched adjoint (no graph: one plain launch).
struct BSlot {
  void* host = nullptr;
  void* dev = nullptr;
  int capacity = 0;
  cudaEvent_t done = nullptr;
  bool in_flight = false;
};

// One internal stream of the host-buffer pipeline and its device staging.
struct HostLane {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;  // after the lane's last operation of a call
  void* dev = nullptr;         // staging of one chunk: depth, normals, mask, points
  size_t bytes = 0;
};
constexpr int kLanes = 2;

}  // namespace

struct nrm_handle {
  int device = 0;
  int sm_count = 0;
  char gpu_name[256] = {0};
  int H = 0, W = 0;
  nrm_intrinsics K = {1, 1, 0, 0};
  nrm_params p;
  nrm_tile_config cfg = {128, 16, 256, 3, 0};
  const FwdKernelSet* ks = nullptr;
  // Persistent grids [u16]: u16 = 1 for batches of uint16 frames only, whose
  // smaller staging buffers let more CTAs share an SM.
  int persistent_grid[2] = {0, 0};
  const void* pts_plain = nullptr;       // the configuration's kernels that also write
  const void* pts_persistent = nullptr;  // point clouds (out dtype of p)
  int persistent_grid_pts[2] = {0, 0};
  const void* param_persistent = nullptr;  // capture-safe kernel (descriptors as a parameter)
  int persistent_grid_param[2] = {0, 0};
  int* d_status = nullptr;
  unsigned long long timeout_ns = kDefaultTimeoutNs;
  Slot slots[kSlots];
  int next_slot = 0;
  BSlot bslots[kSlots];
  int next_bslot = 0;
  bool timing = false;
  nrm_stats stats = {0, 0.0, 0};
  cudaEvent_t last_single = nullptr;  // after the latest plain / backward launch
  double* d_mse_partials = nullptr;   // nrm_angle_mse scratch (3 kMseBlocks doubles)
  unsigned* d_loss_counters = nullptr; // nrm_cosine_loss_scale: 2 x loss_cap zeroed words
  int loss_cap = 0;
  std::vector<nrm::LossCountFrame> scratch_loss;
  HostLane lanes[kLanes];             // nrm_estimate_batched_host pipeline
  cudaEvent_t host_start = nullptr;
  std::vector<FrameDesc> scratch_desc;
  std::vector<int> scratch_tb;               // tile_begin of a parameter-block launch
  std::vector<unsigned char> scratch_param;  // its packed parameter block (+128 for alignment)
};

namespace {

nrm::Globals make_globals(const nrm_handle* h) {
  nrm::Globals g;
  g.alpha = h->p.alpha;
  g.mask_mode = h->p.mask_mode;
  g.tau2 = std::isinf(h->p.tau) ? INFINITY : h->p.tau * h->p.tau;
  g.sign = h->p.orient_to_camera ? -1.0f : 1.0f;
  g.status = h->d_status;
  g.timeout_ns = h->timeout_ns;
  return g;
}

// Records the handle's "latest single launch" event on st, which
// nrm_sync_status waits for; skipped while st is being captured (a captured
// record belongs to the graph, not to this stream's timeline).
int mark_single(nrm_handle* h, cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  NRM_CUDA(cudaStreamIsCapturing(st, &cs), "cudaStreamIsCapturing");
  if (cs == cudaStreamCaptureStatusNone) NRM_CUDA(cudaEventRecord(h->last_single, st), "cudaEventRecord");
  return NRM_OK;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

int set_smem_attr(const void* fn, unsigned bytes) {
  // Per (kernel, device) maximum already granted.
  static std::map<std::pair<const void*, int>, unsigned> granted;
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  int dev = 0;
  cudaGetDevice(&dev);
  auto key = std::make_pair(fn, dev);
  auto it = granted.find(key);
  if (it != granted.end() && it->second >= bytes) return NRM_OK;
  NRM_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes),
           "cudaFuncSetAttribute");
  granted[key] = bytes;
  return NRM_OK;
}

void destroy_slot_graph(Slot& s) {
  if (s.exec) cudaGraphExecDestroy(s.exec);
  if (s.graph) cudaGraphDestroy(s.graph);
  s.exec = nullptr;
  s.graph = nullptr;
  s.copy_node = nullptr;
}

// Waits for a slot's previous launch and folds its kernel time into the stats.
int retire_slot(nrm_handle* h, Slot& s) {
  if (!s.in_flight) return NRM_OK;
  NRM_CUDA(cudaEventSynchronize(s.done), "cudaEventSynchronize");
  if (s.timed_launch) {
    float ms = 0.0f;
    NRM_CUDA(cudaEventElapsedTime(&ms, s.ev_start, s.ev_end), "cudaEventElapsedTime");
    h->stats.launches += 1;
    h->stats.kernel_ms += ms;
    h->stats.tiles += s.tiles;
  }
  s.in_flight = false;
  return NRM_OK;
}

int retire_all(nrm_handle* h) {
  for (auto& s : h->slots) {
    int rc = retire_slot(h, s);
    if (rc) return rc;
  }
  for (auto& b : h->bslots) {
    if (b.in_flight) NRM_CUDA(cudaEventSynchronize(b.done), "cudaEventSynchronize");
    b.in_flight = false;
  }
  if (h->last_single) NRM_CUDA(cudaEventSynchronize(h->last_single), "cudaEventSynchronize");
  return NRM_OK;
}

int configure(nrm_handle* h, const nrm_tile_config& c) {
  const FwdKernelSet* ks = nrm::fwd_kernel_find(c.tile_x, c.tile_y, c.threads);
  if (!ks) return fail(NRM_ERR_UNSUPPORTED, "no compiled kernel for tile %dx%d, %d threads", c.tile_x, c.tile_y, c.threads);
  if (c.stages < 2 || c.stages > 4) return fail(NRM_ERR_UNSUPPORTED, "stages must be 2..4");
  if (c.ctas_per_sm < 0) return fail(NRM_ERR_INVALID_ARG, "ctas_per_sm must be >= 0");
  if (c.tile_y + 2 * h->p.alpha > 256)
    return fail(NRM_ERR_UNSUPPORTED, "tile_y + 2 alpha exceeds the TMA box limit");
  const int out = h->p.out_dtype;
  const unsigned ps = nrm::persistent_smem_bytes(c.tile_x, c.tile_y, h->p.alpha, c.stages);
  const unsigned pl = nrm::plain_smem_bytes(c.tile_x, c.tile_y, h->p.alpha);
  const void* pts_pers = nrm::fwd_points_kernel(c.tile_x, c.tile_y, c.threads, out, true);
  const void* param_pers = nrm::fwd_param_kernel(c.tile_x, c.tile_y, c.threads, out);
  if (!param_pers) return fail(NRM_ERR_UNSUPPORTED, "no capture-safe kernel for this configuration");
  const void* pts_plain = nrm::fwd_points_kernel(c.tile_x, c.tile_y, c.threads, out, false);
  if (!pts_pers || !pts_plain) return fail(NRM_ERR_UNSUPPORTED, "no point-cloud kernel for this configuration");
  int rc = set_smem_attr(ks->persistent[out], ps);
  if (rc) return rc;
  rc = set_smem_attr(ks->plain[out], pl);
  if (rc) return rc;
  rc = set_smem_attr(pts_pers, ps);
  if (rc) return rc;
  rc = set_smem_attr(pts_plain, pl);
  if (rc) return rc;
  rc = set_smem_attr(param_pers, ps);
  if (rc) return rc;
  // CTAs per SM for each kernel and staging size (any dtype / uint16 only).
  int per_sm[3][2];  // [normal / points / parameter kernel][u16]
  const void* pk[3] = {ks->persistent[out], pts_pers, param_pers};
  for (int k = 0; k < 3; ++k)
    for (int u = 0; u < 2; ++u) {
      const unsigned bytes = nrm::persistent_smem_bytes(c.tile_x, c.tile_y, h->p.alpha, c.stages, u ? 2 : 0);
      int occ = 0;
      NRM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pk[k], nrm::persistent_threads(c.threads), bytes),
               "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
      if (occ < 1) return fail(NRM_ERR_UNSUPPORTED, "persistent kernel does not fit on an SM");
      per_sm[k][u] = c.ctas_per_sm > 0 ? std::min(c.ctas_per_sm, occ) : occ;
    }
  // Retire work that used the old graphs before replacing them.
  rc = retire_all(h);
  if (rc) return rc;
  for (auto& s : h->slots) destroy_slot_graph(s);
  h->cfg = c;
  h->ks = ks;
  for (int u = 0; u < 2; ++u) {
    h->persistent_grid[u] = per_sm[0][u] * h->sm_count;
    h->persistent_grid_pts[u] = per_sm[1][u] * h->sm_count;
    h->persistent_grid_param[u] = per_sm[2][u] * h->sm_count;
  }
  h->param_persistent = param_pers;
  h->pts_plain = pts_plain;
  h->pts_persistent = pts_pers;
  return NRM_OK;
}

// (Re)builds a slot's graph: upload node -> [ev_start] -> kernel -> [ev_end];
// with points, the kernel variant that also writes point clouds; with u16,
// staging buffers sized for uint16 frames (and the larger grid that allows).
int build_slot_graph(nrm_handle* h, Slot& s, bool points, bool u16) {
  destroy_slot_graph(s);
  NRM_CUDA(cudaGraphCreate(&s.graph, 0), "cudaGraphCreate");
  NRM_CUDA(cudaGraphAddMemcpyNode1D(&s.copy_node, s.graph, nullptr, 0, s.dev, s.host,
                                    nrm::block_bytes(s.capacity), cudaMemcpyHostToDevice),
           "cudaGraphAddMemcpyNode1D");
  cudaGraphNode_t prev = s.copy_node;
  if (h->timing) {
    cudaGraphNode_t e;
    NRM_CUDA(cudaGraphAddEventRecordNode(&e, s.graph, &prev, 1, s.ev_start), "cudaGraphAddEventRecordNode");
    prev = e;
  }
  nrm::BatchArgs args;
  args.hdr = reinterpret_cast<const nrm::BatchHeader*>(s.dev);
  args.tile_begin = reinterpret_cast<const int*>(static_cast<char*>(s.dev) + nrm::kTileBeginOffset);
  args.frames = reinterpret_cast<const FrameDesc*>(static_cast<char*>(s.dev) + nrm::frames_offset(s.capacity));
  args.stages = h->cfg.stages;
  args.stage_bytes = nrm::stage_bytes_for(h->cfg.tile_x, h->cfg.tile_y, h->p.alpha, u16 ? 2 : 0);
  nrm::Globals g = make_globals(h);
  void* kargs[2] = {&args, &g};
  cudaKernelNodeParams kp;
  std::memset(&kp, 0, sizeof(kp));
  kp.func = const_cast<void*>(points ? h->pts_persistent : h->ks->persistent[h->p.out_dtype]);
  kp.gridDim = dim3(points ? h->persistent_grid_pts[u16] : h->persistent_grid[u16]);
  kp.blockDim = dim3(nrm::persistent_threads(h->cfg.threads));
  kp.sharedMemBytes = nrm::persistent_smem_bytes(h->cfg.tile_x, h->cfg.tile_y, h->p.alpha, h->cfg.stages, u16 ? 2 : 0);
  kp.kernelParams = kargs;
  cudaGraphNode_t kn;
  NRM_CUDA(cudaGraphAddKernelNode(&kn, s.graph, &prev, 1, &kp), "cudaGraphAddKernelNode");
  if (h->timing) {
    cudaGraphNode_t e;
    NRM_CUDA(cudaGraphAddEventRecordNode(&e, s.graph, &kn, 1, s.ev_end), "cudaGraphAddEventRecordNode");
  }
  NRM_CUDA(cudaGraphInstantiate(&s.exec, s.graph, 0), "cudaGraphInstantiate");
  s.graph_timed = h->timing;
  s.graph_points = points;
  s.graph_u16 = u16;
  return NRM_OK;
}

int ensure_slot_capacity(nrm_handle* h, Slot& s, int n) {
  if (s.capacity >= n && s.host && s.dev) return NRM_OK;
  int cap = std::max(64, s.capacity);
  while (cap < n) cap *= 2;
  destroy_slot_graph(s);
  if (s.host) cudaFreeHost(s.host);
  if (s.dev) cudaFree(s.dev);
  s.host = s.dev = nullptr;
  s.capacity = 0;
  const size_t bytes = nrm::block_bytes(cap);
  NRM_CUDA(cudaHostAlloc(&s.host, bytes, cudaHostAllocDefault), "cudaHostAlloc");
  NRM_CUDA(cudaMalloc(&s.dev, bytes), "cudaMalloc");
  std::memset(s.host, 0, bytes);
  s.capacity = cap;
  (void)h;
  return NRM_OK;
}

int validate_frame(const nrm_frame& f, int i, int out_dtype) {
  if (f.H < 0 || f.W < 0) return fail(NRM_ERR_INVALID_ARG, "frame %d: negative size", i);
  if ((long long)f.H * f.W == 0) return NRM_OK;
  if (!f.depth || !f.normals || !f.valid) return fail(NRM_ERR_INVALID_ARG, "frame %d: NULL buffer", i);
  if (f.depth_pitch < f.W || f.out_pitch < f.W) return fail(NRM_ERR_INVALID_ARG, "frame %d: pitch < W", i);
  if (f.in_dtype != NRM_IN_F32_M && f.in_dtype != NRM_IN_U16_MM)
    return fail(NRM_ERR_INVALID_ARG, "frame %d: in_dtype %d", i, f.in_dtype);
  const uintptr_t na = out_dtype == NRM_OUT_F32X4 ? 16 : (out_dtype == NRM_OUT_F16X4 ? 8 : 4);
  if ((uintptr_t)f.normals % na) return fail(NRM_ERR_INVALID_ARG, "frame %d: normals not %d-byte aligned", i, (int)na);
  const int eb = f.in_dtype == NRM_IN_U16_MM ? 2 : 4;
  if ((uintptr_t)f.depth % eb) return fail(NRM_ERR_INVALID_ARG, "frame %d: depth not %d-byte aligned", i, eb);
  if ((uintptr_t)f.points % 16) return fail(NRM_ERR_INVALID_ARG, "frame %d: points not 16-byte aligned", i);
  if (f.H > (1 << 24) || f.W > (1 << 24)) return fail(NRM_ERR_UNSUPPORTED, "frame %d: dimension above 2^24", i);
  return validate_intrinsics(f.K) ? fail(NRM_ERR_INVALID_ARG, "frame %d: bad intrinsics", i) : NRM_OK;
}

// ------------------------------------------------------------- JSON cache

std::map<std::string, std::string> read_cache(const char* path) {
  std::map<std::string, std::string> m;
  std::ifstream in(path);
  if (!in) return m;
  std::stringstream ss;
  ss << in.rdbuf();
  std::string t = ss.str();
  // Flat object: "key": [tx, ty, threads, stages, ctas], ...
  size_t i = 0;
  while (true) {
    size_t k0 = t.find('"', i);
    if (k0 == std::string::npos) break;
    size_t k1 = t.find('"', k0 + 1);
    if (k1 == std::string::npos) break;
    size_t v0 = t.find('[', k1);
    size_t v1 = t.find(']', v0 == std::string::npos ? k1 : v0);
    if (v0 == std::string::npos || v1 == std::string::npos) break;
    m[t.substr(k0 + 1, k1 - k0 - 1)] = t.substr(v0 + 1, v1 - v0 - 1);
    i = v1 + 1;
  }
  return m;
}

bool write_cache(const char* path, const std::map<std::string, std::string>& m) {
  // A temporary name of this process's own, then an atomic rename: processes
  // that tune at the same time (one per GPU) never mix their writes; the
  // last rename wins.
  std::string tmp = std::string(path) + ".tmp." + std::to_string((long long)getpid());
  std::ofstream out(tmp);
  if (!out) return false;
  out << "{\n";
  size_t n = 0;
  for (const auto& kv : m) {
    out << "  \"" << kv.first << "\": [" << kv.second << "]" << (++n < m.size() ? ",\n" : "\n");
  }
  out << "}\n";
  out.close();
  if (!out) return false;
  return std::rename(tmp.c_str(), path) == 0;
}

std::string tune_key(const nrm_handle* h, const nrm_frame* f, int n) {
  long long px = 0;
  int maxw = 0, dtypes = 0;
  for (int i = 0; i < n; ++i) {
    px += (long long)f[i].H * f[i].W;
    maxw = std::max(maxw, f[i].W);
    dtypes |= 1 << f[i].in_dtype;
  }
  int lpx = 0;
  while ((1LL << (lpx + 1)) <= px) ++lpx;
  int lw = 0;
  while ((1 << (lw + 1)) <= maxw) ++lw;
  std::string name = h->gpu_name;
  for (auto& ch : name)
    if (ch == '"' || ch == '\\') ch = '_';
  std::ostringstream k;
  k << name << "|sm" << h->sm_count << "|in" << dtypes << "|out" << h->p.out_dtype << "|a" << h->p.alpha
    << "|px2^" << lpx << "|w2^" << lw;
  return k.str();
}

// The key of a handle as created: GPU, SM count, input dtype of its params,
// output dtype, alpha and the handle's frame size (0 x 0 for batch handles).
std::string handle_key(const nrm_handle* h) {
  std::string name = h->gpu_name;
  for (auto& ch : name)
    if (ch == '"' || ch == '\\') ch = '_';
  std::ostringstream k;
  k << name << "|sm" << h->sm_count << "|in" << (1 << h->p.in_dtype) << "|out" << h->p.out_dtype << "|a"
    << h->p.alpha << "|handle" << h->H << "x" << h->W;
  return k.str();
}

std::mutex g_tune_mu;            // guards g_tune_path and the cache files this process writes
std::string g_tune_path;         // process-wide cache file ("" = none)
bool g_tune_path_set = false;    // set by nrm_set_autotune_cache (else the environment decides)

std::string tune_path(const char* explicit_path) {
  if (explicit_path) return explicit_path;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  if (g_tune_path_set) return g_tune_path;
  const char* env = std::getenv("NRM_AUTOTUNE_CACHE");
  return env ? env : "";
}

bool parse_config(const std::string& v, nrm_tile_config* c) {
  return std::sscanf(v.c_str(), "%d , %d , %d , %d , %d", &c->tile_x, &c->tile_y, &c->threads, &c->stages,
                     &c->ctas_per_sm) == 5;
}

std::string format_config(const nrm_tile_config& c) {
  char buf[128];
  std::snprintf(buf, sizeof(buf), "%d, %d, %d, %d, %d", c.tile_x, c.tile_y, c.threads, c.stages, c.ctas_per_sm);
  return buf;
}

}  // namespace

namespace nrm {

int host_fail(int code, const char* message) { return fail(code, "%s", message); }
void host_clear_error() { g_last_error.clear(); }
int host_validate_params(const nrm_params& p) { return validate_params(p); }
int host_validate_frame(const nrm_frame& f, int index, int out_dtype) { return validate_frame(f, index, out_dtype); }
void host_make_forward_desc(FrameDesc* d, const nrm_frame& f, const nrm_params& p, int tile_x, int tile_y) {
  const int eb = f.in_dtype == NRM_IN_U16_MM ? 2 : 4;
  make_desc(d, f.depth, f.normals, f.valid, f.H, f.W, f.depth_pitch, f.out_pitch, f.K, f.in_dtype, p, tile_x,
            tile_y, tile_x + 2 * pad_x(p.alpha, eb), tile_y + 2 * p.alpha, f.points);
}

}  // namespace nrm

// =================================================================== C ABI

extern "C" {

void nrm_default_params(nrm_params* p) {
  if (!p) return;
  p->alpha = 2;
  p->mask_mode = NRM_MASK_SECANT;
  p->tau = 12.0f;
  p->depth_scale = 0.001f;
  p->in_dtype = NRM_IN_F32_M;
  p->out_dtype = NRM_OUT_F32X4;
  p->orient_to_camera = 0;
}

const char* nrm_status_string(int status) {
  switch (status) {
    case NRM_OK: return "NRM_OK";
    case NRM_ERR_INVALID_ARG: return "NRM_ERR_INVALID_ARG";
    case NRM_ERR_UNSUPPORTED: return "NRM_ERR_UNSUPPORTED";
    case NRM_ERR_CUDA: return "NRM_ERR_CUDA";
    case NRM_ERR_OOM: return "NRM_ERR_OOM";
    case NRM_ERR_TIMEOUT: return "NRM_ERR_TIMEOUT";
    case NRM_ERR_NO_DEVICE: return "NRM_ERR_NO_DEVICE";
    case NRM_ERR_BOUNDS: return "NRM_ERR_BOUNDS";
    default: return "NRM_ERR_UNKNOWN";
  }
}

const char* nrm_last_error(void) { return g_last_error.c_str(); }

const char* nrm_version(void) { return "nrm 0.1 (sm_103a)"; }

int nrm_create(const nrm_intrinsics* K, int H, int W, const nrm_params* p, nrm_handle** out) {
  g_last_error.clear();
  if (!out) return fail(NRM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  nrm_params params;
  nrm_default_params(&params);
  if (p) params = *p;
  int rc = validate_params(params);
  if (rc) return rc;
  if (H < 0 || W < 0) return fail(NRM_ERR_INVALID_ARG, "negative size");
  if ((H > 0) != (W > 0)) return fail(NRM_ERR_INVALID_ARG, "H and W must both be 0 or both positive");
  if (H > 0) {
    if (!K) return fail(NRM_ERR_INVALID_ARG, "K is NULL");
    rc = validate_intrinsics(*K);
    if (rc) return rc;
    if (H > (1 << 24) || W > (1 << 24)) return fail(NRM_ERR_UNSUPPORTED, "dimension above 2^24");
  }
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0) return fail(NRM_ERR_NO_DEVICE, "no CUDA device visible");
  nrm_handle* h = new nrm_handle();
  h->p = params;
  h->H = H;
  h->W = W;
  if (K) h->K = *K;
  cudaGetDevice(&h->device);
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, h->device);
  if (e != cudaSuccess) {
    delete h;
    return cuda_fail(e, "cudaGetDeviceProperties");
  }
  if (prop.major < 10) {
    delete h;
    return fail(NRM_ERR_UNSUPPORTED, "device %s is sm_%d%d; this library is built for sm_103a", prop.name,
                prop.major, prop.minor);
  }
  h->sm_count = prop.multiProcessorCount;
  std::snprintf(h->gpu_name, sizeof(h->gpu_name), "%s", prop.name);
  if ((e = cudaMalloc(&h->d_status, sizeof(int))) != cudaSuccess ||
      (e = cudaMemset(h->d_status, 0, sizeof(int))) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&h->last_single, cudaEventDisableTiming)) != cudaSuccess) {
    nrm_destroy(h);
    return cuda_fail(e, "handle allocation");
  }
  for (auto& s : h->slots) {
    if ((e = cudaEventCreate(&s.ev_start)) != cudaSuccess || (e = cudaEventCreate(&s.ev_end)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming)) != cudaSuccess) {
      nrm_destroy(h);
      return cuda_fail(e, "cudaEventCreate");
    }
  }
  for (auto& b : h->bslots) {
    if ((e = cudaEventCreateWithFlags(&b.done, cudaEventDisableTiming)) != cudaSuccess) {
      nrm_destroy(h);
      return cuda_fail(e, "cudaEventCreate");
    }
  }
  nrm_tile_config c = {128, 16, 256, 3, 0};
  rc = configure(h, c);
  if (rc) {
    std::string msg = g_last_error;
    nrm_destroy(h);
    g_last_error = msg;
    return rc;
  }
  // A tuned geometry for this handle's key from the process-wide cache file.
  const std::string path = tune_path(nullptr);
  if (!path.empty()) {
    std::map<std::string, std::string> cache;
    {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      cache = read_cache(path.c_str());
    }
    auto it = cache.find(handle_key(h));
    nrm_tile_config tuned;
    if (it != cache.end() && parse_config(it->second, &tuned) && configure(h, tuned) != NRM_OK) {
      configure(h, c);  // a stale or foreign entry: keep the default geometry
      g_last_error.clear();
    }
  }
  *out = h;
  return NRM_OK;
}

int nrm_set_autotune_cache(const char* path) {
  g_last_error.clear();
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_path = path ? path : "";
  g_tune_path_set = true;
  return NRM_OK;
}

int nrm_autotune_key(const nrm_handle* h, char* buf, int len) {
  g_last_error.clear();
  if (!h || !buf || len <= 0) return fail(NRM_ERR_INVALID_ARG, "bad arguments");
  const std::string k = handle_key(h);
  if ((int)k.size() + 1 > len) return fail(NRM_ERR_INVALID_ARG, "key needs %d bytes", (int)k.size() + 1);
  std::memcpy(buf, k.c_str(), k.size() + 1);
  return NRM_OK;
}

int nrm_autotune_cache_get(const char* path, const char* key, nrm_tile_config* cfg) {
  g_last_error.clear();
  if (!path || !key || !cfg) return fail(NRM_ERR_INVALID_ARG, "bad arguments");
  std::map<std::string, std::string> cache;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    cache = read_cache(path);
  }
  auto it = cache.find(key);
  if (it == cache.end()) return fail(NRM_ERR_INVALID_ARG, "no entry for this key in %s", path);
  nrm_tile_config c;
  if (!parse_config(it->second, &c)) return fail(NRM_ERR_INVALID_ARG, "malformed entry in %s", path);
  *cfg = c;
  return NRM_OK;
}

int nrm_autotune_cache_put(const char* path, const char* key, const nrm_tile_config* cfg) {
  g_last_error.clear();
  if (!path || !key || !cfg) return fail(NRM_ERR_INVALID_ARG, "bad arguments");
  if (std::strpbrk(key, "\"\\")) return fail(NRM_ERR_INVALID_ARG, "key contains a quote or a backslash");
  std::lock_guard<std::mutex> lock(g_tune_mu);
  std::map<std::string, std::string> cache = read_cache(path);
  cache[key] = format_config(*cfg);
  if (!write_cache(path, cache)) return fail(NRM_ERR_INVALID_ARG, "cannot write %s", path);
  return NRM_OK;
}

void nrm_destroy(nrm_handle* h) {
  if (!h) return;
  DeviceGuard guard(h->device);
  for (auto& s : h->slots) {
    if (s.in_flight && s.done) cudaEventSynchronize(s.done);
    destroy_slot_graph(s);
    if (s.host) cudaFreeHost(s.host);
    if (s.dev) cudaFree(s.dev);
    if (s.ev_start) cudaEventDestroy(s.ev_start);
    if (s.ev_end) cudaEventDestroy(s.ev_end);
    if (s.done) cudaEventDestroy(s.done);
  }
  for (auto& b : h->bslots) {
    if (b.in_flight && b.done) cudaEventSynchronize(b.done);
    if (b.host) cudaFreeHost(b.host);
    if (b.dev) cudaFree(b.dev);
    if (b.done) cudaEventDestroy(b.done);
  }
  if (h->last_single) {
    cudaEventSynchronize(h->last_single);
    cudaEventDestroy(h->last_single);
  }
  for (auto& l : h->lanes) {
    if (l.stream) cudaStreamSynchronize(l.stream);
    if (l.dev) cudaFree(l.dev);
    if (l.done) cudaEventDestroy(l.done);
    if (l.stream) cudaStreamDestroy(l.stream);
  }
  if (h->host_start) cudaEventDestroy(h->host_start);
  if (h->d_status) cudaFree(h->d_status);
  if (h->d_mse_partials) cudaFree(h->d_mse_partials);
  if (h->d_loss_counters) cudaFree(h->d_loss_counters);
  delete h;
}

static int estimate_single(nrm_handle* h, const void* depth, void* normals, uint8_t* valid, float* points,
                           void* cuda_stream) {
  g_last_error.clear();
  if (!h) return fail(NRM_ERR_INVALID_ARG, "handle is NULL");
  if (h->H == 0 || h->W == 0) return fail(NRM_ERR_INVALID_ARG, "handle was created for batched calls only");
  nrm_frame f = {};
  f.depth = depth;
  f.normals = normals;
  f.valid = valid;
  f.H = h->H;
  f.W = h->W;
  f.depth_pitch = h->W;
  f.out_pitch = h->W;
  f.K = h->K;
  f.in_dtype = h->p.in_dtype;
  f.points = points;
  int rc = validate_frame(f, 0, h->p.out_dtype);
  if (rc) return rc;
  DeviceGuard guard(h->device);
  const int TX = h->cfg.tile_x, TY = h->cfg.tile_y;
  const int eb = f.in_dtype == NRM_IN_U16_MM ? 2 : 4;
  FrameDesc d;
  make_desc(&d, depth, normals, valid, f.H, f.W, f.depth_pitch, f.out_pitch, f.K, f.in_dtype, h->p, TX, TY,
            TX + 2 * nrm::pad_x(h->p.alpha, eb), TY + 2 * h->p.alpha, points);
  nrm::Globals g = make_globals(h);
  dim3 grid((f.W + TX - 1) / TX, (f.H + TY - 1) / TY);
  // More tile rows than a launch grid holds: the frame runs as a one-frame
  // batch (the persistent kernel walks a tile list; same per-pixel code).
  if (grid.y > 65535) return nrm_estimate_batched(h, &f, 1, cuda_stream);
  void* args[2] = {&d, &g};
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  NRM_CUDA(cudaLaunchKernel(points ? h->pts_plain : h->ks->plain[h->p.out_dtype], grid, dim3(h->cfg.threads),
                            args, nrm::plain_smem_bytes(TX, TY, h->p.alpha), st),
           "launch fwd_plain_kernel");
  NRM_CHECK(mark_single(h, st));
  return NRM_OK;
}

int nrm_estimate(nrm_handle* h, const void* depth, void* normals, uint8_t* valid, void* cuda_stream) {
  return estimate_single(h, depth, normals, valid, nullptr, cuda_stream);
}

int nrm_estimate_points(nrm_handle* h, const void* depth, void* normals, uint8_t* valid, float* points,
                        void* cuda_stream) {
  if (!points) {
    g_last_error.clear();
    return fail(NRM_ERR_INVALID_ARG, "points is NULL");
  }
  return estimate_single(h, depth, normals, valid, points, cuda_stream);
}

// nrm_estimate_batched with the descriptor block as one kernel parameter
// (frame records and tensor maps in parameter space): no descriptor upload and
// no tensor-map fences. Used for batches of at most kParamMaxFrames frames
// without point buffers, and always while cuda_stream is being captured, when
// the launch is recorded as a single kernel node with no ring slot, events or
// synchronisation. Frames were validated by the caller.
static int estimate_batched_param(nrm_handle* h, const nrm_frame* frames, int n, cudaStream_t st, bool capture) {
  if (n > nrm::kParamMaxFrames)
    return fail(NRM_ERR_UNSUPPORTED, "at most %d frames per call during stream capture", nrm::kParamMaxFrames);
  const int TX = h->cfg.tile_x, TY = h->cfg.tile_y;
  std::vector<FrameDesc>& fd = h->scratch_desc;
  std::vector<int>& tb = h->scratch_tb;
  if (fd.size() < (size_t)n) fd.resize((size_t)n);
  if (tb.size() < (size_t)n + 1) tb.resize((size_t)n + 1);
  bool u16 = true;
  int acc = 0;
  for (int i = 0; i < n; ++i) {
    const nrm_frame& f = frames[i];
    if (f.points && (long long)f.H * f.W > 0)
      return fail(NRM_ERR_UNSUPPORTED, "frame %d: point clouds are not written during stream capture", i);
    u16 = u16 && (f.in_dtype == NRM_IN_U16_MM || (long long)f.H * f.W == 0);
    const int eb = f.in_dtype == NRM_IN_U16_MM ? 2 : 4;
    make_desc(&fd[i], f.depth, f.normals, f.valid, f.H, f.W, f.depth_pitch, f.out_pitch, f.K, f.in_dtype, h->p,
              TX, TY, TX + 2 * nrm::pad_x(h->p.alpha, eb), TY + 2 * h->p.alpha);
    fd[i].tile_begin = acc;
    tb[i] = acc;
    acc += fd[i].tiles_x * ((f.H + TY - 1) / TY);
  }
  tb[n] = acc;
  nrm::BatchHeader hdr;
  std::memset(&hdr, 0, sizeof(hdr));
  hdr.n_frames = n;
  hdr.total_tiles = acc;
  // The parameter block, 128-byte aligned like the records in it.
  std::vector<unsigned char>& raw = h->scratch_param;
  if (raw.size() < nrm::param_batch_bytes() + 128) raw.resize(nrm::param_batch_bytes() + 128);
  void* pb = raw.data() + (128 - reinterpret_cast<uintptr_t>(raw.data()) % 128) % 128;
  nrm::pack_param_batch(pb, hdr, tb.data(), fd.data(), n);
  nrm::BatchArgs ring;
  std::memset(&ring, 0, sizeof(ring));
  ring.stages = h->cfg.stages;
  ring.stage_bytes = nrm::stage_bytes_for(TX, TY, h->p.alpha, u16 ? 2 : 0);
  nrm::Globals g = make_globals(h);
  void* args[3] = {pb, &ring, &g};
  const unsigned smem = nrm::persistent_smem_bytes(TX, TY, h->p.alpha, h->cfg.stages, u16 ? 2 : 0);
  Slot* s = nullptr;
  if (!capture) {
    // A ring slot supplies the completion (and, with timing on, the kernel
    // time) events; its descriptor memory is not used.
    s = &h->slots[h->next_slot];
    h->next_slot = (h->next_slot + 1) % kSlots;
    NRM_CHECK(retire_slot(h, *s));
    if (h->timing) NRM_CUDA(cudaEventRecord(s->ev_start, st), "cudaEventRecord");
  }
  NRM_CUDA(cudaLaunchKernel(h->param_persistent, dim3(h->persistent_grid_param[u16]),
                            dim3(nrm::persistent_threads(h->cfg.threads)), args, smem, st),
           "launch fwd_persistent_param_kernel");
  if (s) {
    if (h->timing) NRM_CUDA(cudaEventRecord(s->ev_end, st), "cudaEventRecord");
    NRM_CUDA(cudaEventRecord(s->done, st), "cudaEventRecord");
    s->in_flight = true;
    s->timed_launch = h->timing;
    s->tiles = acc;
  }
  return NRM_OK;
}

int nrm_estimate_batched(nrm_handle* h, const nrm_frame* frames, int n, void* cuda_stream) {
  g_last_error.clear();
  if (!h) return fail(NRM_ERR_INVALID_ARG, "handle is NULL");
  if (n < 0) return fail(NRM_ERR_INVALID_ARG, "n < 0");
  if (n == 0) return NRM_OK;
  if (!frames) return fail(NRM_ERR_INVALID_ARG, "frames is NULL");
  const int TX = h->cfg.tile_x, TY = h->cfg.tile_y;
  long long total = 0;
  for (int i = 0; i < n; ++i) {
    int rc = validate_frame(frames[i], i, h->p.out_dtype);
    if (rc) return rc;
    const long long tx = (frames[i].W + TX - 1) / TX, ty = (frames[i].H + TY - 1) / TY;
    total += tx * ty;
    if (total >= (1LL << 31) - 1) return fail(NRM_ERR_UNSUPPORTED, "batch exceeds 2^31 tiles");
  }
  if (total == 0) return NRM_OK;
  DeviceGuard guard(h->device);
  cudaStream_t st0 = static_cast<cudaStream_t>(cuda_stream);
  cudaStreamCaptureStatus capture = cudaStreamCaptureStatusNone;
  NRM_CUDA(cudaStreamIsCapturing(st0, &capture), "cudaStreamIsCapturing");
  if (capture == cudaStreamCaptureStatusActive) return estimate_batched_param(h, frames, n, st0, true);
  bool any_points = false;
  for (int i = 0; i < n; ++i) any_points = any_points || (frames[i].points && (long long)frames[i].H * frames[i].W > 0);
  if (n <= nrm::kParamMaxFrames && !any_points) return estimate_batched_param(h, frames, n, st0, false);
  Slot& s = h->slots[h->next_slot];
  h->next_slot = (h->next_slot + 1) % kSlots;
  int rc = retire_slot(h, s);
  if (rc) return rc;
  rc = ensure_slot_capacity(h, s, n);
  if (rc) return rc;
  // Fill the pinned staging block.
  char* base = static_cast<char*>(s.host);
  nrm::BatchHeader* hdr = reinterpret_cast<nrm::BatchHeader*>(base);
  int* tb = reinterpret_cast<int*>(base + nrm::kTileBeginOffset);
  FrameDesc* fd = reinterpret_cast<FrameDesc*>(base + nrm::frames_offset(s.capacity));
  int acc = 0;
  bool points = false, u16 = true;
  for (int i = 0; i < n; ++i) {
    const nrm_frame& f = frames[i];
    points = points || (f.points && (long long)f.H * f.W > 0);
    u16 = u16 && (f.in_dtype == NRM_IN_U16_MM || (long long)f.H * f.W == 0);
    const int eb = f.in_dtype == NRM_IN_U16_MM ? 2 : 4;
    make_desc(&fd[i], f.depth, f.normals, f.valid, f.H, f.W, f.depth_pitch, f.out_pitch, f.K, f.in_dtype, h->p,
              TX, TY, TX + 2 * nrm::pad_x(h->p.alpha, eb), TY + 2 * h->p.alpha, f.points);
    fd[i].tile_begin = acc;
    tb[i] = acc;
    acc += fd[i].tiles_x * ((f.H + TY - 1) / TY);
  }
  tb[n] = acc;
  hdr->n_frames = n;
  hdr->total_tiles = acc;
  if (!s.exec || s.graph_timed != h->timing || s.graph_points != points || s.graph_u16 != u16) {
    rc = build_slot_graph(h, s, points, u16);
    if (rc) return rc;
  }
  // Upload only the used part: header + tile_begin, and the used descriptors.
  const size_t used = nrm::frames_offset(s.capacity) + sizeof(FrameDesc) * (size_t)n;
  NRM_CUDA(cudaGraphExecMemcpyNodeSetParams1D(s.exec, s.copy_node, s.dev, s.host, used, cudaMemcpyHostToDevice),
           "cudaGraphExecMemcpyNodeSetParams1D");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  NRM_CUDA(cudaGraphLaunch(s.exec, st), "cudaGraphLaunch");
  NRM_CUDA(cudaEventRecord(s.done, st), "cudaEventRecord");
  s.in_flight = true;
  s.timed_launch = s.graph_timed;
  s.tiles = acc;
  return NRM_OK;
}

// ---------------------------------------------------------- host buffers

namespace {

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// Bytes of one frame's dense device staging: depth, normals, mask, points.
struct StageSizes {
  size_t depth, normals, valid, points;
  size_t total() const { return depth + normals + valid + points; }
};

StageSizes stage_sizes(const nrm_frame& f, int out_dtype) {
  const size_t px = (size_t)f.H * (size_t)f.W;
  const size_t eb = f.in_dtype == NRM_IN_U16_MM ? 2 : 4;
  const size_t ob = out_dtype == NRM_OUT_F32X4 ? 16 : (out_dtype == NRM_OUT_F16X4 ? 8 : 4);
  return {align256(px * eb), align256(px * ob), align256(px), f.points ? align256(px * 16) : 0};
}

// Row copy of a (H x row_bytes) block between pitched host memory and dense
// device memory (one cudaMemcpyAsync when the host rows are contiguous).
int copy_rows(void* dst, size_t dpitch, const void* src, size_t spitch, size_t row_bytes, int rows,
              cudaMemcpyKind kind, cudaStream_t st) {
  if (dpitch == row_bytes && spitch == row_bytes) {
    NRM_CUDA(cudaMemcpyAsync(dst, src, row_bytes * (size_t)rows, kind, st), "cudaMemcpyAsync");
  } else {
    NRM_CUDA(cudaMemcpy2DAsync(dst, dpitch, src, spitch, row_bytes, rows, kind, st), "cudaMemcpy2DAsync");
  }
  return NRM_OK;
}

}  // namespace

int nrm_estimate_batched_host(nrm_handle* h, const nrm_frame* frames, int n, void* cuda_stream) {
  g_last_error.clear();
  if (!h) return fail(NRM_ERR_INVALID_ARG, "handle is NULL");
  if (n < 0) return fail(NRM_ERR_INVALID_ARG, "n < 0");
  if (n == 0) return NRM_OK;
  if (!frames) return fail(NRM_ERR_INVALID_ARG, "frames is NULL");
  const int out = h->p.out_dtype;
  for (int i = 0; i < n; ++i) {
    const nrm_frame& f = frames[i];
    if (f.H < 0 || f.W < 0) return fail(NRM_ERR_INVALID_ARG, "frame %d: negative size", i);
    if ((long long)f.H * f.W == 0) continue;
    if (!f.depth || !f.normals || !f.valid) return fail(NRM_ERR_INVALID_ARG, "frame %d: NULL buffer", i);
    if (f.depth_pitch < f.W || f.out_pitch < f.W) return fail(NRM_ERR_INVALID_ARG, "frame %d: pitch < W", i);
    if (f.in_dtype != NRM_IN_F32_M && f.in_dtype != NRM_IN_U16_MM)
      return fail(NRM_ERR_INVALID_ARG, "frame %d: in_dtype %d", i, f.in_dtype);
    if (f.H > (1 << 24) || f.W > (1 << 24)) return fail(NRM_ERR_UNSUPPORTED, "frame %d: dimension above 2^24", i);
    if (validate_intrinsics(f.K)) return fail(NRM_ERR_INVALID_ARG, "frame %d: bad intrinsics", i);
  }
  // Chunks of consecutive frames with at least kChunkBytes of staging (or one
  // frame), alternating between the lanes: a chunk's upload and kernel overlap
  // the downloads of the chunks before it.
  constexpr size_t kChunkBytes = size_t(96) << 20;
  std::vector<std::pair<int, int>> chunks;  // [first, last)
  size_t max_chunk = 0;
  for (int i = 0; i < n;) {
    size_t bytes = 0;
    int j = i;
    while (j < n && (j == i || bytes < kChunkBytes)) {
      bytes += stage_sizes(frames[j], out).total();
      ++j;
    }
    chunks.emplace_back(i, j);
    max_chunk = std::max(max_chunk, bytes);
    i = j;
  }
  DeviceGuard guard(h->device);
  if (!h->host_start) NRM_CUDA(cudaEventCreateWithFlags(&h->host_start, cudaEventDisableTiming), "cudaEventCreate");
  for (auto& l : h->lanes) {
    if (!l.stream) NRM_CUDA(cudaStreamCreateWithFlags(&l.stream, cudaStreamNonBlocking), "cudaStreamCreate");
    if (!l.done) NRM_CUDA(cudaEventCreateWithFlags(&l.done, cudaEventDisableTiming), "cudaEventCreate");
    if (l.bytes < max_chunk) {
      NRM_CUDA(cudaStreamSynchronize(l.stream), "cudaStreamSynchronize");
      if (l.dev) cudaFree(l.dev);
      l.dev = nullptr;
      l.bytes = 0;
      NRM_CUDA(cudaMalloc(&l.dev, max_chunk), "cudaMalloc");
      l.bytes = max_chunk;
    }
  }
  cudaStream_t caller = static_cast<cudaStream_t>(cuda_stream);
  NRM_CUDA(cudaEventRecord(h->host_start, caller), "cudaEventRecord");
  for (auto& l : h->lanes) NRM_CUDA(cudaStreamWaitEvent(l.stream, h->host_start, 0), "cudaStreamWaitEvent");
  std::vector<nrm_frame> dev_frames;
  std::vector<size_t> offs;
  for (size_t c = 0; c < chunks.size(); ++c) {
    HostLane& l = h->lanes[c % kLanes];
    char* base = static_cast<char*>(l.dev);
    const int i0 = chunks[c].first, i1 = chunks[c].second;
    dev_frames.clear();
    size_t off = 0;
    for (int i = i0; i < i1; ++i) {
      const nrm_frame& f = frames[i];
      const StageSizes sz = stage_sizes(f, out);
      nrm_frame d = f;
      d.depth = base + off;
      d.normals = base + off + sz.depth;
      d.valid = reinterpret_cast<uint8_t*>(base + off + sz.depth + sz.normals);
      d.points = f.points ? reinterpret_cast<float*>(base + off + sz.depth + sz.normals + sz.valid) : nullptr;
      d.depth_pitch = f.W;
      d.out_pitch = f.W;
      if ((long long)f.H * f.W > 0) {
        const size_t eb = f.in_dtype == NRM_IN_U16_MM ? 2 : 4;
        int rc = copy_rows(const_cast<void*>(d.depth), (size_t)f.W * eb, f.depth, (size_t)f.depth_pitch * eb,
                           (size_t)f.W * eb, f.H, cudaMemcpyHostToDevice, l.stream);
        if (rc) return rc;
      }
      dev_frames.push_back(d);
      off += sz.total();
    }
    int rc = nrm_estimate_batched(h, dev_frames.data(), (int)dev_frames.size(), l.stream);
    if (rc) return rc;
    for (int i = i0; i < i1; ++i) {
      const nrm_frame& f = frames[i];
      const nrm_frame& d = dev_frames[i - i0];
      if ((long long)f.H * f.W == 0) continue;
      const size_t ob = out == NRM_OUT_F32X4 ? 16 : (out == NRM_OUT_F16X4 ? 8 : 4);
      rc = copy_rows(f.normals, (size_t)f.out_pitch * ob, d.normals, (size_t)f.W * ob, (size_t)f.W * ob, f.H,
                     cudaMemcpyDeviceToHost, l.stream);
      if (rc) return rc;
      rc = copy_rows(f.valid, (size_t)f.out_pitch, d.valid, (size_t)f.W, (size_t)f.W, f.H, cudaMemcpyDeviceToHost,
                     l.stream);
      if (rc) return rc;
      if (f.points) {
        rc = copy_rows(f.points, (size_t)f.out_pitch * 16, d.points, (size_t)f.W * 16, (size_t)f.W * 16, f.H,
                       cudaMemcpyDeviceToHost, l.stream);
        if (rc) return rc;
      }
    }
  }
  for (auto& l : h->lanes) {
    NRM_CUDA(cudaEventRecord(l.done, l.stream), "cudaEventRecord");
    NRM_CUDA(cudaStreamWaitEvent(caller, l.done, 0), "cudaStreamWaitEvent");
  }
  return NRM_OK;
}

int nrm_backward(nrm_handle* h, const void* depth, const float* grad_normals, const uint8_t* valid,
                 float* grad_depth, void* cuda_stream) {
  g_last_error.clear();
  if (!h) return fail(NRM_ERR_INVALID_ARG, "handle is NULL");
  if (h->H == 0 || h->W == 0) return fail(NRM_ERR_INVALID_ARG, "handle was created for batched calls only");
  if (h->p.in_dtype != NRM_IN_F32_M) return fail(NRM_ERR_UNSUPPORTED, "backward needs float32 depth");
  if (!depth || !grad_normals || !valid || !grad_depth) return fail(NRM_ERR_INVALID_ARG, "NULL buffer");
  if ((uintptr_t)grad_normals % 16) return fail(NRM_ERR_INVALID_ARG, "grad_normals not 16-byte aligned");
  if ((uintptr_t)depth % 4 || (uintptr_t)grad_depth % 4) return fail(NRM_ERR_INVALID_ARG, "depth not 4-byte aligned");
  DeviceGuard guard(h->device);
  FrameDesc d;
  nrm::BwdMaps maps;
  make_bwd_desc(&d, &maps, static_cast<const float*>(depth), grad_normals, valid, grad_depth, h->H, h->W, h->W,
                h->W, h->K, h->p);
  if ((h->H + nrm::kBwdTileY - 1) / nrm::kBwdTileY > 65535) {
    // More tile rows than a launch grid holds: a one-frame batched adjoint
    // (one grid row of all the frame's tiles; same per-tile code).
    nrm_grad_frame gf = {};
    gf.depth = static_cast<const float*>(depth);
    gf.grad_normals = grad_normals;
    gf.valid = valid;
    gf.grad_depth = grad_depth;
    gf.H = h->H;
    gf.W = h->W;
    gf.depth_pitch = h->W;
    gf.out_pitch = h->W;
    gf.K = h->K;
    return nrm_backward_batched(h, &gf, 1, cuda_stream);
  }
  nrm::Globals g = make_globals(h);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  NRM_CUDA(nrm::launch_backward(d, maps, g, st), "launch bwd_kernel");
  NRM_CHECK(mark_single(h, st));
  return NRM_OK;
}

static int backward_batched(nrm_handle* h, const nrm_grad_frame* frames, int n, const float* scale,
                            void* cuda_stream);

int nrm_backward_batched(nrm_handle* h, const nrm_grad_frame* frames, int n, void* cuda_stream) {
  g_last_error.clear();
  return backward_batched(h, frames, n, nullptr, cuda_stream);
}

int nrm_backward_batched_scaled(nrm_handle* h, const nrm_grad_frame* frames, int n, const float* scale,
                                void* cuda_stream) {
  g_last_error.clear();
  if (n > 0 && !scale) return fail(NRM_ERR_INVALID_ARG, "scale is NULL");
  if ((uintptr_t)scale % 4) return fail(NRM_ERR_INVALID_ARG, "scale not 4-byte aligned");
  return backward_batched(h, frames, n, scale, cuda_stream);
}

int nrm_cosine_loss_scale(nrm_handle* h, const nrm_grad_frame* frames, int n, float* scale, void* cuda_stream) {
  g_last_error.clear();
  if (!h) return fail(NRM_ERR_INVALID_ARG, "handle is NULL");
  if (n < 0) return fail(NRM_ERR_INVALID_ARG, "n < 0");
  if (n == 0) return NRM_OK;
  if (!frames || !scale) return fail(NRM_ERR_INVALID_ARG, "frames or scale is NULL");
  if ((uintptr_t)scale % 4) return fail(NRM_ERR_INVALID_ARG, "scale not 4-byte aligned");
  std::vector<nrm::LossCountFrame>& cf = h->scratch_loss;
  cf.resize((size_t)n);
  for (int i = 0; i < n; ++i) {
    const nrm_grad_frame& f = frames[i];
    if (f.H < 0 || f.W < 0) return fail(NRM_ERR_INVALID_ARG, "frame %d: negative size", i);
    const bool empty = (long long)f.H * f.W == 0;
    if (!empty && !f.valid) return fail(NRM_ERR_INVALID_ARG, "frame %d: valid is NULL", i);
    if (!empty && f.out_pitch < f.W) return fail(NRM_ERR_INVALID_ARG, "frame %d: pitch < W", i);
    cf[i] = {f.valid, empty ? 0 : f.H, empty ? 0 : f.W, f.out_pitch};
  }
  DeviceGuard guard(h->device);
  if (n > h->loss_cap) {
    if (h->d_loss_counters) {
      NRM_CUDA(cudaDeviceSynchronize(), "cudaDeviceSynchronize");  // earlier calls may still use the counters
      cudaFree(h->d_loss_counters);
      h->d_loss_counters = nullptr;
      h->loss_cap = 0;
    }
    const int cap = std::max(n, 64);
    NRM_CUDA(cudaMalloc(&h->d_loss_counters, sizeof(unsigned) * 2 * (size_t)cap), "cudaMalloc");
    NRM_CUDA(cudaMemset(h->d_loss_counters, 0, sizeof(unsigned) * 2 * (size_t)cap), "cudaMemset");
    h->loss_cap = cap;
  }
  NRM_CUDA(nrm::launch_loss_scale(cf.data(), n, h->d_loss_counters, h->d_loss_counters + h->loss_cap, scale,
                                  static_cast<cudaStream_t>(cuda_stream)),
           "launch loss_scale_kernel");
  return NRM_OK;
}

static int backward_batched(nrm_handle* h, const nrm_grad_frame* frames, int n, const float* scale,
                            void* cuda_stream) {
  if (!h) return fail(NRM_ERR_INVALID_ARG, "handle is NULL");
  if (n < 0) return fail(NRM_ERR_INVALID_ARG, "n < 0");
  if (n == 0) return NRM_OK;
  if (!frames) return fail(NRM_ERR_INVALID_ARG, "frames is NULL");
  if (n > 65535) return fail(NRM_ERR_UNSUPPORTED, "at most 65535 frames per batched adjoint");
  const int TX = nrm::kBwdTileX, TY = nrm::kBwdTileY;
  long long total = 0;
  for (int i = 0; i < n; ++i) {
    const nrm_grad_frame& f = frames[i];
    if (f.H < 0 || f.W < 0) return fail(NRM_ERR_INVALID_ARG, "frame %d: negative size", i);
    if ((long long)f.H * f.W == 0) continue;
    if (!f.depth || !f.grad_normals || !f.valid || !f.grad_depth)
      return fail(NRM_ERR_INVALID_ARG, "frame %d: NULL buffer", i);
    if (f.depth_pitch < f.W || f.out_pitch < f.W) return fail(NRM_ERR_INVALID_ARG, "frame %d: pitch < W", i);
    if ((uintptr_t)f.grad_normals % 16) return fail(NRM_ERR_INVALID_ARG, "frame %d: grad_normals not 16-byte aligned", i);
    if ((uintptr_t)f.depth % 4 || (uintptr_t)f.grad_depth % 4)
      return fail(NRM_ERR_INVALID_ARG, "frame %d: depth buffers not 4-byte aligned", i);
    if (f.H > (1 << 24) || f.W > (1 << 24)) return fail(NRM_ERR_UNSUPPORTED, "frame %d: dimension above 2^24", i);
    if (validate_intrinsics(f.K)) return fail(NRM_ERR_INVALID_ARG, "frame %d: bad intrinsics", i);
    total += (long long)((f.W + TX - 1) / TX) * ((f.H + TY - 1) / TY);
    if (total >= (1LL << 31) - 1) return fail(NRM_ERR_UNSUPPORTED, "batch exceeds 2^31 tiles");
  }
  if (total == 0) return NRM_OK;
  DeviceGuard guard(h->device);
  if (n > nrm::kBwdParamMaxFrames) {
    // The descriptor ring is uploaded from host memory that later calls reuse:
    // a captured upload would replay stale or freed host memory.
    cudaStreamCaptureStatus capture = cudaStreamCaptureStatusNone;
    NRM_CUDA(cudaStreamIsCapturing(static_cast<cudaStream_t>(cuda_stream), &capture), "cudaStreamIsCapturing");
    if (capture == cudaStreamCaptureStatusActive)
      return fail(NRM_ERR_UNSUPPORTED, "at most %d frames per batched adjoint during stream capture",
                  nrm::kBwdParamMaxFrames);
  }
  if (n <= nrm::kBwdParamMaxFrames) {
    // Small batches: records and tensor maps as one kernel parameter (no
    // upload, no ring slot, no tensor-map fences; also capture-safe).
    std::vector<FrameDesc> fdv((size_t)n);
    std::vector<nrm::BwdMaps> mapv((size_t)n);
    int max_tiles = 0;
    for (int i = 0; i < n; ++i) {
      const nrm_grad_frame& f = frames[i];
      make_bwd_desc(&fdv[i], &mapv[i], f.depth, f.grad_normals, f.valid, f.grad_depth, f.H, f.W, f.depth_pitch,
                    f.out_pitch, f.K, h->p);
      max_tiles = std::max(max_tiles, fdv[i].tiles_x * ((f.H + TY - 1) / TY));
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    NRM_CUDA(nrm::launch_backward_batched_param(fdv.data(), mapv.data(), n, max_tiles, make_globals(h), st, scale),
             "launch bwd_batched_param_kernel");
    NRM_CHECK(mark_single(h, st));
    return NRM_OK;
  }
  BSlot& s = h->bslots[h->next_bslot];
  h->next_bslot = (h->next_bslot + 1) % kSlots;
  if (s.in_flight) {
    NRM_CUDA(cudaEventSynchronize(s.done), "cudaEventSynchronize");
    s.in_flight = false;
  }
  if (s.capacity < n || !s.host || !s.dev) {
    int cap = std::max(64, s.capacity);
    while (cap < n) cap *= 2;
    if (s.host) cudaFreeHost(s.host);
    if (s.dev) cudaFree(s.dev);
    s.host = s.dev = nullptr;
    s.capacity = 0;
    NRM_CUDA(cudaHostAlloc(&s.host, nrm::bwd_block_bytes(cap), cudaHostAllocDefault), "cudaHostAlloc");
    NRM_CUDA(cudaMalloc(&s.dev, nrm::bwd_block_bytes(cap)), "cudaMalloc");
    s.capacity = cap;
  }
  char* base = static_cast<char*>(s.host);
  std::memset(base, 0, nrm::frames_offset(s.capacity));
  nrm::BatchHeader* hdr = reinterpret_cast<nrm::BatchHeader*>(base);
  int* tb = reinterpret_cast<int*>(base + nrm::kTileBeginOffset);
  FrameDesc* fd = reinterpret_cast<FrameDesc*>(base + nrm::frames_offset(s.capacity));
  nrm::BwdMaps* maps = reinterpret_cast<nrm::BwdMaps*>(base + nrm::bwd_maps_offset(s.capacity));
  int acc = 0;
  for (int i = 0; i < n; ++i) {
    const nrm_grad_frame& f = frames[i];
    make_bwd_desc(&fd[i], &maps[i], f.depth, f.grad_normals, f.valid, f.grad_depth, f.H, f.W, f.depth_pitch,
                  f.out_pitch, f.K, h->p);
    fd[i].tile_begin = acc;
    tb[i] = acc;
    acc += fd[i].tiles_x * ((f.H + TY - 1) / TY);
  }
  tb[n] = acc;
  hdr->n_frames = n;
  hdr->total_tiles = acc;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const size_t used = nrm::bwd_maps_offset(s.capacity) + sizeof(nrm::BwdMaps) * (size_t)n;
  NRM_CUDA(cudaMemcpyAsync(s.dev, s.host, used, cudaMemcpyHostToDevice, st), "cudaMemcpyAsync");
  nrm::BwdBatchArgs args;
  char* dbase = static_cast<char*>(s.dev);
  args.hdr = reinterpret_cast<const nrm::BatchHeader*>(dbase);
  args.tile_begin = reinterpret_cast<const int*>(dbase + nrm::kTileBeginOffset);
  args.frames = reinterpret_cast<const FrameDesc*>(dbase + nrm::frames_offset(s.capacity));
  args.maps = reinterpret_cast<const nrm::BwdMaps*>(dbase + nrm::bwd_maps_offset(s.capacity));
  nrm::Globals g = make_globals(h);
  int max_tiles = 0;
  for (int i = 0; i < n; ++i) max_tiles = std::max(max_tiles, fd[i].tiles_x * ((frames[i].H + TY - 1) / TY));
  NRM_CUDA(nrm::launch_backward_batched(args, n, max_tiles, g, st, scale), "launch bwd_batched_kernel");
  NRM_CUDA(cudaEventRecord(s.done, st), "cudaEventRecord");
  s.in_flight = true;
  return NRM_OK;
}

static int check_eval_args(const float* n, const uint8_t* v, int H, int W, long long pitch) {
  if (H < 0 || W < 0) return fail(NRM_ERR_INVALID_ARG, "negative size");
  if ((long long)H * W == 0) return NRM_OK;
  if (!n || !v) return fail(NRM_ERR_INVALID_ARG, "NULL buffer");
  if (pitch < W) return fail(NRM_ERR_INVALID_ARG, "pitch < W");
  if ((uintptr_t)n % 16) return fail(NRM_ERR_INVALID_ARG, "normals not 16-byte aligned");
  return NRM_OK;
}

int nrm_spherical(const float* normals, const uint8_t* valid, int H, int W, long long pitch, float* phi,
                  float* theta, void* cuda_stream) {
  g_last_error.clear();
  int rc = check_eval_args(normals, valid, H, W, pitch);
  if (rc) return rc;
  if ((long long)H * W == 0) return NRM_OK;
  if (!phi || !theta) return fail(NRM_ERR_INVALID_ARG, "NULL output");
  if ((uintptr_t)phi % 4 || (uintptr_t)theta % 4) return fail(NRM_ERR_INVALID_ARG, "outputs not 4-byte aligned");
  NRM_CUDA(nrm::launch_spherical(normals, valid, H, W, pitch, phi, theta, static_cast<cudaStream_t>(cuda_stream)),
           "launch spherical_kernel");
  return NRM_OK;
}

int nrm_angle_mse(nrm_handle* h, const float* normals, const uint8_t* valid, const float* ref_normals,
                  const uint8_t* ref_valid, int H, int W, long long pitch, double* out, void* cuda_stream) {
  g_last_error.clear();
  if (!h) return fail(NRM_ERR_INVALID_ARG, "handle is NULL");
  if (!out || (uintptr_t)out % 8) return fail(NRM_ERR_INVALID_ARG, "out must be 8-byte aligned device memory");
  int rc = check_eval_args(normals, valid, H, W, pitch);
  if (rc) return rc;
  rc = check_eval_args(ref_normals, ref_valid, H, W, pitch);
  if (rc) return rc;
  DeviceGuard guard(h->device);
  if (!h->d_mse_partials)
    NRM_CUDA(cudaMalloc(&h->d_mse_partials, sizeof(double) * 3 * nrm::kMseBlocks), "cudaMalloc");
  NRM_CUDA(nrm::launch_angle_mse(normals, valid, ref_normals, ref_valid, H, W, pitch, h->d_mse_partials, out,
                                 static_cast<cudaStream_t>(cuda_stream)),
           "launch mse kernels");
  NRM_CHECK(mark_single(h, static_cast<cudaStream_t>(cuda_stream)));
  return NRM_OK;
}

// Checks a scale set and fills ms.K, ms.alpha and ms.alpha_max.
static int make_scales(const nrm_scales* scales, nrm::MsConsts& ms) {
  if (!scales) return fail(NRM_ERR_INVALID_ARG, "scales is NULL");
  const int K = scales->n_scales;
  if (K < 1 || K > NRM_MAX_SCALES) return fail(NRM_ERR_UNSUPPORTED, "n_scales %d outside 1..%d", K, NRM_MAX_SCALES);
  if (scales->form != NRM_MS_PAIR && scales->form != NRM_MS_QUAD)
    return fail(NRM_ERR_INVALID_ARG, "form %d", scales->form);
  std::memset(&ms, 0, sizeof(ms));
  ms.K = K;
  for (int i = 0; i < K; ++i) {
    const int a = scales->alpha[i];
    if (a < 1 || a > NRM_MAX_ALPHA) return fail(NRM_ERR_UNSUPPORTED, "alpha[%d] = %d outside 1..%d", i, a, NRM_MAX_ALPHA);
    ms.alpha[i] = a;
    ms.alpha_max = std::max(ms.alpha_max, a);
  }
  return NRM_OK;
}

int nrm_estimate_batched_multiscale(nrm_handle* h, const nrm_frame* frames, int n, const nrm_scales* scales,
                                    void* cuda_stream) {
  g_last_error.clear();
  if (!h) return fail(NRM_ERR_INVALID_ARG, "handle is NULL");
  if (n < 0) return fail(NRM_ERR_INVALID_ARG, "n < 0");
  nrm::MsConsts ms;
  int rc = make_scales(scales, ms);
  if (rc) return rc;
  if (n == 0) return NRM_OK;
  if (!frames) return fail(NRM_ERR_INVALID_ARG, "frames is NULL");
  const int TX = nrm::kMsTileX, TY = nrm::kMsTileY;
  long long total = 0;
  bool u16 = true;
  for (int i = 0; i < n; ++i) {
    rc = validate_frame(frames[i], i, h->p.out_dtype);
    if (rc) return rc;
    if (frames[i].points) return fail(NRM_ERR_UNSUPPORTED, "frame %d: the multi-scale variant writes no point clouds", i);
    total += (long long)((frames[i].W + TX - 1) / TX) * ((frames[i].H + TY - 1) / TY);
    if (total >= (1LL << 31) - 1) return fail(NRM_ERR_UNSUPPORTED, "batch exceeds 2^31 tiles");
    u16 = u16 && (frames[i].in_dtype == NRM_IN_U16_MM || (long long)frames[i].H * frames[i].W == 0);
  }
  if (total == 0) return NRM_OK;
  DeviceGuard guard(h->device);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  cudaStreamCaptureStatus capture = cudaStreamCaptureStatusNone;
  NRM_CUDA(cudaStreamIsCapturing(st, &capture), "cudaStreamIsCapturing");
  const bool captured = capture == cudaStreamCaptureStatusActive;
  // Up to kParamMaxFrames frames (and always during capture) the descriptor
  // block is one kernel parameter; larger batches upload it into a ring slot.
  const bool param = n <= nrm::kParamMaxFrames;
  if (captured && !param)
    return fail(NRM_ERR_UNSUPPORTED, "at most %d frames per call during stream capture", nrm::kParamMaxFrames);
  Slot* sp = nullptr;
  if (!captured) {
    sp = &h->slots[h->next_slot];
    h->next_slot = (h->next_slot + 1) % kSlots;
    NRM_CHECK(retire_slot(h, *sp));
    if (!param) NRM_CHECK(ensure_slot_capacity(h, *sp, n));
  }
  std::vector<FrameDesc> fdv;
  std::vector<int> tbv;
  nrm::BatchHeader hdr_local;
  std::memset(&hdr_local, 0, sizeof(hdr_local));
  nrm::BatchHeader* hdr = &hdr_local;
  FrameDesc* fd;
  int* tb;
  if (param) {
    fdv.resize((size_t)n);
    tbv.resize((size_t)n + 1);
    fd = fdv.data();
    tb = tbv.data();
  } else {
    char* base = static_cast<char*>(sp->host);
    hdr = reinterpret_cast<nrm::BatchHeader*>(base);
    tb = reinterpret_cast<int*>(base + nrm::kTileBeginOffset);
    fd = reinterpret_cast<FrameDesc*>(base + nrm::frames_offset(sp->capacity));
  }
  const double q = scales->form == NRM_MS_QUAD ? 4.0 : 1.0;
  int acc = 0;
  for (int i = 0; i < n; ++i) {
    const nrm_frame& f = frames[i];
    const int eb = f.in_dtype == NRM_IN_U16_MM ? 2 : 4;
    make_desc(&fd[i], f.depth, f.normals, f.valid, f.H, f.W, f.depth_pitch, f.out_pitch, f.K, f.in_dtype, h->p,
              TX, TY, TX + 2 * nrm::pad_x(ms.alpha_max, eb), TY + 2 * ms.alpha_max);
    // Per-frame bases; the kernel scales them by alpha_i (a, b) and alpha_i^2 (c).
    const double sc = f.in_dtype == NRM_IN_U16_MM ? (double)h->p.depth_scale : 1.0;
    fd[i].a = (float)(sc * sc / (q * f.K.fy * ms.K));
    fd[i].b = (float)(sc * sc / (q * f.K.fx * ms.K));
    fd[i].c = (float)(sc * sc / (q * f.K.fx * f.K.fy * ms.K));
    fd[i].tile_begin = acc;
    tb[i] = acc;
    acc += fd[i].tiles_x * ((f.H + TY - 1) / TY);
  }
  tb[n] = acc;
  hdr->n_frames = n;
  hdr->total_tiles = acc;
  nrm::BatchArgs args;
  std::memset(&args, 0, sizeof(args));
  nrm::Globals g = make_globals(h);
  if (param) {
    std::vector<unsigned char> raw(nrm::param_batch_bytes() + 128);
    void* pb = raw.data() + (128 - reinterpret_cast<uintptr_t>(raw.data()) % 128) % 128;
    nrm::pack_param_batch(pb, *hdr, tb, fd, n);
    NRM_CUDA(nrm::launch_multiscale_batched(args, ms, g, h->p.out_dtype, scales->form, acc, u16, st, pb),
             "launch fwd_ms_persistent_param_kernel");
  } else {
    const size_t used = nrm::frames_offset(sp->capacity) + sizeof(FrameDesc) * (size_t)n;
    NRM_CUDA(cudaMemcpyAsync(sp->dev, sp->host, used, cudaMemcpyHostToDevice, st), "cudaMemcpyAsync");
    args.hdr = reinterpret_cast<const nrm::BatchHeader*>(sp->dev);
    args.tile_begin = reinterpret_cast<const int*>(static_cast<char*>(sp->dev) + nrm::kTileBeginOffset);
    args.frames = reinterpret_cast<const FrameDesc*>(static_cast<char*>(sp->dev) + nrm::frames_offset(sp->capacity));
    NRM_CUDA(nrm::launch_multiscale_batched(args, ms, g, h->p.out_dtype, scales->form, acc, u16, st),
             "launch fwd_ms_persistent_kernel");
  }
  if (sp) {
    NRM_CUDA(cudaEventRecord(sp->done, st), "cudaEventRecord");
    sp->in_flight = true;
    sp->timed_launch = false;
    sp->tiles = acc;
  }
  return NRM_OK;
}

int nrm_estimate_multiscale(nrm_handle* h, const void* depth, void* normals, uint8_t* valid,
                            const nrm_scales* scales, void* cuda_stream) {
  g_last_error.clear();
  if (!h) return fail(NRM_ERR_INVALID_ARG, "handle is NULL");
  if (h->H == 0 || h->W == 0) return fail(NRM_ERR_INVALID_ARG, "handle was created for batched calls only");
  nrm::MsConsts ms;
  int rc0 = make_scales(scales, ms);
  if (rc0) return rc0;
  const int K = ms.K;
  nrm_frame f = {};
  f.depth = depth;
  f.normals = normals;
  f.valid = valid;
  f.H = h->H;
  f.W = h->W;
  f.depth_pitch = h->W;
  f.out_pitch = h->W;
  f.K = h->K;
  f.in_dtype = h->p.in_dtype;
  int rc = validate_frame(f, 0, h->p.out_dtype);
  if (rc) return rc;
  if ((long long)f.H * f.W == 0) return NRM_OK;
  // More tile rows than a launch grid holds: a one-frame batched call.
  if ((f.H + nrm::kMsTileY - 1) / nrm::kMsTileY > 65535)
    return nrm_estimate_batched_multiscale(h, &f, 1, scales, cuda_stream);
  // Per-scale constants in FP64, rounded once, with 1/K, the depth scale^2 and
  // the orientation sign folded in (Eq. 1-3 or Eq. 4-6). The products are
  // formed in the order of the single-scale constants, so one NRM_MS_QUAD
  // scale reproduces nrm_estimate bit for bit.
  const double s = f.in_dtype == NRM_IN_U16_MM ? (double)h->p.depth_scale : 1.0;
  const double sign = h->p.orient_to_camera ? -1.0 : 1.0;
  const double q = scales->form == NRM_MS_QUAD ? 4.0 : 1.0;
  for (int i = 0; i < K; ++i) {
    const double a = ms.alpha[i];
    ms.A[i] = (float)(-sign * (a / (q * f.K.fy) * s * s) / K);
    ms.B[i] = (float)(-sign * (a / (q * f.K.fx) * s * s) / K);
    ms.C[i] = (float)(sign * (a * a / (q * f.K.fx * f.K.fy) * s * s) / K);
  }
  DeviceGuard guard(h->device);
  const int TX = nrm::kMsTileX, TY = nrm::kMsTileY;
  const int eb = f.in_dtype == NRM_IN_U16_MM ? 2 : 4;
  FrameDesc d;
  make_desc(&d, depth, normals, valid, f.H, f.W, f.depth_pitch, f.out_pitch, f.K, f.in_dtype, h->p, TX, TY,
            TX + 2 * nrm::pad_x(ms.alpha_max, eb), TY + 2 * ms.alpha_max);
  nrm::Globals g = make_globals(h);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  NRM_CUDA(nrm::launch_multiscale(d, ms, g, h->p.out_dtype, scales->form, st), "launch fwd_ms_kernel");
  NRM_CHECK(mark_single(h, st));
  return NRM_OK;
}

int nrm_plane_fit(nrm_handle* h, const void* depth, float* normals, uint8_t* valid, int radius,
                  void* cuda_stream) {
  g_last_error.clear();
  if (!h) return fail(NRM_ERR_INVALID_ARG, "handle is NULL");
  if (h->H == 0 || h->W == 0) return fail(NRM_ERR_INVALID_ARG, "handle was created for batched calls only");
  if (radius < 1 || radius > NRM_MAX_PLANE_RADIUS)
    return fail(NRM_ERR_UNSUPPORTED, "radius %d outside 1..%d", radius, NRM_MAX_PLANE_RADIUS);
  nrm_frame f = {};
  f.depth = depth;
  f.normals = normals;
  f.valid = valid;
  f.H = h->H;
  f.W = h->W;
  f.depth_pitch = h->W;
  f.out_pitch = h->W;
  f.K = h->K;
  f.in_dtype = h->p.in_dtype;
  int rc = validate_frame(f, 0, NRM_OUT_F32X4);
  if (rc) return rc;
  if ((h->H + 7) / 8 > 65535) return fail(NRM_ERR_UNSUPPORTED, "too many tile rows for the plane-fit launch");
  DeviceGuard guard(h->device);
  FrameDesc d;
  std::memset(&d, 0, sizeof(d));
  d.depth = depth;
  d.normals = normals;
  d.valid = valid;
  d.H = f.H;
  d.W = f.W;
  d.depth_pitch = f.depth_pitch;
  d.out_pitch = f.out_pitch;
  d.inv_fx = (float)(1.0 / f.K.fx);
  d.inv_fy = (float)(1.0 / f.K.fy);
  d.cx = (float)f.K.cx;
  d.cy = (float)f.K.cy;
  d.in_dtype = f.in_dtype;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  NRM_CUDA(nrm::launch_plane_fit(d, radius, h->p.orient_to_camera ? -1.0f : 1.0f, st), "launch plane_fit_kernel");
  NRM_CHECK(mark_single(h, st));
  return NRM_OK;
}

int nrm_selftest_wait_expiry(unsigned long long timeout_ns, float* elapsed_ms) {
  g_last_error.clear();
  if (timeout_ns < 1000ull || timeout_ns > 1000000000ull)
    return fail(NRM_ERR_INVALID_ARG, "timeout_ns outside 1e3 .. 1e9");
  int* d = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int host[2] = {0, 0};
  int rc = NRM_OK;
  cudaError_t e = cudaMalloc(&d, 2 * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(d, 0, 2 * sizeof(int));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, 0);
  if (e == cudaSuccess) e = nrm::launch_wait_expiry(timeout_ns, d, 0);
  if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaMemcpy(host, d, 2 * sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && elapsed_ms) e = cudaEventElapsedTime(elapsed_ms, e0, e1);
  if (e != cudaSuccess) rc = fail(NRM_ERR_CUDA, "self-test: %s", cudaGetErrorString(e));
  else if (host[0] != NRM_ERR_TIMEOUT || host[1] != NRM_ERR_TIMEOUT)
    rc = fail(NRM_ERR_CUDA, "self-test: waits reported %d and %d instead of NRM_ERR_TIMEOUT", host[0], host[1]);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (d) cudaFree(d);
  return rc;
}

int nrm_selftest_bounds(int* results) {
  g_last_error.clear();
  if (!results) return fail(NRM_ERR_INVALID_ARG, "results is NULL");
  int* d = nullptr;
  int host[9] = {0};
  cudaError_t e = cudaMalloc(&d, 9 * sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(d, 0, 9 * sizeof(int));
  if (e == cudaSuccess) e = nrm::launch_bounds_selftest(d, d + 8, 0);
  if (e == cudaErrorNotSupported) {
    cudaFree(d);
    return fail(NRM_ERR_UNSUPPORTED, "not the checking build (build.py --debug)");
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(host, d, 9 * sizeof(int), cudaMemcpyDeviceToHost);
  if (d) cudaFree(d);
  if (e != cudaSuccess) return fail(NRM_ERR_CUDA, "bounds self-test: %s", cudaGetErrorString(e));
  for (int i = 0; i < 7; ++i) results[i] = host[i];
  results[7] = host[8];  // the status word
  return NRM_OK;
}

int nrm_sync_status(nrm_handle* h) {
  if (!h) return fail(NRM_ERR_INVALID_ARG, "handle is NULL");
  DeviceGuard guard(h->device);
  int rc = retire_all(h);
  if (rc) return rc;
  int st = 0;
  NRM_CUDA(cudaMemcpy(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost), "cudaMemcpy status");
  NRM_CUDA(cudaMemset(h->d_status, 0, sizeof(int)), "cudaMemset status");
  if (st != NRM_OK) return fail(st, "device reported %s", nrm_status_string(st));
  return NRM_OK;
}

int nrm_get_config(const nrm_handle* h, nrm_tile_config* cfg) {
  if (!h || !cfg) return fail(NRM_ERR_INVALID_ARG, "NULL argument");
  *cfg = h->cfg;
  return NRM_OK;
}

int nrm_set_config(nrm_handle* h, const nrm_tile_config* cfg) {
  if (!h || !cfg) return fail(NRM_ERR_INVALID_ARG, "NULL argument");
  DeviceGuard guard(h->device);
  return configure(h, *cfg);
}

int nrm_enable_timing(nrm_handle* h, int enable) {
  if (!h) return fail(NRM_ERR_INVALID_ARG, "handle is NULL");
  h->timing = enable != 0;
  return NRM_OK;
}

int nrm_get_stats(nrm_handle* h, nrm_stats* out) {
  if (!h || !out) return fail(NRM_ERR_INVALID_ARG, "NULL argument");
  DeviceGuard guard(h->device);
  int rc = retire_all(h);
  if (rc) return rc;
  *out = h->stats;
  return NRM_OK;
}

int nrm_reset_stats(nrm_handle* h) {
  if (!h) return fail(NRM_ERR_INVALID_ARG, "handle is NULL");
  DeviceGuard guard(h->device);
  int rc = retire_all(h);
  if (rc) return rc;
  h->stats = nrm_stats{0, 0.0, 0};
  return NRM_OK;
}

int nrm_autotune(nrm_handle* h, const nrm_frame* frames, int n, void* cuda_stream, const char* cache_path) {
  g_last_error.clear();
  if (!h || (!frames && n > 0) || n < 0) return fail(NRM_ERR_INVALID_ARG, "bad arguments");
  if (n == 0) return NRM_OK;
  DeviceGuard guard(h->device);
  const std::string key = tune_key(h, frames, n);
  const std::string path = tune_path(cache_path);
  std::map<std::string, std::string> cache;
  if (!path.empty()) {
    {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      cache = read_cache(path.c_str());
    }
    auto it = cache.find(key);
    nrm_tile_config c;
    if (it != cache.end() && parse_config(it->second, &c) && configure(h, c) == NRM_OK) return NRM_OK;
  }
  const bool timing_was = h->timing;
  h->timing = false;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  cudaEvent_t e0, e1;
  NRM_CUDA(cudaEventCreate(&e0), "cudaEventCreate");
  NRM_CUDA(cudaEventCreate(&e1), "cudaEventCreate");
  const nrm_tile_config start = h->cfg;
  nrm_tile_config best = start;
  float best_ms = INFINITY;
  int rc = NRM_OK;
  // The batch decides which staging size (and so which occupancy) applies.
  bool points = false, u16 = true;
  for (int i = 0; i < n; ++i) {
    points = points || frames[i].points;
    u16 = u16 && (frames[i].in_dtype == NRM_IN_U16_MM || (long long)frames[i].H * frames[i].W == 0);
  }
  // Candidates: every compiled tile shape x pipeline depth x CTAs per SM from
  // 2 up to the occupancy limit (fewer concurrent CTAs can write to HBM
  // faster, so the limit is not always best).
  std::vector<nrm_tile_config> cands;
  for (int i = 0; i < nrm::fwd_kernel_count(); ++i) {
    const FwdKernelSet* k = nrm::fwd_kernel(i);
    for (int stages = 2; stages <= 4; ++stages) {
      nrm_tile_config c = {k->tile_x, k->tile_y, k->threads, stages, 0};
      if (configure(h, c) != NRM_OK) continue;  // e.g. does not fit
      const int grid = points ? h->persistent_grid_pts[u16] : h->persistent_grid[u16];
      const int occ = h->sm_count > 0 ? grid / h->sm_count : 1;
      for (int ctas = std::min(2, occ); ctas <= occ; ++ctas) {
        c.ctas_per_sm = ctas;
        cands.push_back(c);
      }
    }
  }
  for (size_t ci = 0; ci < cands.size() && rc == NRM_OK; ++ci) {
    {
      const nrm_tile_config c = cands[ci];
      if (configure(h, c) != NRM_OK) continue;
      for (int w = 0; w < 2 && rc == NRM_OK; ++w) rc = nrm_estimate_batched(h, frames, n, cuda_stream);
      if (rc) break;
      const int reps = 5;
      cudaEventRecord(e0, st);
      for (int r = 0; r < reps && rc == NRM_OK; ++r) rc = nrm_estimate_batched(h, frames, n, cuda_stream);
      cudaEventRecord(e1, st);
      if (rc) break;
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        rc = fail(NRM_ERR_CUDA, "autotune: launch failed");
        break;
      }
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best_ms) {
        best_ms = ms;
        best = c;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->timing = timing_was;
  int rc2 = configure(h, rc == NRM_OK ? best : start);
  if (rc) return rc;
  if (rc2) return rc2;
  if (!path.empty()) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    cache = read_cache(path.c_str());  // entries other processes added meanwhile
    cache[key] = format_config(best);
    cache[handle_key(h)] = format_config(best);
    write_cache(path.c_str(), cache);
  }
  return NRM_OK;
}

}  // extern "C"
