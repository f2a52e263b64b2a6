// nrm_estimate_batched_noalloc: the batched launch for callers that cannot
// allocate device memory (declared in include/nrm.h).
//
// The batched kernel needs a per-launch descriptor block in device memory
// (header, work-list offsets, one FrameDesc with its TMA tensor map per frame).
// Here that block lives in one file-scope static device array of fixed size,
// reserved when the library is loaded and held by every GPU that loads it until
// the process exits. A call copies the block from host memory into that array
// (cudaMemcpyAsync from pageable host memory, which returns once the source has
// been read) and launches the persistent kernel on the caller's stream. No call
// allocates device memory.
//
// The host needs the device address of the array: in host code the array's
// name is only a host-side stand-in. It is looked up with cudaGetSymbolAddress,
// with the device current, on every call (a cheap runtime query): the first
// call on a device, and the first call after the device's context was reset
// (the address may then differ), also set the kernels' shared-memory limit.
//
// A call refuses a stream that is being captured: it copies the descriptors
// from a host array that the next call overwrites, so a captured copy would
// replay whatever the latest call left there.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "nrm.h"
#include "nrm_internal.h"

namespace {

constexpr int kMaxFrames = NRM_NOALLOC_MAX_FRAMES;
constexpr size_t kScratchBytes = nrm::block_bytes(kMaxFrames);
constexpr int kTileX = 128, kTileY = 16, kThreads = 256, kStages = 3;
constexpr int kMaxDevices = 64;
constexpr unsigned long long kTimeoutNs = 2000000000ull;

// The scratch: header (which also holds the status word used when the caller
// passes none), work-list offsets and frame descriptors of the latest call.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Byte offset of the fallback status word inside the header's padding; the
// upload of each call writes it to zero.
constexpr size_t kStatusOffset = 8;

struct DeviceState {
  bool ready = false;
  unsigned char* scratch = nullptr;  // device address of g_scratch on this device
  int sm_count = 0;
};

std::mutex g_mutex;                       // guards g_devices and g_host_block
DeviceState g_devices[kMaxDevices];
alignas(256) unsigned char g_host_block[kScratchBytes];  // host image of the block

int setup_device(int device, DeviceState& st) {
  void* ptr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
  if (e != cudaSuccess) return nrm::host_fail(NRM_ERR_CUDA, cudaGetErrorString(e));
  if (st.ready && st.scratch == ptr) return NRM_OK;
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) return nrm::host_fail(NRM_ERR_CUDA, cudaGetErrorString(e));
  const nrm::FwdKernelSet* ks = nrm::fwd_kernel_find(kTileX, kTileY, kThreads);
  const unsigned smem_max = nrm::persistent_smem_bytes(kTileX, kTileY, NRM_MAX_ALPHA, kStages);
  for (int out = 0; out < 3; ++out) {
    e = cudaFuncSetAttribute(ks->persistent[out], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
    if (e != cudaSuccess) return nrm::host_fail(NRM_ERR_CUDA, cudaGetErrorString(e));
  }
  st.scratch = static_cast<unsigned char*>(ptr);
  st.sm_count = sms;
  st.ready = true;
  return NRM_OK;
}

}  // namespace

extern "C" int nrm_estimate_batched_noalloc(const nrm_frame* frames, int n, const nrm_params* params,
                                            int* device_status, void* cuda_stream) {
  nrm::host_clear_error();
  if (n < 0) return nrm::host_fail(NRM_ERR_INVALID_ARG, "n < 0");
  if (n == 0) return NRM_OK;
  if (!frames) return nrm::host_fail(NRM_ERR_INVALID_ARG, "frames is NULL");
  if (n > kMaxFrames)
    return nrm::host_fail(NRM_ERR_UNSUPPORTED,
                          "nrm_estimate_batched_noalloc takes at most NRM_NOALLOC_MAX_FRAMES frames per call");
  nrm_params p;
  nrm_default_params(&p);
  if (params) p = *params;
  int rc = nrm::host_validate_params(p);
  if (rc) return rc;
  long long total = 0;
  for (int i = 0; i < n; ++i) {
    rc = nrm::host_validate_frame(frames[i], i, p.out_dtype);
    if (rc) return rc;
    if (frames[i].points)
      return nrm::host_fail(NRM_ERR_UNSUPPORTED, "nrm_estimate_batched_noalloc writes no point clouds");
    total += (long long)((frames[i].W + kTileX - 1) / kTileX) * ((frames[i].H + kTileY - 1) / kTileY);
  }
  if (total == 0) return NRM_OK;
  if (total >= (1LL << 31) - 1) return nrm::host_fail(NRM_ERR_UNSUPPORTED, "batch exceeds 2^31 tiles");

  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  cudaStreamCaptureStatus capture = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(stream, &capture);
  if (e != cudaSuccess) return nrm::host_fail(NRM_ERR_CUDA, cudaGetErrorString(e));
  if (capture != cudaStreamCaptureStatusNone)
    return nrm::host_fail(NRM_ERR_UNSUPPORTED,
                          "nrm_estimate_batched_noalloc cannot be recorded by stream capture (its descriptor "
                          "copy reads a host array that later calls overwrite)");

  int device = 0;
  e = cudaGetDevice(&device);
  if (e != cudaSuccess) return nrm::host_fail(NRM_ERR_NO_DEVICE, cudaGetErrorString(e));
  if (device < 0 || device >= kMaxDevices) return nrm::host_fail(NRM_ERR_UNSUPPORTED, "device index too large");

  std::lock_guard<std::mutex> lock(g_mutex);
  DeviceState& st = g_devices[device];
  rc = setup_device(device, st);
  if (rc) return rc;

  // Build the block in host memory: every byte the kernel reads is written,
  // and the fallback status word starts at zero.
  const size_t foff = nrm::frames_offset(kMaxFrames);
  std::memset(g_host_block, 0, foff);
  nrm::BatchHeader* hdr = reinterpret_cast<nrm::BatchHeader*>(g_host_block);
  int* tile_begin = reinterpret_cast<int*>(g_host_block + nrm::kTileBeginOffset);
  nrm::FrameDesc* fd = reinterpret_cast<nrm::FrameDesc*>(g_host_block + foff);
  int acc = 0;
  for (int i = 0; i < n; ++i) {
    nrm::host_make_forward_desc(&fd[i], frames[i], p, kTileX, kTileY);
    fd[i].tile_begin = acc;
    tile_begin[i] = acc;
    acc += fd[i].tiles_x * ((frames[i].H + kTileY - 1) / kTileY);
  }
  tile_begin[n] = acc;
  hdr->n_frames = n;
  hdr->total_tiles = acc;

  const size_t used = foff + sizeof(nrm::FrameDesc) * (size_t)n;
  e = cudaMemcpyAsync(st.scratch, g_host_block, used, cudaMemcpyHostToDevice, stream);
  if (e != cudaSuccess) return nrm::host_fail(NRM_ERR_CUDA, cudaGetErrorString(e));

  const nrm::FwdKernelSet* ks = nrm::fwd_kernel_find(kTileX, kTileY, kThreads);
  const void* kernel = ks->persistent[p.out_dtype];
  const unsigned smem = nrm::persistent_smem_bytes(kTileX, kTileY, p.alpha, kStages);
  const int threads = nrm::persistent_threads(kThreads);
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, smem);
  if (e != cudaSuccess) return nrm::host_fail(NRM_ERR_CUDA, cudaGetErrorString(e));
  if (occ < 1) return nrm::host_fail(NRM_ERR_UNSUPPORTED, "persistent kernel does not fit on an SM");

  nrm::BatchArgs args;
  args.hdr = reinterpret_cast<const nrm::BatchHeader*>(st.scratch);
  args.tile_begin = reinterpret_cast<const int*>(st.scratch + nrm::kTileBeginOffset);
  args.frames = reinterpret_cast<const nrm::FrameDesc*>(st.scratch + foff);
  args.stages = kStages;
  args.stage_bytes = nrm::stage_bytes_for(kTileX, kTileY, p.alpha);
  nrm::Globals g;
  g.alpha = p.alpha;
  g.mask_mode = p.mask_mode;
  g.tau2 = std::isinf(p.tau) ? INFINITY : p.tau * p.tau;
  g.sign = p.orient_to_camera ? -1.0f : 1.0f;
  g.status = device_status ? device_status : reinterpret_cast<int*>(st.scratch + kStatusOffset);
  g.timeout_ns = kTimeoutNs;
  void* kargs[2] = {&args, &g};
  const int grid = occ * st.sm_count;
  e = cudaLaunchKernel(kernel, dim3(grid), dim3(threads), kargs, smem, stream);
  if (e != cudaSuccess) return nrm::host_fail(NRM_ERR_CUDA, cudaGetErrorString(e));
  return NRM_OK;
}
