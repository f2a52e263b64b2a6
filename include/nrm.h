/*
 * nrm.h - C ABI of the GB300 (sm_103a) surface-normal library.
 *
 * Method: Moradi, Memarmoghadam and Laurendeau, "Fast, Accurate and Object
 * Boundary-Aware Surface Normal Estimation from Depth Maps", arXiv 2209.08241.
 *
 * For every pixel of an organised depth map the library computes the
 * multi-direction normal of Section 3.1 (the average of four perpendicular
 * tangent-pair cross products), evaluated through its reformulation as one
 * cross product 1/4 s24 x s35 in the closed form of Eq. 4-6:
 *   n_x = -alpha/(4 f_y) (d3 + d5)(d2 - d4)
 *   n_y = -alpha/(4 f_x) (d2 + d4)(d3 - d5)
 *   n_z = -u1 n_x - v1 n_y + alpha^2/(4 f_x f_y) (d2 + d4)(d3 + d5)
 * with u1 = (col - cx)/fx, v1 = (row - cy)/fy (Section 2, definitions below
 * Eq. 3), neighbours 2/4 at +-alpha along the column axis and 3/5 at +-alpha
 * along the row axis (Fig. 2). It then normalises n and removes normals at
 * depth discontinuities by thresholding the length statistic of Section 3.2
 * (Eq. "veclength"), applying the mask to the normal map (Section 4, Fig. 8).
 *
 * Conventions (the paper is silent on them):
 *   - A pixel is invalid when any of its five stencil depths lies outside the
 *     image or is not a positive finite number (uint16: raw value 0).
 *   - Mask statistic: NRM_MASK_RAW thresholds r = ||n|| (the paper's literal
 *     statistic, in m^2); NRM_MASK_SECANT thresholds r ||ray|| / (n . ray) with
 *     ray = (u1, v1, 1), which equals 1/cos of the angle between the normal and
 *     the viewing ray and does not depend on depth, alpha or focal length.
 *   - A pixel is valid iff stat <= tau. Masked pixels get the normal (0,0,0,0)
 *     and mask byte 0; valid pixels get mask byte 1.
 *   - Sign: the paper's normal points away from the camera (n . P1 > 0);
 *     orient_to_camera = 1 negates it.
 *   - Numerical domain: the kernels evaluate Eq. 4-6 and the statistic in
 *     FP32. For depths d (metres, after depth_scale) with
 *     2^-28 <= alpha d / f <= 2^28 for f = fx and fy (at f = 525 px and
 *     alpha = 2: about 1e-6 m to 7e10 m) no product under- or overflows, the
 *     normal is within 1e-6 rad of the FP64 definition and the mask decides
 *     like it except where the statistic lies within 1e-6 relative of tau
 *     (tested at both ends). Below that range q = n . n falls under FLT_MIN
 *     and pixels are reported invalid; above it the statistic overflows and
 *     results are unspecified.
 *
 * Memory and ownership: every depth, normal, mask and gradient pointer passed
 * to this library is a DEVICE pointer owned by the caller (except in
 * nrm_estimate_batched_host, which takes host pointers). The library cannot
 * see the extent of a buffer: each must hold the pixels its size and pitch
 * describe. Normals are stored
 * as 4 components per pixel (x, y, z, 0): float32 (16 B/px) or IEEE half
 * (8 B/px). The mask is one uint8 per pixel. All images are row-major.
 * A handle owns only small device state: per-frame descriptors and TMA tensor
 * maps, a status word and captured CUDA graphs.
 *
 * Errors: every call returns an nrm_status. Arguments are checked on the host
 * before anything is launched; a rejected call launches nothing and sets a
 * thread-local message readable with nrm_last_error(). Launches are
 * asynchronous on the caller's stream (NULL = the legacy default stream).
 * Device-side failures (a bounded wait that ran out) are written to the
 * handle's status word and reported by nrm_sync_status().
 *
 * Threading: a handle may be used from one host thread at a time.
 */
#ifndef NRM_H_
#define NRM_H_

#include <stdint.h>

#if defined(__GNUC__)
#define NRM_API __attribute__((visibility("default")))
#else
#define NRM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  NRM_OK = 0,
  NRM_ERR_INVALID_ARG = 1, /* bad pointer, size, pitch or parameter */
  NRM_ERR_UNSUPPORTED = 2, /* valid but outside what the kernels support */
  NRM_ERR_CUDA = 3,        /* a CUDA runtime call failed (see nrm_last_error) */
  NRM_ERR_OOM = 4,         /* a device or pinned allocation failed */
  NRM_ERR_TIMEOUT = 5,     /* a bounded device wait ran out */
  NRM_ERR_NO_DEVICE = 6,   /* no CUDA device is visible */
  NRM_ERR_BOUNDS = 7       /* checking build only: an index left its buffer (the access was skipped) */
} nrm_status;

/* Pinhole intrinsics in pixels (Section 2: f_x, f_y, o_x, o_y); fx, fy > 0. */
typedef struct {
  double fx, fy, cx, cy;
} nrm_intrinsics;

typedef enum { NRM_IN_F32_M = 0, NRM_IN_U16_MM = 1 } nrm_in_dtype;
/* Normal map encodings: 4 x float32 (x, y, z, 0), 16 B/px; 4 x IEEE half, 8 B/px;
 * or the octahedral code of the unit normal in 2 x int16, 4 B/px (low half x,
 * high half y; p = round(32767 q) with q = n.xy / |n|_1 folded over the diagonals
 * where n_z < 0; decode: v = (q_x, q_y, 1 - |q_x| - |q_y|), and where v_z < 0,
 * (v_x, v_y) = (1 - |q_y|, 1 - |q_x|) with the signs of (q_x, q_y); normalise v).
 * Masked pixels get code 0 (the mask, not the code, says which pixels are valid). */
typedef enum { NRM_OUT_F32X4 = 0, NRM_OUT_F16X4 = 1, NRM_OUT_OCT16 = 2 } nrm_out_dtype;
typedef enum { NRM_MASK_RAW = 0, NRM_MASK_SECANT = 1 } nrm_mask_mode;

/* Largest pixel distance alpha the kernels accept. */
#define NRM_MAX_ALPHA 16

typedef struct {
  int alpha;            /* pixel distance alpha, 1..NRM_MAX_ALPHA (Section 3.1) */
  int mask_mode;        /* nrm_mask_mode */
  float tau;            /* threshold: valid iff stat <= tau; tau >= 0 (may be +inf) */
  float depth_scale;    /* metres per uint16 unit (default 0.001) */
  int in_dtype;         /* nrm_in_dtype of nrm_estimate / nrm_backward input */
  int out_dtype;        /* nrm_out_dtype of the normal map */
  int orient_to_camera; /* 0 = paper sign (default), 1 = negated */
} nrm_params;

/* Defaults: alpha 2, SECANT, tau 12, depth_scale 0.001, f32 in, f32x4 out. */
NRM_API void nrm_default_params(nrm_params* p);

typedef struct nrm_handle nrm_handle;

/* One frame of a batch. Pitches are in elements of the respective buffer:
 * depth_pitch in depth elements (>= W); out_pitch in pixels for the normal
 * map, the mask and the point cloud (>= W).
 * points (optional, may be NULL): the organised point cloud of the frame,
 * written in the same pass, H x W x 4 float32 (x, y, z, 0) in metres,
 * P = d (u, v, 1) (Section 2, the back-projection below Eq. 3), the origin
 * where the depth is invalid (independent of the normal mask); 16-byte
 * aligned device memory. */
typedef struct {
  const void* depth;
  void* normals;
  uint8_t* valid;
  int H, W;
  long long depth_pitch;
  long long out_pitch;
  nrm_intrinsics K;
  int in_dtype;
  float* points;
} nrm_frame;

/* Creates a handle for H x W frames with intrinsics K (used by nrm_estimate and
 * nrm_backward; batched calls carry their own sizes and intrinsics). H = W = 0
 * (K may then be NULL) makes a handle for batched calls only. p = NULL takes
 * the defaults. Allocates the handle's device state on the current device. */
NRM_API int nrm_create(const nrm_intrinsics* K, int H, int W, const nrm_params* p, nrm_handle** out);

/* Releases the handle and its device state. Waits for its pending work. */
NRM_API void nrm_destroy(nrm_handle* h);

/* Single frame, one plain launch (one CTA per tile, TMA-staged halo tiles).
 * depth: H x W (dense, pitch W) of the handle's in_dtype; normals: H x W x 4
 * (dense) of the handle's out_dtype; valid: H x W bytes (dense).
 * Sizes: H and W up to 2^24 (NRM_ERR_UNSUPPORTED above). A frame with more
 * tile rows than one launch grid holds (65535) runs as a one-frame
 * nrm_estimate_batched call, whose results are bitwise the same. */
NRM_API int nrm_estimate(nrm_handle* h, const void* depth, void* normals, uint8_t* valid,
                 void* cuda_stream);

/* nrm_estimate that also writes the frame's organised point cloud (see
 * nrm_frame.points: H x W x 4 float32, pitch W, 16-byte aligned device memory;
 * NULL is NRM_ERR_INVALID_ARG). */
NRM_API int nrm_estimate_points(nrm_handle* h, const void* depth, void* normals, uint8_t* valid, float* points,
                                void* cuda_stream);

/* n frames of any sizes, intrinsics and input dtypes in ONE persistent launch
 * over a (frame, tile) work list. The handle's alpha, mask mode, tau,
 * depth_scale, out_dtype and orientation apply to all frames. n = 0 is a
 * no-op. The frames' buffers must not overlap.
 * Up to 100 frames without point buffers: the frame records and their TMA
 * tensor maps travel as one kernel parameter (no descriptor upload, no
 * tensor-map fences). Larger batches, or batches with point buffers: a CUDA
 * graph per descriptor slot (upload node, then the kernel node), replayed
 * from a ring of slots. Either way the host may return before the GPU has
 * started; it blocks only when every slot of the ring is still in use.
 * Stream capture: while cuda_stream is being captured (any capture mode), the
 * call records a single kernel node with the parameter form and no events or
 * host synchronisation, so the captured graph can be replayed freely while
 * the frames' buffers stay valid; then n is at most 100 and frames may not
 * carry point buffers (NRM_ERR_UNSUPPORTED). The handle must have been
 * configured (created, or set_config / autotune) before the capture begins. */
NRM_API int nrm_estimate_batched(nrm_handle* h, const nrm_frame* frames, int n, void* cuda_stream);

/* Adjoint of nrm_estimate for float32 depth (derivatives of Eq. 4-6 and of the
 * normalisation), with the mask held fixed:
 *   grad_depth[q] = sum over valid p whose stencil holds q of
 *                   g[p] . d(n_hat[p]) / d(depth[q]),
 * g = grad_normals, H x W x 4 float32 (the 4th component is ignored).
 * valid: the mask nrm_estimate produced for this depth (a pixel it marks valid
 * must have a positive finite five-point stencil; other masks give undefined
 * gradients). Deterministic (gather, no atomics).
 * Returns NRM_ERR_UNSUPPORTED for a uint16 handle. A frame with more than 65535
 * tile rows runs as a one-frame nrm_backward_batched call (same results). */
NRM_API int nrm_backward(nrm_handle* h, const void* depth, const float* grad_normals,
                 const uint8_t* valid, float* grad_depth, void* cuda_stream);

/* One frame of a batched adjoint. depth and grad_depth: H x W float32 with pitch
 * depth_pitch elements; grad_normals (float4 per pixel, 4th component ignored)
 * and valid (the mask the forward produced): pitch out_pitch pixels. */
typedef struct {
  const float* depth;
  const float* grad_normals;
  const uint8_t* valid;
  float* grad_depth;
  int H, W;
  long long depth_pitch;
  long long out_pitch;
  nrm_intrinsics K;
} nrm_grad_frame;

/* nrm_backward for n float32 frames of any sizes and intrinsics in one launch
 * over all their tiles (the handle's alpha and orientation apply). Same
 * per-pixel arithmetic as nrm_backward. n = 0 is a no-op. Up to 60 frames the
 * frame records and tensor maps travel as one kernel parameter (nothing to
 * upload; the call can be recorded by stream capture); larger batches use a
 * ring of device descriptor blocks and return NRM_ERR_UNSUPPORTED while the
 * stream is being captured. */
NRM_API int nrm_backward_batched(nrm_handle* h, const nrm_grad_frame* frames, int n, void* cuda_stream);

/* nrm_backward_batched with the upstream gradient of frame i equal to
 * scale[i] times its grad_normals buffer: the normal estimator as a loss layer
 * without forming dL/dn_hat in a separate pass. For the cosine loss
 * L = mean over valid pixels of (1 - n_hat . t), whose gradient is
 * dL/dn_hat = -t / N_valid on valid pixels, pass the target normals t as
 * grad_normals (float4, 4th component ignored) and scale[i] = -1 / N_valid(i).
 * scale: a device array of n floats (4-byte aligned; NRM_ERR_INVALID_ARG if
 * NULL), read by the kernel, so it may be computed on the GPU in the same
 * stream. Otherwise exactly nrm_backward_batched (bit for bit equal to it on
 * grad_normals = scale[i] * t rounded to float32). */
NRM_API int nrm_backward_batched_scaled(nrm_handle* h, const nrm_grad_frame* frames, int n, const float* scale,
                                        void* cuda_stream);

/* The per-frame factor of that cosine loss: scale[i] = -1 / max(N_valid(i), 1),
 * N_valid(i) the number of nonzero bytes of frames[i].valid (H x W, pitch
 * out_pitch pixels; the other fields are not read). One launch per 128
 * frames; the count is exact (integer sums) and the division is IEEE float32,
 * so the result equals -1 / max(N, 1) formed in float32. scale: n floats of
 * device memory (4-byte aligned), written asynchronously on the stream, where
 * nrm_backward_batched_scaled on the same stream then reads it. Uses counters
 * owned by the handle (allocated on first use and when n grows): calls on one
 * handle must not overlap on the GPU. n = 0 is a no-op. */
NRM_API int nrm_cosine_loss_scale(nrm_handle* h, const nrm_grad_frame* frames, int n, float* scale,
                                  void* cuda_stream);

/* Spherical angle images of a normal map (Section 4, the I_phi and I_theta
 * images, normalised to [0, 2 pi]): for each valid pixel
 *   phi = atan2(n_y, n_x) in [0, 2 pi),  theta = atan2(sqrt(n_x^2 + n_y^2), n_z) in [0, pi];
 * masked pixels get 0. Each angle is within about 3e-7 rad of the exact
 * value of its float32 inputs (atan2's signed-zero conventions included;
 * phi may round up to 2 pi itself just below the cut). normals: H x W x 4
 * float32; valid: H x W bytes; phi and theta: H x W float32; one pitch
 * (pixels) for all four. Device pointers; asynchronous on the stream. */
NRM_API int nrm_spherical(const float* normals, const uint8_t* valid, int H, int W, long long pitch, float* phi,
                          float* theta, void* cuda_stream);

/* Mean squared error of the angle images (Section 4, Tables 2-5) between an
 * estimate and a reference normal map, over the pixels valid in both, with
 * plain differences of the [0, 2 pi) values. out: 3 doubles in device memory,
 * {MSE of I_theta, MSE of I_phi, number of pixels}. Deterministic: a fixed
 * reduction order, no atomics. Uses scratch owned by the handle (allocated on
 * the first call); calls on one handle must not overlap on the GPU. */
NRM_API int nrm_angle_mse(nrm_handle* h, const float* normals, const uint8_t* valid, const float* ref_normals,
                          const uint8_t* ref_valid, int H, int W, long long pitch, double* out, void* cuda_stream);

/* Multi-scale variant (Section 2: the authors' previous method averages its
 * closed-form normal over pixel distances alpha_1..alpha_K to reduce noise).
 * For each pixel the unnormalised per-scale normals are averaged,
 *   n = (1/K) sum_i n(alpha_i),
 * with every neighbour depth sampled at its own scale's distance alpha_i, and
 * n(alpha) one of
 *   NRM_MS_PAIR  the previous method's single tangent pair, Eq. 1-3:
 *                neighbours (col + alpha, row) and (col, row + alpha);
 *   NRM_MS_QUAD  the four-direction form of this paper, Eq. 4-6.
 * The handle's mask mode and tau (Section 3.2, applied to the averaged n),
 * depth dtype, depth scale, output dtype and orientation apply; its alpha is
 * ignored. A pixel is valid only if every depth that any scale uses is inside
 * the image and valid. Buffers as for nrm_estimate (device pointers, pitch W,
 * asynchronous on the stream). A frame with more than 65535 tile rows runs as a
 * one-frame nrm_estimate_batched_multiscale call (whose per-scale constants
 * are formed on the GPU, so results can differ in the last bits). */
#define NRM_MAX_SCALES 8
typedef enum { NRM_MS_PAIR = 0, NRM_MS_QUAD = 1 } nrm_ms_form;
typedef struct {
  int n_scales;                /* K, 1..NRM_MAX_SCALES */
  int alpha[NRM_MAX_SCALES];   /* alpha_1..alpha_K, each 1..NRM_MAX_ALPHA; order does not matter */
  int form;                    /* nrm_ms_form */
} nrm_scales;
NRM_API int nrm_estimate_multiscale(nrm_handle* h, const void* depth, void* normals, uint8_t* valid,
                                    const nrm_scales* scales, void* cuda_stream);

/* nrm_estimate_batched on frames whose depth, normals, valid and points are
 * HOST pointers (page-locked memory for asynchronous copies; pageable memory
 * works, with copies that return only once done). The library stages the
 * frames in handle-owned device memory (allocated on first use and when a
 * larger chunk is needed), splits the batch into chunks of consecutive frames
 * (about 96 MB of staging each) on two internal streams, and for each chunk
 * uploads the depth, runs the batched kernel and downloads normals, masks and
 * points, so that uploads and kernels overlap earlier chunks' downloads. The
 * work starts after everything already queued on cuda_stream, and cuda_stream
 * waits for all of it: synchronise cuda_stream before reading the host
 * outputs, and keep every buffer valid until then. Pitches are those of the
 * host buffers. Results are those of nrm_estimate_batched, bit for bit. If an
 * error is returned part of the batch may already be queued. */
NRM_API int nrm_estimate_batched_host(nrm_handle* h, const nrm_frame* frames, int n, void* cuda_stream);

/* nrm_estimate_multiscale for n frames of any sizes, dtypes and intrinsics in
 * one persistent launch (the batched pipeline of nrm_estimate_batched, tile
 * 128 x 16, 256 compute threads). Frames as for nrm_estimate_batched; their
 * points must be NULL (NRM_ERR_UNSUPPORTED otherwise). The per-scale constants
 * are formed on the GPU from each frame's intrinsics, so results can differ
 * from nrm_estimate_multiscale's in the last bits. n = 0 is a no-op. Up to 100
 * frames the descriptors travel as one kernel parameter, and while the stream
 * is being captured the call records a single kernel node (then n <= 100). */
NRM_API int nrm_estimate_batched_multiscale(nrm_handle* h, const nrm_frame* frames, int n, const nrm_scales* scales,
                                            void* cuda_stream);

/* Plane-fitting ("plane-PCA") normals, the ground truth the paper evaluates
 * against on real data (Section 1 describes the fit; Section 4 uses it with 25
 * neighbouring points, i.e. radius 2). For each pixel: the back-projected
 * points P = d (u, v, 1) of its (2 radius + 1) x (2 radius + 1) window, their
 * scatter matrix about the centroid, and the unit eigenvector of its smallest
 * eigenvalue, oriented like the method's normal (n . P > 0, or n . P < 0 with
 * orient_to_camera). A pixel is valid iff every depth of its window lies in the
 * image and is positive and finite (uint16: nonzero); other pixels get normal
 * (0, 0, 0, 0) and mask byte 0.
 * Uses the handle's H, W, intrinsics, in_dtype and orient_to_camera (the depth
 * scale cancels from the direction). depth: H x W in_dtype values, pitch W;
 * normals: H x W x 4 float32 (w = 0), 16-byte aligned; valid: H x W bytes.
 * Device pointers, asynchronous on the stream. radius in 1..NRM_MAX_PLANE_RADIUS,
 * else NRM_ERR_UNSUPPORTED. FP32 arithmetic on coordinates taken relative to the
 * window's centre point; the eigenproblem by cyclic Jacobi rotations. One CTA
 * per 32 x 8 tile: H above 65535 x 8 rows is NRM_ERR_UNSUPPORTED. */
#define NRM_MAX_PLANE_RADIUS 4
NRM_API int nrm_plane_fit(nrm_handle* h, const void* depth, float* normals, uint8_t* valid, int radius,
                          void* cuda_stream);

/* Self-test of the bounded waits (no counterpart in the paper; a deployment
 * check of failure reporting). On the current device, launches one block
 * whose threads wait on a shared-memory barrier that nothing completes, with
 * the same bounded waits every kernel here uses (warp-level and per-thread),
 * for timeout_ns of GPU global time each (1e3 .. 1e9 ns, else
 * NRM_ERR_INVALID_ARG). Both must give up and report NRM_ERR_TIMEOUT through a
 * device status word. Synchronous. Returns NRM_OK if both reported the
 * timeout (*elapsed_ms, if not NULL, gets the kernel's duration), or
 * NRM_ERR_CUDA. Leaves the context usable; allocates and frees 8 bytes. */
NRM_API int nrm_selftest_wait_expiry(unsigned long long timeout_ns, float* elapsed_ms);

/* Self-test of the range checks of the checking build (build.py --debug; no
 * counterpart in the paper). Evaluates the checks on addresses inside and
 * just outside a shared-memory block, a global array and an index range,
 * forming and comparing addresses only (nothing outside a buffer is touched),
 * and writes results[0..6] (1 = accepted, 0 = rejected; right is
 * 1, 1, 0, 0, 1, 0, 0) and results[7] = the status word (NRM_ERR_BOUNDS after
 * the rejections). Synchronous; allocates and frees 36 bytes. Returns
 * NRM_ERR_UNSUPPORTED in the ordinary build. */
NRM_API int nrm_selftest_bounds(int* results);

/* Waits for the handle's work, returns the device status word (NRM_OK or the
 * first device-side error since the last call) and clears it. */
NRM_API int nrm_sync_status(nrm_handle* h);

/* Launch geometry of the forward kernels. (tile_x, tile_y, threads) must be one
 * of the compiled shapes: (128,16,256) (the default), (128,8,256), (128,32,256),
 * (128,8,128), (128,16,128), (128,32,512), (128,64,512), (64,16,128),
 * (64,32,256), (64,64,256). threads counts the compute threads; the persistent
 * kernel adds one producer warp. stages in {2, 3, 4} (persistent kernel only);
 * ctas_per_sm 0 = as many as fit. */
typedef struct {
  int tile_x, tile_y, threads, stages, ctas_per_sm;
} nrm_tile_config;

NRM_API int nrm_get_config(const nrm_handle* h, nrm_tile_config* cfg);
NRM_API int nrm_set_config(nrm_handle* h, const nrm_tile_config* cfg);

/* Times every supported configuration on the given batch (which must stay
 * valid during the call; outputs are overwritten), keeps the fastest in the
 * handle and records it in the JSON cache file cache_path, keyed by GPU name,
 * SM count, frame-size class, dtypes and alpha. cache_path = NULL takes the
 * process-wide cache file (nrm_set_autotune_cache), if any. If the cache
 * already holds the key, loads it without timing. The tuned configuration is
 * also recorded under the handle's own key (nrm_autotune_key), which
 * nrm_create looks up. Synchronous. */
NRM_API int nrm_autotune(nrm_handle* h, const nrm_frame* frames, int n, void* cuda_stream,
                 const char* cache_path);

/* Kernel-time statistics of batched launches: CUDA events recorded around the
 * kernel node inside the graph. Enabling timing adds two event nodes. */
typedef struct {
  long long launches; /* completed timed launches */
  double kernel_ms;   /* sum of their kernel durations */
  long long tiles;    /* tiles processed by them */
} nrm_stats;

NRM_API int nrm_enable_timing(nrm_handle* h, int enable);
NRM_API int nrm_get_stats(nrm_handle* h, nrm_stats* out); /* waits for pending launches */
NRM_API int nrm_reset_stats(nrm_handle* h);

/* Autotune cache: a JSON object mapping keys to [tile_x, tile_y, threads,
 * stages, ctas_per_sm]. These calls need no GPU.
 *
 * nrm_set_autotune_cache sets the process-wide cache file (path = NULL clears
 * it; without a call, the environment variable NRM_AUTOTUNE_CACHE names it).
 * With a cache file set, nrm_create configures a new handle from the entry of
 * its key, if there is one, instead of the default geometry, so a process
 * that tuned a workload once lets later processes skip the sweep.
 * nrm_autotune_key writes a handle's key (GPU name, SM count, input and output
 * dtypes, alpha, H x W of the handle) to buf (NUL-terminated; NRM_ERR_INVALID_ARG
 * if it does not fit in len bytes). nrm_autotune_cache_get reads the entry of
 * key from the file at path (NRM_ERR_INVALID_ARG if the file or the key is
 * absent or malformed); nrm_autotune_cache_put adds or replaces it (written to
 * a temporary file and renamed over path; NRM_ERR_INVALID_ARG if it cannot be
 * written or key contains a quote or a backslash). */
NRM_API int nrm_set_autotune_cache(const char* path);
NRM_API int nrm_autotune_key(const nrm_handle* h, char* buf, int len);
NRM_API int nrm_autotune_cache_get(const char* path, const char* key, nrm_tile_config* cfg);
NRM_API int nrm_autotune_cache_put(const char* path, const char* key, const nrm_tile_config* cfg);

/* Largest number of frames nrm_estimate_batched_noalloc accepts per call. */
#define NRM_NOALLOC_MAX_FRAMES 256

/* The batched launch of nrm_estimate_batched for callers that cannot allocate
 * device memory. The paper has no counterpart: this is a deployment interface,
 * not part of the method.
 *
 * Who needs it: a handle allocates device memory when it is created and again
 * when a batch outgrows its descriptor slots. Some callers must not do that:
 * programs that reserve their whole device memory budget up front (embedded
 * and robotics perception loops, where an allocation that fails or stalls in
 * the middle of a run is not acceptable), and code whose device memory belongs
 * to another allocator, such as a framework's caching allocator, which must
 * not call cudaMalloc or cudaFree itself (cudaFree also waits for the whole
 * device). This entry point takes no handle and allocates nothing.
 *
 * Frames, their buffers and the results are exactly those of
 * nrm_estimate_batched (same per-pixel arithmetic, bit for bit) with the
 * default launch geometry (tile 128 x 16, 256 compute threads, 3 stages).
 * p = NULL takes the defaults; p->in_dtype is ignored (each frame has its own).
 * device_status: a caller-owned device int, or NULL. The first device-side
 * error of this launch (NRM_ERR_TIMEOUT) is written there; the caller zeroes it
 * and reads it after synchronising. With NULL such an error is not reported.
 *
 * Scratch: the per-launch descriptors (about 65 KB for NRM_NOALLOC_MAX_FRAMES
 * frames) live in a static device array inside this library. Every GPU that
 * loads the library holds that array until the process exits. Every call
 * shares it and overwrites what the previous call left there, so calls whose
 * work overlaps on the GPU (for example on two streams, or from two threads)
 * race; calls on one stream are ordered and safe. The host copy of the
 * descriptors goes through cudaMemcpyAsync from pageable memory, which returns
 * once the source has been read.
 *
 * Every call looks up the array's device address (cudaGetSymbolAddress) with
 * the current device; the first call on a device, and the first call after
 * that device's context was reset (cudaDeviceReset), also set the kernel's
 * shared-memory limit.
 *
 * Stream capture: not supported. The descriptor copy reads a host array that
 * the next call overwrites, so a captured copy would replay stale descriptors;
 * a call on a stream that is being captured returns NRM_ERR_UNSUPPORTED and
 * records nothing (the capture stays valid).
 *
 * Errors: NRM_ERR_UNSUPPORTED for n > NRM_NOALLOC_MAX_FRAMES, a frame with a
 * point-cloud buffer (this entry point writes normals and masks only) or a
 * capturing stream, with nothing launched; otherwise as nrm_estimate_batched. */
NRM_API int nrm_estimate_batched_noalloc(const nrm_frame* frames, int n, const nrm_params* p,
                                         int* device_status, void* cuda_stream);

NRM_API const char* nrm_status_string(int status);
NRM_API const char* nrm_last_error(void); /* thread-local, "" if none */
NRM_API const char* nrm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* NRM_H_ */
