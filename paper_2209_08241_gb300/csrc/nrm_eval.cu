// Evaluation kernels (arXiv 2209.08241, Section 4): the spherical angle images
// I_phi, I_theta of a normal map and the mean squared error of those images
// between an estimate and a reference (Tables 2-5).
//
//   phi   = atan2(n_y, n_x), taken into [0, 2 pi)
//   theta = atan2(sqrt(n_x^2 + n_y^2), n_z), in [0, pi]
//
// over valid pixels (masked pixels get 0). The MSE is the mean, over pixels
// valid in both maps, of the squared plain differences of the angle images.
// It is reduced deterministically: a fixed grid of kMseBlocks blocks, each
// summing a fixed set of rows (per thread in FP32, across the block in FP64)
// in a fixed order, then one block summing the partials in a fixed order. No
// atomics.
#include "nrm_device.cuh"

namespace nrm {

namespace {

constexpr int kThreads = 256;

// atan2(y, x) for the angle images: the quotient of the smaller by the larger
// magnitude, t in [0, 1], gives atan(t) from a polynomial in t^2 (our own
// near-minimax fit, atan_fit.py beside this file: 3.8e-8 rad, 1.1e-7 rad as
// evaluated in FP32), then the octant is restored: pi/2 - r where |y| > |x|,
// pi - r where x is negative (its sign bit set, so that -0 counts as
// negative, as in IEEE atan2), and the sign of y is copied onto the result
// (y = +-0 then gives +-0 or +-pi). Both zero gives +-0 or +-pi the same way.
// Accurate to about 3e-7 rad over the whole plane (tests/test_atan_fit.py).
__device__ __forceinline__ float atan2_fit(float y, float x) {
  const float ax = fabsf(x), ay = fabsf(y);
  const float hi = fmaxf(ax, ay), lo = fminf(ax, ay);
  const float t = lo * dev::rcp_ftz(fmaxf(hi, 1.17549435e-38f));
  const float s = t * t;
  float p = -4.054556135e-03f;
  p = fmaf(p, s, 2.186293714e-02f);
  p = fmaf(p, s, -5.591233820e-02f);
  p = fmaf(p, s, 9.642202407e-02f);
  p = fmaf(p, s, -1.390863359e-01f);
  p = fmaf(p, s, 1.994656771e-01f);
  p = fmaf(p, s, -3.332986236e-01f);
  p = fmaf(p, s, 9.999993443e-01f);
  float r = t * p;
  r = ay > ax ? 1.57079632679489662f - r : r;
  r = signbit(x) ? 3.14159265358979324f - r : r;
  return copysignf(r, y);
}

__device__ __forceinline__ void angles(float4 n, float& phi, float& theta) {
  phi = atan2_fit(n.y, n.x);
  phi = phi < 0.0f ? phi + 6.28318530717958647692f : phi;
  theta = atan2_fit(sqrtf(fmaf(n.x, n.x, n.y * n.y)), n.z);
}

constexpr int kSphRows = 4;  // rows per thread of the angle-image kernel
constexpr int kMsePx = 4;    // pixels per thread and step of the MSE kernel

__global__ void __launch_bounds__(kThreads)
    spherical_kernel(const float4* __restrict__ n, const uint8_t* __restrict__ valid, int H, int W,
                     long long pitch, float* __restrict__ phi, float* __restrict__ theta) {
  NRM_DEBUG_ENTRY(nullptr);
  const int x = blockIdx.x * kThreads + threadIdx.x;
  if (x >= W) return;
  // Each thread takes kSphRows rows of its column per step and issues all
  // their loads (mask byte and normal, independent of the mask) before the
  // first angle, so that several memory latencies overlap; a masked pixel's
  // stored normal is (0, 0, 0, 0).
  for (int y0 = blockIdx.y * kSphRows; y0 < H; y0 += gridDim.y * kSphRows) {
    uint8_t v[kSphRows];
    float4 nn[kSphRows];
#pragma unroll
    for (int r = 0; r < kSphRows; ++r) {
      v[r] = 0;
      nn[r] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (y0 + r < H) {
        const long long o = (long long)(y0 + r) * pitch + x;
        v[r] = __ldg(valid + o);
        nn[r] = __ldg(n + o);
      }
    }
#pragma unroll
    for (int r = 0; r < kSphRows; ++r) {
      if (y0 + r >= H) break;
      const long long o = (long long)(y0 + r) * pitch + x;
      float p = 0.0f, t = 0.0f;
      if (v[r]) angles(nn[r], p, t);
      if (NRM_GOK(phi + o, phi, dev::dbg_span(H, W, pitch, 4))) __stcs(phi + o, p);
      if (NRM_GOK(theta + o, theta, dev::dbg_span(H, W, pitch, 4))) __stcs(theta + o, t);
    }
  }
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  return v;
}

// Sums three values over the block in a fixed order; thread 0 gets the totals.
__device__ __forceinline__ void block_sum3(double& a, double& b, double& c) {
  __shared__ double s[3][kThreads / 32];
  a = warp_sum(a);
  b = warp_sum(b);
  c = warp_sum(c);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    s[0][warp] = a;
    s[1][warp] = b;
    s[2][warp] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    a = b = c = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) {
      a += s[0][w];
      b += s[1][w];
      c += s[2][w];
    }
  }
}

// Block b sums rows b, b + gridDim.x, ...; partials[3 b + {0,1,2}] =
// (sum of dtheta^2, sum of dphi^2, count).
__global__ void __launch_bounds__(kThreads)
    mse_partial_kernel(const float4* __restrict__ na, const uint8_t* __restrict__ va,
                       const float4* __restrict__ nb, const uint8_t* __restrict__ vb, int H, int W,
                       long long pitch, double* __restrict__ partials) {
  // Each thread sums its own pixels in FP32 (a few hundred terms at most for
  // frames up to 2^24 pixels: relative error ~1e-5), then the block and the
  // final pass add the per-thread sums in FP64.
  NRM_DEBUG_ENTRY(nullptr);
  float st = 0.0f, sp = 0.0f;
  int cnt = 0;
  // A thread takes kMsePx pixels of a row (kThreads apart) per step and issues
  // all their loads (masks and normals, independent of the masks) before the
  // first angle, so that the memory latencies overlap; the sums still run
  // over the thread's pixels in increasing column order.
  for (int y = blockIdx.x; y < H; y += gridDim.x) {
    const long long row = (long long)y * pitch;
    for (int x0 = threadIdx.x; x0 < W; x0 += kMsePx * kThreads) {
      uint8_t a[kMsePx], b[kMsePx];
      float4 ma[kMsePx], mb[kMsePx];
#pragma unroll
      for (int k = 0; k < kMsePx; ++k) {
        const int x = x0 + k * kThreads;
        a[k] = b[k] = 0;
        ma[k] = mb[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (x < W) {
          const long long o = row + x;
          a[k] = __ldg(va + o);
          b[k] = __ldg(vb + o);
          ma[k] = __ldg(na + o);
          mb[k] = __ldg(nb + o);
        }
      }
#pragma unroll
      for (int k = 0; k < kMsePx; ++k) {
        if (a[k] && b[k]) {
          float pa, ta, pb, tb;
          angles(ma[k], pa, ta);
          angles(mb[k], pb, tb);
          const float dt = ta - tb, dp = pa - pb;
          st = fmaf(dt, dt, st);
          sp = fmaf(dp, dp, sp);
          ++cnt;
        }
      }
    }
  }
  double dst = st, dsp = sp, dcnt = cnt;
  block_sum3(dst, dsp, dcnt);
  if (threadIdx.x == 0 && NRM_IOK(3 * (long long)blockIdx.x + 2, 3LL * kMseBlocks)) {
    partials[3 * blockIdx.x + 0] = dst;
    partials[3 * blockIdx.x + 1] = dsp;
    partials[3 * blockIdx.x + 2] = dcnt;
  }
}

__global__ void __launch_bounds__(kThreads) mse_final_kernel(const double* __restrict__ partials, int n,
                                                             double* __restrict__ out) {
  NRM_DEBUG_ENTRY(nullptr);
  double st = 0.0, sp = 0.0, cnt = 0.0;
  for (int i = threadIdx.x; i < n && NRM_IOK(3LL * i + 2, 3LL * kMseBlocks); i += kThreads) {
    st += partials[3 * i + 0];
    sp += partials[3 * i + 1];
    cnt += partials[3 * i + 2];
  }
  block_sum3(st, sp, cnt);
  if (threadIdx.x == 0) {
    out[0] = cnt > 0.0 ? st / cnt : 0.0;
    out[1] = cnt > 0.0 ? sp / cnt : 0.0;
    out[2] = cnt;
  }
}

}  // namespace

cudaError_t launch_spherical(const float* normals, const uint8_t* valid, int H, int W, long long pitch, float* phi,
                             float* theta, cudaStream_t stream) {
  const int row_steps = (H + kSphRows - 1) / kSphRows;
  dim3 grid((W + kThreads - 1) / kThreads, row_steps < 65535 ? row_steps : 65535);
  const float4* n4 = reinterpret_cast<const float4*>(normals);
  void* args[7] = {&n4, &valid, &H, &W, &pitch, &phi, &theta};
  return cudaLaunchKernel((const void*)spherical_kernel, grid, dim3(kThreads), args, 0, stream);
}

cudaError_t launch_angle_mse(const float* na, const uint8_t* va, const float* nb, const uint8_t* vb, int H, int W,
                             long long pitch, double* partials, double* out, cudaStream_t stream) {
  const float4* a4 = reinterpret_cast<const float4*>(na);
  const float4* b4 = reinterpret_cast<const float4*>(nb);
  void* pargs[8] = {&a4, &va, &b4, &vb, &H, &W, &pitch, &partials};
  cudaError_t e = cudaLaunchKernel((const void*)mse_partial_kernel, dim3(kMseBlocks), dim3(kThreads), pargs, 0, stream);
  if (e != cudaSuccess) return e;
  int nblocks = kMseBlocks;
  void* fargs[3] = {&partials, &nblocks, &out};
  return cudaLaunchKernel((const void*)mse_final_kernel, dim3(1), dim3(kThreads), fargs, 0, stream);
}

}  // namespace nrm
