// Local plane fitting ("plane-PCA"), the ground truth the paper compares
// against (arXiv 2209.08241: Section 1 describes it; Section 4 uses it with 25
// neighbouring points): for each pixel, the unit eigenvector of the scatter
// matrix of the back-projected points of its (2R+1) x (2R+1) window for the
// smallest eigenvalue, oriented away from the camera (n . P > 0).
//
// FP32 with care for cancellation: points are taken relative to the window's
// centre point P0 = z0 (u0, v0, 1) as
//   q = ((z - z0) u + z0 dcol/fx,  (z - z0) v + z0 drow/fy,  z - z0),
// whose terms are all small, so each has a relative error of a few ulp. The
// scatter matrix is then sum q q^T - (sum q)(sum q)^T / n: relative to P0 the
// window's mean is small (it is zero for the in-plane offsets of a symmetric
// window), so the subtraction loses little. The symmetric 3 x 3 eigenproblem is
// solved by cyclic Jacobi rotations until the off-diagonal part is below 1e-7
// of the diagonal (at most 6 sweeps; quadratic convergence makes 3-4 usual).
// The normal direction does not depend on the depth unit, so uint16 depth is
// used in its raw integer units (exact in FP32) without the depth scale.
// A pixel is valid iff every depth of its window is inside the image and
// positive and finite (the decoded tile holds NaN elsewhere, which propagates).
#include "nrm_device.cuh"

namespace nrm {

namespace {

constexpr int PX = 32, PY = 8, PT = PX * PY;

// One Jacobi rotation zeroing a[p][q] of the symmetric matrix a, accumulated
// into the eigenvector columns of v.
template <int p, int q>
__device__ __forceinline__ void jacobi_rotate(float (&a)[3][3], float (&v)[3][3]) {
  const float apq = a[p][q];
  if (fabsf(apq) < 1e-35f) return;
  // t = tan of the rotation angle, the smaller root of t^2 + 2 theta t - 1 = 0.
  // Approximate reciprocal and square root suffice: c and s are formed from t
  // so that c^2 + s^2 = 1 to rounding whatever t's last bits, and an error of a
  // few ulp in t only leaves an off-diagonal residue of a few ulp of |a_pq|,
  // the size of the rounding already in S.
  const float theta = __fdividef(a[q][q] - a[p][p], 2.0f * apq);
  const float at = fabsf(theta);
  float t;
  if (at > 1e18f) {
    t = __fdividef(0.5f, theta);  // theta^2 would overflow; t = 1 / (2 theta) to rounding
  } else {
    const float h = fmaf(theta, theta, 1.0f);
    t = __fdividef(copysignf(1.0f, theta), fmaf(h, rsqrtf(h), at));
  }
  const float c = rsqrtf(fmaf(t, t, 1.0f));
  const float s = t * c;
  a[p][p] -= t * apq;
  a[q][q] += t * apq;
  a[p][q] = a[q][p] = 0.0f;
  constexpr int r = 3 - p - q;
  const float arp = a[r][p], arq = a[r][q];
  a[r][p] = a[p][r] = c * arp - s * arq;
  a[r][q] = a[q][r] = s * arp + c * arq;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float vkp = v[k][p], vkq = v[k][q];
    v[k][p] = c * vkp - s * vkq;
    v[k][q] = s * vkp + c * vkq;
  }
}

template <int R>
__global__ void __launch_bounds__(PT)
    plane_fit_kernel(const __grid_constant__ FrameDesc fd, float sign) {
  constexpr int tw = PX + 2 * R, th = PY + 2 * R;
  __shared__ __align__(16) float tile[tw * th];
  NRM_DEBUG_ENTRY(nullptr);
  const int x0 = blockIdx.x * PX - R, y0 = blockIdx.y * PY - R;
  const bool u16 = fd.in_dtype == NRM_IN_U16_MM;
  for (int i = threadIdx.x; i < tw * th; i += PT) {
    const int ly = i / tw, lx = i - ly * tw;
    const int x = x0 + lx, y = y0 + ly;
    float z = __int_as_float(0x7fc00000);
    if (x >= 0 && y >= 0 && x < fd.W && y < fd.H) {
      const long long o = (long long)y * fd.depth_pitch + x;
      z = u16 ? dev::decode_depth_u16(__ldg(reinterpret_cast<const uint16_t*>(fd.depth) + o))
              : dev::decode_depth(__ldg(reinterpret_cast<const float*>(fd.depth) + o));
    }
    if (NRM_IOK(i, tw * th)) tile[i] = z;
  }
  __syncthreads();
  const int lx = threadIdx.x & (PX - 1), ly = threadIdx.x / PX;
  const int px = blockIdx.x * PX + lx, py = blockIdx.y * PY + ly;
  if (px >= fd.W || py >= fd.H) return;
  const int ci = (ly + R) * tw + (lx + R);
  const float* c0 = tile + ci;
  const float z0 = NRM_IOK(ci, tw * th) ? c0[0] : 0.0f;
  const float u0 = ((float)px - fd.cx) * fd.inv_fx, v0 = ((float)py - fd.cy) * fd.inv_fy;
  float sx = 0.f, sy = 0.f, sz = 0.f;
  float a00 = 0.f, a01 = 0.f, a02 = 0.f, a11 = 0.f, a12 = 0.f, a22 = 0.f;
#pragma unroll
  for (int dy = -R; dy <= R; ++dy) {
    const float v = v0 + (float)dy * fd.inv_fy;
    const float ey = z0 * ((float)dy * fd.inv_fy);
#pragma unroll
    for (int dx = -R; dx <= R; ++dx) {
      const float dz = (NRM_IOK(ci + dy * tw + dx, tw * th) ? c0[dy * tw + dx] : 0.0f) - z0;
      const float qx = fmaf(dz, u0 + (float)dx * fd.inv_fx, z0 * ((float)dx * fd.inv_fx));
      const float qy = fmaf(dz, v, ey);
      sx += qx;
      sy += qy;
      sz += dz;
      a00 = fmaf(qx, qx, a00);
      a01 = fmaf(qx, qy, a01);
      a02 = fmaf(qx, dz, a02);
      a11 = fmaf(qy, qy, a11);
      a12 = fmaf(qy, dz, a12);
      a22 = fmaf(dz, dz, a22);
    }
  }
  const long long oo = (long long)py * fd.out_pitch + px;
  float4* out = reinterpret_cast<float4*>(fd.normals) + oo;
  [[maybe_unused]] const long long nlen = dev::dbg_span(fd.H, fd.W, fd.out_pitch, 16);
  [[maybe_unused]] const long long mlen = dev::dbg_span(fd.H, fd.W, fd.out_pitch, 1);
  if (!(fabsf(sx) + fabsf(sy) + fabsf(sz) <= 3.402823466e38f)) {  // a NaN depth in the window
    if (NRM_GOK(out, fd.normals, nlen)) *out = make_float4(0.f, 0.f, 0.f, 0.f);
    if (NRM_GOK(fd.valid + oo, fd.valid, mlen)) fd.valid[oo] = 0;
    return;
  }
  constexpr float inv_n = 1.0f / (float)((2 * R + 1) * (2 * R + 1));
  const float mx = sx * inv_n, my = sy * inv_n, mz = sz * inv_n;
  float a[3][3];
  a[0][0] = fmaf(-mx, sx, a00);
  a[0][1] = a[1][0] = fmaf(-mx, sy, a01);
  a[0][2] = a[2][0] = fmaf(-mx, sz, a02);
  a[1][1] = fmaf(-my, sy, a11);
  a[1][2] = a[2][1] = fmaf(-my, sz, a12);
  a[2][2] = fmaf(-mz, sz, a22);
  float vec[3][3] = {{1.f, 0.f, 0.f}, {0.f, 1.f, 0.f}, {0.f, 0.f, 1.f}};
#pragma unroll 1
  for (int sweep = 0; sweep < 6; ++sweep) {
    jacobi_rotate<0, 1>(a, vec);
    jacobi_rotate<0, 2>(a, vec);
    jacobi_rotate<1, 2>(a, vec);
    const float off = fmaf(a[0][1], a[0][1], fmaf(a[0][2], a[0][2], a[1][2] * a[1][2]));
    const float diag = fmaf(a[0][0], a[0][0], fmaf(a[1][1], a[1][1], a[2][2] * a[2][2]));
    if (off <= 1e-14f * diag) break;
  }
  // Column of the smallest diagonal entry, chosen by selects (no dynamic indexing).
  float nx = vec[0][0], ny = vec[1][0], nz = vec[2][0], lmin = a[0][0];
  if (a[1][1] < lmin) {
    lmin = a[1][1];
    nx = vec[0][1];
    ny = vec[1][1];
    nz = vec[2][1];
  }
  if (a[2][2] < lmin) {
    nx = vec[0][2];
    ny = vec[1][2];
    nz = vec[2][2];
  }
  const float inv = rsqrtf(fmaf(nx, nx, fmaf(ny, ny, nz * nz)));
  // Away from the camera (n . (u0, v0, 1) > 0), then the caller's orientation.
  const float o = (fmaf(nx, u0, fmaf(ny, v0, nz)) < 0.0f ? -inv : inv) * sign;
  if (NRM_GOK(out, fd.normals, nlen)) *out = make_float4(nx * o, ny * o, nz * o, 0.0f);
  if (NRM_GOK(fd.valid + oo, fd.valid, mlen)) fd.valid[oo] = 1;
}

}  // namespace

cudaError_t launch_plane_fit(const FrameDesc& fd, int radius, float sign, cudaStream_t stream) {
  dim3 grid((fd.W + PX - 1) / PX, (fd.H + PY - 1) / PY);
  const void* fn = nullptr;
  switch (radius) {
    case 1: fn = (const void*)plane_fit_kernel<1>; break;
    case 2: fn = (const void*)plane_fit_kernel<2>; break;
    case 3: fn = (const void*)plane_fit_kernel<3>; break;
    case 4: fn = (const void*)plane_fit_kernel<4>; break;
    default: return cudaErrorInvalidValue;
  }
  FrameDesc d = fd;
  float sg = sign;
  void* args[2] = {&d, &sg};
  return cudaLaunchKernel(fn, grid, dim3(PT), args, 0, stream);
}

}  // namespace nrm
