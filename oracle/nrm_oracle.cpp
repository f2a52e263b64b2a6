// FP64 CPU oracle for boundary-aware surface-normal estimation from depth maps
// (Moradi, Memarmoghadam and Laurendeau, "Fast, Accurate and Object
// Boundary-Aware Surface Normal Estimation from Depth Maps", arXiv 2209.08241).
//
// TEST INFRASTRUCTURE. This file is the slow, obviously correct statement of
// what the GPU path must compute. Only the test suite, the package smoke check
// and the benchmark's CPU-baseline leg may load it. It shares no code, header,
// constant or helper with the CUDA library and includes nothing from it.
//
// What it follows, step by step:
//   * Section 2, definitions below Eq. 3: d_i = g(r_i, c_i), u_i = (. - o_x)/f_x,
//     v_i = (. - o_y)/f_y. Section 3.1, the s24 / s35 vectors: a pixel with depth d
//     back-projects to P = (u d, v d, d).
//   * Section 3.1 and Fig. 2: four "main direction" neighbours at pixel distance
//     alpha. Point 2 = +alpha along u (the column), 3 = +alpha along v (the row),
//     4 = -alpha along u, 5 = -alpha along v. (The figure is missing from the
//     text; this is the only layout for which Eq. 1-3 equal s12 x s13 and
//     Eq. 4-6 equal 1/4 s24 x s35. The tests pin it.)
//   * Section 3.1, Eq. "proof of efficiency", first two lines: n is the average of
//     the four perpendicular tangent-pair cross products
//     s12 x s13 + s13 x s14 + s14 x s15 + s15 x s12. The oracle evaluates this
//     DIRECT form; it never uses the reformulation 1/4 s24 x s35 or Eq. 4-6.
//   * Section 3.2, Eq. "veclength": r = ||n||_2 grows at depth discontinuities;
//     thresholding r gives the outlier mask, which is applied to the normal map
//     (Section 4, Fig. 8).
//
// Readings where the paper is silent (each listed in the design notes):
//   * border: a pixel within alpha of an image edge has a neighbour outside the
//     image and is invalid;
//   * invalid depth: any of d1..d5 equal to 0, negative or non-finite makes the
//     pixel invalid (d1 is checked although the closed form does not use it);
//   * statistic: mode RAW uses r itself (the paper's literal statistic, in m^2);
//     mode SECANT uses r * ||ray|| / (n . ray) with ray = (u1, v1, 1), the
//     depth-invariant 1/cos of the angle between the normal and the viewing ray;
//   * threshold: a pixel is valid iff stat <= tau;
//   * masked pixels carry the normal (0, 0, 0);
//   * sign: the paper's normal satisfies n . P1 > 0 (it points away from the
//     camera); orient = 1 negates the unit normal.
// The value of tau and the zero-normal convention for masked pixels are
// conventions, not facts from the paper: parity unpinned for those two choices.
//
// Gradient: nrm_oracle_vjp differentiates the same direct-form code by the
// complex-step method (perturb one depth by i*h, read the imaginary part), with
// the validity mask held fixed. It contains no hand-derived derivative.

#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <limits>
#include <thread>
#include <vector>

namespace {

enum { DEPTH_F32 = 0, DEPTH_U16 = 1, DEPTH_F64 = 2 };
enum { STAT_RAW = 0, STAT_SECANT = 1 };

template <class T>
struct Vec3 {
  T x, y, z;
};

template <class T>
Vec3<T> operator+(const Vec3<T>& a, const Vec3<T>& b) {
  return {a.x + b.x, a.y + b.y, a.z + b.z};
}

template <class T>
Vec3<T> operator-(const Vec3<T>& a, const Vec3<T>& b) {
  return {a.x - b.x, a.y - b.y, a.z - b.z};
}

template <class T>
Vec3<T> scaled(const Vec3<T>& a, T s) {
  return {a.x * s, a.y * s, a.z * s};
}

template <class T>
Vec3<T> cross(const Vec3<T>& a, const Vec3<T>& b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

template <class T>
T dot(const Vec3<T>& a, const Vec3<T>& b) {
  return a.x * b.x + a.y * b.y + a.z * b.z;
}

struct Camera {
  double fx, fy, cx, cy;
};

struct Frame {
  const void* depth;
  int dtype;
  int H, W;
  long long pitch;  // elements between rows
  double depth_scale;
};

// Depth g(row, col) in metres, or ok = false when the pixel is outside the image
// or its depth is not a positive finite number.
double read_depth(const Frame& f, int col, int row, bool* ok) {
  if (col < 0 || row < 0 || col >= f.W || row >= f.H) {
    *ok = false;
    return 0.0;
  }
  long long i = (long long)row * f.pitch + col;
  double d;
  if (f.dtype == DEPTH_F32) {
    d = (double)((const float*)f.depth)[i];
  } else if (f.dtype == DEPTH_U16) {
    d = (double)((const uint16_t*)f.depth)[i] * f.depth_scale;
  } else {
    d = ((const double*)f.depth)[i];
  }
  *ok = std::isfinite(d) && d > 0.0;
  return d;
}

// P = d * (u, v, 1) with u = (col - cx)/fx, v = (row - cy)/fy.
template <class T>
Vec3<T> back_project(T d, int col, int row, const Camera& K) {
  double u = ((double)col - K.cx) / K.fx;
  double v = ((double)row - K.cy) / K.fy;
  return {T(u) * d, T(v) * d, d};
}

// Section 3.1, first two lines of the "proof of efficiency" equation:
// n = 1/4 (s12 x s13 + s13 x s14 + s14 x s15 + s15 x s12), s1k = Pk - P1.
// d[0..4] hold d1..d5.
template <class T>
Vec3<T> multi_direction_normal(const T d[5], int col, int row, int alpha, const Camera& K) {
  Vec3<T> P1 = back_project(d[0], col, row, K);
  Vec3<T> P2 = back_project(d[1], col + alpha, row, K);
  Vec3<T> P3 = back_project(d[2], col, row + alpha, K);
  Vec3<T> P4 = back_project(d[3], col - alpha, row, K);
  Vec3<T> P5 = back_project(d[4], col, row - alpha, K);
  Vec3<T> s12 = P2 - P1;
  Vec3<T> s13 = P3 - P1;
  Vec3<T> s14 = P4 - P1;
  Vec3<T> s15 = P5 - P1;
  Vec3<T> sum = cross(s12, s13) + cross(s13, s14) + cross(s14, s15) + cross(s15, s12);
  return scaled(sum, T(0.25));
}

struct Params {
  int alpha;
  int stat_mode;
  double tau;
  int orient;
};

struct PixelResult {
  double n[3];     // unnormalised multi-direction normal
  double nhat[3];  // unit normal, zero when masked
  double r;        // ||n||_2 (NaN when the stencil is invalid)
  double stat;     // the thresholded statistic (NaN when the stencil is invalid)
  uint8_t valid;
};

// Reads the five stencil depths of pixel (col, row). Returns false if any of
// them is outside the image or not a valid depth.
bool gather_stencil(const Frame& f, int col, int row, int alpha, double d[5]) {
  bool ok[5];
  d[0] = read_depth(f, col, row, &ok[0]);
  d[1] = read_depth(f, col + alpha, row, &ok[1]);
  d[2] = read_depth(f, col, row + alpha, &ok[2]);
  d[3] = read_depth(f, col - alpha, row, &ok[3]);
  d[4] = read_depth(f, col, row - alpha, &ok[4]);
  return ok[0] && ok[1] && ok[2] && ok[3] && ok[4];
}

PixelResult evaluate_pixel(const Frame& f, const Camera& K, const Params& p, int col, int row) {
  PixelResult out;
  std::memset(&out, 0, sizeof(out));
  const double nan = std::numeric_limits<double>::quiet_NaN();
  double d[5];
  if (!gather_stencil(f, col, row, p.alpha, d)) {
    out.r = nan;
    out.stat = nan;
    out.valid = 0;
    return out;
  }
  Vec3<double> n = multi_direction_normal<double>(d, col, row, p.alpha, K);
  out.n[0] = n.x;
  out.n[1] = n.y;
  out.n[2] = n.z;
  // Section 3.2: r, the length of the estimated normal vector.
  double r = std::sqrt(dot(n, n));
  out.r = r;
  double stat;
  if (p.stat_mode == STAT_RAW) {
    stat = r;
  } else {
    Vec3<double> ray = {((double)col - K.cx) / K.fx, ((double)row - K.cy) / K.fy, 1.0};
    double along = dot(n, ray);
    stat = along > 0.0 ? r * std::sqrt(dot(ray, ray)) / along
                       : std::numeric_limits<double>::infinity();
  }
  out.stat = stat;
  // Section 3.2 / Fig. 8: threshold the statistic, apply the mask to the normals.
  out.valid = (r > 0.0 && stat <= p.tau) ? 1 : 0;
  if (out.valid) {
    double s = (p.orient ? -1.0 : 1.0) / r;
    out.nhat[0] = n.x * s;
    out.nhat[1] = n.y * s;
    out.nhat[2] = n.z * s;
  }
  return out;
}

template <class Fn>
void parallel_rows(int row0, int row1, int nthreads, Fn fn) {
  int rows = row1 - row0;
  if (rows <= 0) return;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > rows) nthreads = rows;
  if (nthreads == 1) {
    fn(row0, row1);
    return;
  }
  std::vector<std::thread> pool;
  int per = (rows + nthreads - 1) / nthreads;
  for (int t = 0; t < nthreads; ++t) {
    int a = row0 + t * per;
    int b = a + per < row1 ? a + per : row1;
    if (a >= b) break;
    pool.emplace_back([=]() { fn(a, b); });
  }
  for (auto& th : pool) th.join();
}

// Unit normal of pixel (col, row) as a function of a complex-perturbed depth
// map: depth (qcol, qrow) is replaced by its value plus i*h. ||n|| is the
// analytic sqrt(n . n), so the result is holomorphic in the perturbation.
Vec3<std::complex<double>> perturbed_unit_normal(const Frame& f, const Camera& K, const Params& p,
                                                 int col, int row, int qcol, int qrow, double h) {
  typedef std::complex<double> C;
  double dr[5];
  gather_stencil(f, col, row, p.alpha, dr);
  const int cols[5] = {col, col + p.alpha, col, col - p.alpha, col};
  const int rows[5] = {row, row, row + p.alpha, row, row - p.alpha};
  C d[5];
  for (int k = 0; k < 5; ++k) {
    d[k] = C(dr[k], (cols[k] == qcol && rows[k] == qrow) ? h : 0.0);
  }
  Vec3<C> n = multi_direction_normal<C>(d, col, row, p.alpha, K);
  C len = std::sqrt(dot(n, n));
  C s = C(p.orient ? -1.0 : 1.0) / len;
  return scaled(n, s);
}

}  // namespace

extern "C" {

// Forward oracle over rows [row0, row1) of one depth map.
//   depth:      H x W depth map, row pitch `pitch` elements; dtype 0 = float32
//               metres, 1 = uint16 (metres = raw * depth_scale), 2 = float64 metres.
//   K:          fx, fy, cx, cy (pixels).
//   alpha:      pixel distance (>= 1).
//   stat_mode:  0 = RAW (r), 1 = SECANT (r ||ray|| / (n . ray)).
//   tau:        a pixel is valid iff its statistic is <= tau.
//   orient:     0 = paper sign (n . P1 > 0), 1 = negated.
// Outputs are full-frame H*W arrays (row-major, pitch W); only rows
// [row0, row1) are written. Any output pointer may be NULL.
//   n_raw, n_hat: H*W*3 doubles; r, stat: H*W doubles; valid: H*W bytes.
// Returns 0, or -1 on invalid arguments.
int nrm_oracle_forward(const void* depth, int dtype, int H, int W, long long pitch,
                       const double* K4, int alpha, int stat_mode, double tau,
                       double depth_scale, int orient, int row0, int row1,
                       double* n_raw, double* n_hat, double* r, double* stat,
                       uint8_t* valid, int nthreads) {
  if (H < 0 || W < 0 || alpha < 1 || pitch < W || K4 == nullptr) return -1;
  if (dtype < DEPTH_F32 || dtype > DEPTH_F64) return -1;
  if (stat_mode != STAT_RAW && stat_mode != STAT_SECANT) return -1;
  if (row0 < 0) row0 = 0;
  if (row1 > H) row1 = H;
  if (H > 0 && W > 0 && depth == nullptr) return -1;
  Frame f = {depth, dtype, H, W, pitch, depth_scale};
  Camera K = {K4[0], K4[1], K4[2], K4[3]};
  Params p = {alpha, stat_mode, tau, orient};
  parallel_rows(row0, row1, nthreads, [&](int a, int b) {
    for (int row = a; row < b; ++row) {
      for (int col = 0; col < W; ++col) {
        PixelResult px = evaluate_pixel(f, K, p, col, row);
        long long i = (long long)row * W + col;
        if (n_raw) {
          n_raw[3 * i + 0] = px.n[0];
          n_raw[3 * i + 1] = px.n[1];
          n_raw[3 * i + 2] = px.n[2];
        }
        if (n_hat) {
          n_hat[3 * i + 0] = px.nhat[0];
          n_hat[3 * i + 1] = px.nhat[1];
          n_hat[3 * i + 2] = px.nhat[2];
        }
        if (r) r[i] = px.r;
        if (stat) stat[i] = px.stat;
        if (valid) valid[i] = px.valid;
      }
    }
  });
  return 0;
}

// Vector-Jacobian product of the unit normal map with respect to depth, with the
// validity mask held fixed, by complex-step differentiation of the direct form.
//   grad[q] = sum over valid pixels p whose stencil contains q of
//             g[p] . d(n_hat[p]) / d(depth[q]),
// for every q in the crop rows [y0, y0+h) x cols [x0, x0+w).
//   depth: dtype 0 (float32) or 2 (float64), H x W, pitch elements.
//   g:     H*W*3 doubles (upstream gradient dL/dn_hat, pitch W).
//   valid: H*W bytes (pitch W), the fixed mask.
//   grad:  h*w doubles (pitch w).
//   step:  the complex step (e.g. 1e-30).
int nrm_oracle_vjp(const void* depth, int dtype, int H, int W, long long pitch,
                   const double* K4, int alpha, int orient, const double* g,
                   const uint8_t* valid, int y0, int x0, int h, int w, double* grad,
                   double step, int nthreads) {
  if (dtype != DEPTH_F32 && dtype != DEPTH_F64) return -1;
  if (H < 0 || W < 0 || alpha < 1 || pitch < W || h < 0 || w < 0) return -1;
  if (y0 < 0 || x0 < 0 || y0 + h > H || x0 + w > W) return -1;
  if (!(step > 0.0)) return -1;
  Frame f = {depth, dtype, H, W, pitch, 1.0};
  Camera K = {K4[0], K4[1], K4[2], K4[3]};
  Params p = {alpha, STAT_RAW, 0.0, orient};
  parallel_rows(y0, y0 + h, nthreads, [&](int a, int b) {
    for (int qrow = a; qrow < b; ++qrow) {
      for (int qcol = x0; qcol < x0 + w; ++qcol) {
        // Pixels whose five-point stencil contains q.
        const int pc[5] = {qcol, qcol - alpha, qcol, qcol + alpha, qcol};
        const int pr[5] = {qrow, qrow, qrow - alpha, qrow, qrow + alpha};
        double acc = 0.0;
        for (int k = 0; k < 5; ++k) {
          int col = pc[k], row = pr[k];
          if (col < 0 || row < 0 || col >= W || row >= H) continue;
          long long ip = (long long)row * W + col;
          if (!valid[ip]) continue;
          Vec3<std::complex<double>> nh = perturbed_unit_normal(f, K, p, col, row, qcol, qrow, step);
          acc += (g[3 * ip + 0] * nh.x.imag() + g[3 * ip + 1] * nh.y.imag() +
                  g[3 * ip + 2] * nh.z.imag()) / step;
        }
        grad[(long long)(qrow - y0) * w + (qcol - x0)] = acc;
      }
    }
  });
  return 0;
}

}  // extern "C"
