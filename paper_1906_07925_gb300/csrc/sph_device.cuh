// Device-side building blocks of the sm_103a relaxation step: parameter blocks
// passed by value to kernels, the Wendland C2 kernel, the analytic target field,
// the level set and its projection, the split-precision cell frame, and the
// Philox4x32-10 counter-based generator used by the initial sampling.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace sph {

constexpr int kMaxLevels = 8;
constexpr int kMaxShapes = 4;
constexpr int kMaxListCapacity = 0x7FFF;  // neighbour-list entries per particle (15-bit counts)
// Staged pass A (FP32, 256-target blocks): the distinct neighbours of a block's
// lists are gathered into shared memory once per step, at most kStageCap of
// them (40 KB of views); kStageHash slots of the hash set that finds them
constexpr int kStageBlock = 256;
constexpr int kStageCap = 2560;
constexpr int kStageHash = 4096;

// error bits latched in the device error word (1 << sph_status value)
constexpr int kErrNonfinite = 1 << 4;
constexpr int kErrOutOfDomain = 1 << 5;
constexpr int kErrListOverflow = 1 << 6;
constexpr int kErrTimeout = 1 << 7;

template <class T>
struct alignas(sizeof(T) * 4) V4 {
  T x, y, z, w;
};

// Geometry + target field (Sec. 2.3, 3.1, 3.2) in the working precision T.
template <class T>
struct Geom {
  int dim, n_shapes, field_kind, dist_shape, n_poly;
  int kind[kMaxShapes], keep_inside[kMaxShapes];
  T lo[3], hi[3], ext[3];
  T center[kMaxShapes][3], size[kMaxShapes][3];
  T s0, a, b;
  T poly[8];
  T hfac;      // tau * rho_scale^(-1/d): h = hfac * s * (1 + P)^(-1/d)
  T rho_scale;
  // Cartesian background mesh (Sec. 3.1, 3.2): node values (x fastest) of the
  // level set (shapes of kind 2) and of the target spacing (field kind 3);
  // device pointers, null when unused
  const double* bg_phi;
  const double* bg_s;
  int bg_n[3];
  T bg_lo[3], bg_h[3], bg_inv_h[3];
};

// Multi-resolution cell grid. Level l has cells of edge c0 2^l; a particle is
// filed at the level of its smoothing length. Positions are integers (see
// Frame), so the level-l cell index of a coordinate X is X >> (cshift + l).
template <class T>
struct Grid {
  int n_levels, dim, cshift;
  int nx[kMaxLevels], ny[kMaxLevels], nz[kMaxLevels];
  uint32_t base[kMaxLevels + 1];
  T cellv[kMaxLevels];   // cell edge in view units
  T inv_h0;              // level(h) = floor(log2(h / h0)), h physical
  T lip_h;               // |grad h| bound: neighbours' h within h_i +- lip_h r
  T rfac;                // kappa h_i rfac covers r < kappa max(h_i, h_j)
};

// Position frames. The state of a particle is an int64 coordinate per axis,
// X = (x - lo) / q64, exact and independent of the level. Pair arithmetic
// uses a "view" refreshed every step: for FP32, the low 32 bits of X >> sv
// (differences taken modulo 2^32 are exact for nearby particles, whatever the
// domain size); for FP64, physical coordinates relative to lo.
template <class T>
struct Frame {
  double q64, inv_q64;   // physical length of one state unit and its inverse
  double s2v;            // state units -> view units (2^-cshift)
  double lod[3];         // box origin
  long long xmax[3];     // state coordinate of the upper box face
  int sv;                // FP32 view integer = round(X / 2^sv) = 2^-kViewBits c0
  int mbits;             // FP32: bits of 1.5 * 2^(23 - kCoarseBits); adding d encodes d 2^-kCoarseBits
  float mbias;           // FP32: 1.5 * 2^(23 - kCoarseBits)
  float vscale;          // FP32: 2^-kViewBits, one view integer in view units
  T qv, inv_qv;          // physical length of one view unit (the finest cell edge c0)
  T q64t, inv_q64t;
  T lo[3];
  T skin;                // list skin as a fraction of kappa h
};

// The view unit is the level-0 cell edge c0. FP32 view integers are 2^-24 c0;
// the coarse inside/outside test of a listed pair uses them shifted down to
// 2^-16 c0, whose differences convert exactly without the conversion unit
// while they stay below 2^22 coarse integers = 64 c0 per axis: every list of
// the coarser levels qualifies (a list whose pairs reach beyond that range
// takes the exact test alone).
constexpr int kViewBits = 24;
constexpr int kCoarseBits = 16;

template <class T>
struct Phys {
  T P0, gamma, kappa, inv_tau;
  T alpha;  // dimensionless Wendland constant: 7/pi (2D), 21/(2 pi) (3D)
};

// Per-block partials of the pass-A reductions (FP64), reduced in fixed order.
struct Partial {
  double min_rc_a, max_a, sum_rho, err_l2, err_max;
  long long ipairs, fpairs;
  long long lentries;  // neighbour-list entries scanned
  long long amin;      // index (current order) of min_rc_a; -1: none
};

// Step scalars written by the last block of pass A, read by pass B.
struct Scalars {
  double dt1, dt2, min_rc_a, max_a, sum_rho, err_l2, err_max, sigma;
  long long ipairs, fpairs, wall_moved, step_of_stats;
  long long lentries;
  long long argmin;  // particle (current order) where min r_c/|a| sits; -1: none
};

// Surface-tension schedule (Eq. sph_st_sigma), step counter and the
// neighbour-list bookkeeping. `buf` selects the buffer holding the state in its
// current order, `vp` the current view buffer; `need_rebuild` is raised by
// pass B when a particle has moved half its skin since the list was built.
struct StepCtl {
  long long step;
  double t0, t1, sigma0;
  int buf, vp, rebuild, need_rebuild;
  int lmax, pad_;  // longest neighbour list of the last build
  long long rebuilds;
  // automatic start of the ramp (Sec. 3.3 convergence test): on, run length in
  // steps, relative tolerance, ramp fraction; state: current run, its opening
  // count (-1: none yet), fired
  int auto_on, auto_window, auto_stable, auto_done;
  double auto_tol, auto_theta;
  long long auto_ref;
  // step-size history of a reverse-pass run (device array of {dt1, dt2} per
  // step, step counter dt_base at entry 0): mode 1 records the sizes each step
  // chose, mode 2 makes each step use the recorded ones; 0: neither
  double* dt_hist;
  long long dt_base;
  int dt_len, dt_mode;
};

__device__ __forceinline__ double sigma_of(const StepCtl& c, long long t) {
  if (c.t0 < 0.0 || (double)t <= c.t0) return c.sigma0;
  if ((double)t <= c.t1) return c.sigma0 * (1.0 - (c.t0 - (double)t) / (c.t0 - c.t1));
  return 0.0;
}

// ---------------------------------------------------------------- math ----

template <class T> __device__ __forceinline__ T dsqrt(T x);
template <> __device__ __forceinline__ float dsqrt<float>(float x) { return sqrtf(x); }
template <> __device__ __forceinline__ double dsqrt<double>(double x) { return sqrt(x); }

template <class T> __device__ __forceinline__ T drsqrt(T x);
template <> __device__ __forceinline__ float drsqrt<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double drsqrt<double>(double x) { return rsqrt(x); }

template <class T> __device__ __forceinline__ T drcp(T x);
template <> __device__ __forceinline__ float drcp<float>(float x) { return __fdividef(1.0f, x); }
template <> __device__ __forceinline__ double drcp<double>(double x) { return 1.0 / x; }

template <class T> __device__ __forceinline__ T dfloor(T x);
template <> __device__ __forceinline__ float dfloor<float>(float x) { return floorf(x); }
template <> __device__ __forceinline__ double dfloor<double>(double x) { return floor(x); }

// small integer -> floating point without the conversion unit:
// for |v| < 2^22, the bit pattern of 1.5*2^23 + v read as a float is exactly
// 12582912 + v (the integer lands in the low mantissa bits).
template <class T> __device__ __forceinline__ T small_int_to_fp(int v);
template <> __device__ __forceinline__ float small_int_to_fp<float>(int v) {
  return __int_as_float(0x4B400000 + v) - 12582912.0f;
}
template <> __device__ __forceinline__ double small_int_to_fp<double>(int v) {
  return __longlong_as_double(0x4338000000000000LL + (long long)v) - 6755399441055744.0;
}

template <int D, class T>
__device__ __forceinline__ T pow_d(T x) {  // x^D
  return D == 2 ? x * x : x * x * x;
}

// (h / tau)^(2D) = 1 / rho_t^2 (unit mass, h = tau rho_t^(-1/d))
template <int D, class T>
__device__ __forceinline__ T inv_rho_t2(T h, T inv_tau) {
  T t = h * inv_tau;
  T t2 = t * t;
  return D == 2 ? t2 * t2 : t2 * t2 * t2;
}

// ------------------------------------------------------------ geometry ----

// Node values v of the background mesh interpolated at x: multilinear
// (bilinear in 2D, trilinear in 3D) in the mesh cell that holds x, x clamped
// into the mesh box; grad (may be null) receives the interpolant's gradient.
template <class T>
__device__ __forceinline__ T bg_interp(const Geom<T>& g, const double* __restrict__ v, const T* x, int dim,
                                       T* grad) {
  int i0[3] = {0, 0, 0};
  T f[3] = {0, 0, 0};
  for (int k = 0; k < dim; ++k) {
    const int n = g.bg_n[k];
    T t = (x[k] - g.bg_lo[k]) * g.bg_inv_h[k];
    t = t < T(0) ? T(0) : (t > T(n - 1) ? T(n - 1) : t);
    int i = (int)dfloor(t);
    i = i > n - 2 ? n - 2 : i;
    i0[k] = i;
    f[k] = t - (T)i;
  }
  T val = 0, gr[3] = {0, 0, 0};
  for (int c = 0; c < (1 << dim); ++c) {
    long long idx = 0, stride = 1;
    T w = 1, dw[3] = {1, 1, 1};
    for (int k = 0; k < dim; ++k) {
      const int b = (c >> k) & 1;
      idx += (long long)(i0[k] + b) * stride;
      stride *= g.bg_n[k];
      const T wk = b ? f[k] : T(1) - f[k];
      const T dk = (b ? T(1) : T(-1)) * g.bg_inv_h[k];
      for (int m = 0; m < dim; ++m) dw[m] *= (m == k) ? dk : wk;
      w *= wk;
    }
    const T node = (T)v[idx];
    val += w * node;
    for (int m = 0; m < dim; ++m) gr[m] += dw[m] * node;
  }
  if (grad)
    for (int k = 0; k < 3; ++k) grad[k] = k < dim ? gr[k] : T(0);
  return val;
}

// signed distance, positive inside shape s (kind 2: the background level set)
template <class T>
__device__ __forceinline__ T shape_inside(const Geom<T>& g, int s, const T* x, int dim) {
  if (g.kind[s] == 2) return bg_interp(g, g.bg_phi, x, dim, (T*)nullptr);
  if (g.kind[s] == 0) {
    T r2 = 0;
    for (int k = 0; k < dim; ++k) {
      T d = x[k] - g.center[s][k];
      r2 += d * d;
    }
    return g.size[s][0] - dsqrt(r2);
  }
  T out2 = 0, qmax = -1e30;
  for (int k = 0; k < dim; ++k) {
    T q = fabs(x[k] - g.center[s][k]) - g.size[s][k];
    if (q > 0) out2 += q * q;
    qmax = q > qmax ? q : qmax;
  }
  T inside = qmax < 0 ? qmax : T(0);
  return -(dsqrt(out2) + inside);
}

template <class T>
__device__ __forceinline__ T constraint_phi(const Geom<T>& g, int s, const T* x, int dim) {
  T v = shape_inside(g, s, x, dim);
  return g.keep_inside[s] ? v : -v;
}

// Eq. displacement_surface for one shape constraint violated at x (phi < 0):
// move to the closest point of its surface. Returns 1 if x moved.
template <class T>
__device__ __forceinline__ int project_shape(const Geom<T>& g, int s, T* x, int dim) {
  if (!(constraint_phi(g, s, x, dim) < 0)) return 0;
  if (g.kind[s] == 2) {
    // interpolated level set: three Newton steps x <- x - phi grad / |grad|^2
    // (the printed step when |grad phi| = 1)
    const T sg = g.keep_inside[s] ? T(1) : T(-1);
    for (int it = 0; it < 3; ++it) {
      T gr[3];
      const T v = sg * bg_interp(g, g.bg_phi, x, dim, gr);
      T g2 = 0;
      for (int k = 0; k < dim; ++k) g2 += gr[k] * gr[k];
      if (!(g2 > T(0))) break;
      for (int k = 0; k < dim; ++k) x[k] -= v * sg * gr[k] / g2;
    }
    return 1;
  }
  if (g.kind[s] == 0) {
    T d[3] = {0, 0, 0}, r2 = 0;
    for (int k = 0; k < dim; ++k) {
      d[k] = x[k] - g.center[s][k];
      r2 += d[k] * d[k];
    }
    T r = dsqrt(r2);
    if (r == 0) {
      d[0] = 1;
      r = 1;
    }
    for (int k = 0; k < dim; ++k) x[k] = g.center[s][k] + g.size[s][0] * d[k] / r;
    return 1;
  }
  if (g.keep_inside[s]) {
    for (int k = 0; k < dim; ++k) {
      T lo = g.center[s][k] - g.size[s][k], hi = g.center[s][k] + g.size[s][k];
      x[k] = x[k] < lo ? lo : (x[k] > hi ? hi : x[k]);
    }
    return 1;
  }
  int best = 0;
  T bestd = 1e30, sign = 1;
  for (int k = 0; k < dim; ++k) {
    T dlo = x[k] - (g.center[s][k] - g.size[s][k]);
    T dhi = (g.center[s][k] + g.size[s][k]) - x[k];
    if (dlo < bestd) { bestd = dlo; best = k; sign = -1; }
    if (dhi < bestd) { bestd = dhi; best = k; sign = 1; }
  }
  x[best] = g.center[s][best] + sign * g.size[s][best];
  return 1;
}

// ------------------------------------------- feature-surface particles ----
// Sec. 3.5: a feature-surface particle belongs to the constraint surface
// nearest to it (constraint value of smallest magnitude, the bounding box
// first on ties); N is that constraint's unit normal, the gradient of its
// signed distance (pointing into the region).
constexpr uint32_t kSurfaceBit = 0x100u;  // in the particle's meta word, above its colour

// signed distance inside the bounding box and its gradient
template <class T>
__device__ __forceinline__ T box_inside(const Geom<T>& g, const T* x, int dim, T* gr) {
  T q[3] = {0, 0, 0}, out2 = 0, qmax = T(-1e30);
  int kmax = 0;
  for (int k = 0; k < dim; ++k) {
    const T c = T(0.5) * (g.lo[k] + g.hi[k]);
    q[k] = fabs(x[k] - c) - T(0.5) * (g.hi[k] - g.lo[k]);
    if (q[k] > 0) out2 += q[k] * q[k];
    if (q[k] > qmax) { qmax = q[k]; kmax = k; }
  }
  for (int k = 0; k < 3; ++k) gr[k] = T(0);
  const T o = dsqrt(out2);
  if (out2 > 0) {
    for (int k = 0; k < dim; ++k)
      if (q[k] > 0) gr[k] = -q[k] * (x[k] >= T(0.5) * (g.lo[k] + g.hi[k]) ? T(1) : T(-1)) / o;
  } else if (qmax < 0) {
    gr[kmax] = -(x[kmax] >= T(0.5) * (g.lo[kmax] + g.hi[kmax]) ? T(1) : T(-1));
  }
  return -(o + (qmax < 0 ? qmax : T(0)));
}

// gradient of shape s's signed inside distance (the branch the value takes)
template <class T>
__device__ __forceinline__ void shape_grad(const Geom<T>& g, int s, const T* x, int dim, T* gr) {
  for (int k = 0; k < 3; ++k) gr[k] = T(0);
  if (g.kind[s] == 2) {
    bg_interp(g, g.bg_phi, x, dim, gr);
    return;
  }
  if (g.kind[s] == 0) {
    T r2 = 0;
    for (int k = 0; k < dim; ++k) r2 += (x[k] - g.center[s][k]) * (x[k] - g.center[s][k]);
    const T r = dsqrt(r2);
    if (r > 0)
      for (int k = 0; k < dim; ++k) gr[k] = -(x[k] - g.center[s][k]) / r;
    return;
  }
  T q[3] = {0, 0, 0}, out2 = 0, qmax = T(-1e30);
  int kmax = 0;
  for (int k = 0; k < dim; ++k) {
    q[k] = fabs(x[k] - g.center[s][k]) - g.size[s][k];
    if (q[k] > 0) out2 += q[k] * q[k];
    if (q[k] > qmax) { qmax = q[k]; kmax = k; }
  }
  if (out2 > 0) {
    const T o = dsqrt(out2);
    for (int k = 0; k < dim; ++k)
      if (q[k] > 0) gr[k] = -q[k] * (x[k] >= g.center[s][k] ? T(1) : T(-1)) / o;
  } else if (qmax < 0) {
    gr[kmax] = -(x[kmax] >= g.center[s][kmax] ? T(1) : T(-1));
  }
}

// the nearest constraint at x: its value phi and gradient (region positive);
// returns -1 for the bounding box, else the shape index
template <class T>
__device__ __forceinline__ int nearest_constraint(const Geom<T>& g, const T* x, int dim, T& phi, T* gr) {
  phi = box_inside(g, x, dim, gr);
  int best = -1;
  for (int s = 0; s < g.n_shapes; ++s) {
    const T v = constraint_phi(g, s, x, dim);
    if (fabs(v) < fabs(phi)) {
      phi = v;
      best = s;
    }
  }
  if (best >= 0) {
    shape_grad(g, best, x, dim, gr);
    if (!g.keep_inside[best])
      for (int k = 0; k < 3; ++k) gr[k] = -gr[k];
  }
  return best;
}

// unit normal N(x) of the surface a feature-surface particle belongs to
template <class T>
__device__ __forceinline__ void surface_normal(const Geom<T>& g, const T* x, int dim, T* N) {
  T phi;
  nearest_constraint(g, x, dim, phi, N);
  T n2 = 0;
  for (int k = 0; k < dim; ++k) n2 += N[k] * N[k];
  const T inv = n2 > T(0) ? T(1) / dsqrt(n2) : T(0);
  for (int k = 0; k < 3; ++k) N[k] *= inv;
}

// Eq. displacement_surface for a feature-surface particle, after every drift:
// r <- r - phi N onto the nearest constraint surface (the closest point for
// the sphere's and the box's exact distances; three Newton steps for the
// background level set)
template <class T>
__device__ __forceinline__ void project_to_surface(const Geom<T>& g, T* x, int dim) {
  T phi, gr[3];
  const int s = nearest_constraint(g, x, dim, phi, gr);
  if (s >= 0 && g.kind[s] == 2) {
    const T sg = g.keep_inside[s] ? T(1) : T(-1);
    for (int it = 0; it < 3; ++it) {
      T gg[3];
      const T v = sg * bg_interp(g, g.bg_phi, x, dim, gg);
      T g2 = 0;
      for (int k = 0; k < dim; ++k) g2 += gg[k] * gg[k];
      if (!(g2 > T(0))) break;
      for (int k = 0; k < dim; ++k) x[k] -= v * sg * gg[k] / g2;
    }
    return;
  }
  for (int k = 0; k < dim; ++k) x[k] -= phi * gr[k];
}

// inside the region (box and every shape constraint)?
template <class T>
__device__ __forceinline__ bool in_region(const Geom<T>& g, const T* x) {
  for (int k = 0; k < g.dim; ++k)
    if (x[k] < g.lo[k] || x[k] > g.hi[k]) return false;
  for (int s = 0; s < g.n_shapes; ++s)
    if (!(constraint_phi(g, s, x, g.dim) > 0)) return false;
  return true;
}

// ---------------------------------------------------------------- field ----

// polynomial modulation factor 1 + sum_k poly_k b_k(x~)
template <class T>
__device__ __forceinline__ T poly_factor(const Geom<T>& g, const T* x) {
  if (g.n_poly == 0) return T(1);
  T t[3];
  for (int k = 0; k < g.dim; ++k) t[k] = T(2) * (x[k] - g.lo[k]) / g.ext[k] - T(1);
  T b[8];
  if (g.dim == 2) {
    T X = t[0], Y = t[1];
    b[0] = X; b[1] = Y; b[2] = X * X; b[3] = X * Y; b[4] = Y * Y;
    b[5] = X * X * X; b[6] = X * X * Y; b[7] = X * Y * Y;
  } else {
    T X = t[0], Y = t[1], Z = t[2];
    b[0] = X; b[1] = Y; b[2] = Z; b[3] = X * X; b[4] = Y * Y; b[5] = Z * Z;
    b[6] = X * Y; b[7] = Y * Z;
  }
  T f = 1;
  for (int k = 0; k < g.n_poly; ++k) f += g.poly[k] * b[k];
  return f;
}

template <class T> __device__ __forceinline__ T dtanh(T x);
template <> __device__ __forceinline__ float dtanh<float>(float x) { return tanhf(x); }
template <> __device__ __forceinline__ double dtanh<double>(double x) { return tanh(x); }

// target spacing s(x): uniform, linear or tanh in the distance to a shape
// (field kinds 0, 1, 2) or sampled on the background mesh (kind 3)
template <class T>
__device__ __forceinline__ T spacing_of(const Geom<T>& g, const T* x) {
  if (g.field_kind == 0) return g.s0;
  if (g.field_kind == 3) return bg_interp(g, g.bg_s, x, g.dim, (T*)nullptr);
  const T dist = fabs(shape_inside(g, g.dist_shape, x, g.dim));
  if (g.field_kind == 2) return g.a + g.b * dtanh(g.s0 * dist);
  return g.a + g.b * dist;
}

// ds/d|dist| of the distance fields
template <class T>
__device__ __forceinline__ T spacing_slope(const Geom<T>& g, T dist) {
  if (g.field_kind == 2) {
    const T t = dtanh(g.s0 * fabs(dist));
    return g.b * g.s0 * (T(1) - t * t);
  }
  return g.b;
}

// smoothing length h = tau rho_t^(-1/d) with rho_t = rho_scale s^-d (1+P)
// (Eq. scale_SPH_particle, unit mass) = hfac * s * (1+P)^(-1/d)
template <int D, class T>
__device__ __forceinline__ T h_of(const Geom<T>& g, const T* x) {
  T h = g.hfac * spacing_of(g, x);
  if (g.n_poly) {
    T f = poly_factor(g, x);
    if (D == 2) h *= drsqrt(f);
    else h *= (T)rcbrt((double)f);
  }
  return h;
}

template <>
__device__ __forceinline__ float h_of<3, float>(const Geom<float>& g, const float* x) {
  float h = g.hfac * spacing_of(g, x);
  if (g.n_poly) h *= rcbrtf(poly_factor(g, x));
  return h;
}

// ---------------------------------------------------------------- grid ----

template <class T>
__device__ __forceinline__ int level_of_h(const Grid<T>& G, T h) {
  T r = h * G.inv_h0;
  if (!(r >= T(2))) return 0;
  int l = ilogb(r);
  return l < G.n_levels - 1 ? l : G.n_levels - 1;
}

template <class T>
__device__ __forceinline__ int level_of_key(const Grid<T>& G, uint32_t key) {
  int l = 0;
#pragma unroll
  for (int q = 1; q < kMaxLevels; ++q)
    if (q < G.n_levels && key >= G.base[q]) l = q;
  return l;
}

// ------------------------------------------------------------- Philox ----
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32
// multiplies with the published multipliers and Weyl key increments.
__device__ __forceinline__ uint4 philox4x32_10(uint4 ctr, uint2 key) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0 = __umulhi(M0, ctr.x), lo0 = M0 * ctr.x;
    uint32_t hi1 = __umulhi(M1, ctr.z), lo1 = M1 * ctr.z;
    uint4 n;
    n.x = hi1 ^ ctr.y ^ key.x;
    n.y = lo1;
    n.z = hi0 ^ ctr.w ^ key.y;
    n.w = lo0;
    ctr = n;
    key.x += W0;
    key.y += W1;
  }
  return ctr;
}

__device__ __forceinline__ double u01(uint32_t v) {  // (0, 1)
  return ((double)v + 0.5) * 2.3283064365386963e-10;
}

}  // namespace sph
