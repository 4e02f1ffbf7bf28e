// Reverse pass of the relaxation step (sensitivities), templated on the
// dimension D and the working precision T; instantiated in sph_adjoint_2d.cu /
// sph_adjoint_3d.cu.
//
// The step of Algorithm 1 maps the state x to x' through
//   a_i  = sum_j S_ij (x_i - x_j),      S_ij = -coef_ij F(r_ij, H_ij)
//   v~_i = dt1 a_i / 2,                  eta_i = rho_t,i 0.1 r_c,i |v~_i|
//   a~_i = sum_j K_ij (v~_i - v~_j),    K_ij = hm(eta_i, eta_j) (T_i + T_j) F(r_ij, H_ij)
//   y_i  = x_i + dt2 (v~_i + dt2 a~_i / 2),   x'_i = projection(y_i)
// with F = (dW/dr)/r, H_ij = kappa (h_i + h_j)/2, T = 1/rho_t^2,
// coef_ij = Q_i + Q_j + beta_ij P0 (T_i + T_j), Q = p/rho^2 (P0 T at gamma = 2)
// and hm the harmonic mean. Given the adjoint of x' (by particle id), the
// kernels below return the adjoint of x and accumulate those of sigma0,
// gamma, P0 and the density-polynomial coefficients. Every pair sum is a
// gather over particle i's own neighbours (the pair terms are symmetric), so
// no atomics are used and every reduction runs in a fixed order.
//
// Kernels, in launch order per step (state, list and forward quantities of the
// step already in place):
//   k_bwd_out    projection and drift: adjoints of y, v~ (partly) and a~
//   k_bwd_visc   viscous pairs and eta: adjoints of v~, a, h, T, rho_t; its
//                last block adds the argmin particle's share of recomputed
//                step sizes
//   k_bwd_force  pressure / surface-tension pairs and the equation of state
//                (gamma = 2 form: then also the target field, as below)
//   k_bwd_local  density pairs (where rho has an adjoint), then the target
//                field rho_t(x) and h(x): adjoint of x by particle id
// k_obj computes the objective and seeds the same accumulators at the end
// state; k_bwd_local then finishes its gradient.
#pragma once

#include "sph_step_impl.cuh"

// resident 256-thread blocks per SM asked of the FP32 k_bwd_force (caps its
// registers: 4 -> 64)
#ifndef SPH_BWD_FORCE_MIN_BLOCKS
#define SPH_BWD_FORCE_MIN_BLOCKS 4
#endif

namespace sph {

// Wendland C2 pieces in physical units, c = alpha_d (7/pi, 21/(2 pi)):
//   W = c H^-d (1-q)^4 (1+4q),  dW/dr = -20 c H^-(d+1) q (1-q)^3,
//   dW/dH = -c H^-(d+1) (d (1-q)^4 (1+4q) - 20 q^2 (1-q)^3),
//   F = (dW/dr)/r = -20 c H^-(d+2) (1-q)^3,
//   dF/dr = 60 c H^-(d+3) (1-q)^2,  dF/dH = 20 c H^-(d+3) (1-q)^2 ((d+2)(1-q) - 3q)
template <int D, class T>
__device__ __forceinline__ T ipow_d(T iH) {
  return D == 2 ? iH * iH : iH * iH * iH;
}
template <int D, class T>
struct KernelD {
  T W, Wr, WH;  // W, dW/dr, dW/dH
};
template <int D, class T>
__device__ __forceinline__ KernelD<D, T> wendland(T r, T H, T c) {
  KernelD<D, T> k{T(0), T(0), T(0)};
  const T iH = drcp<T>(H), q = r * iH;
  if (!(q < T(1))) return k;
  const T u = T(1) - q, u3 = u * u * u;
  const T cH = c * ipow_d<D, T>(iH);  // c H^-d
  k.W = cH * u3 * u * (T(1) + T(4) * q);
  k.Wr = T(-20) * cH * iH * q * u3;
  k.WH = -cH * iH * (T(D) * u3 * u * (T(1) + T(4) * q) - T(20) * q * q * u3);
  return k;
}
template <int D, class T>
struct ForceD {
  T F, Fr, FH;
};
template <int D, class T>
__device__ __forceinline__ ForceD<D, T> force_fn(T r, T H, T c) {
  ForceD<D, T> k{T(0), T(0), T(0)};
  const T iH = drcp<T>(H), q = r * iH;
  if (!(q < T(1))) return k;
  const T u = T(1) - q, u2 = u * u;
  const T cH3 = c * ipow_d<D, T>(iH) * iH * iH * iH;  // c H^-(d+3)
  k.F = T(-20) * cH3 * H * u2 * u;
  k.Fr = T(60) * cH3 * u2;
  k.FH = T(20) * cH3 * u2 * (T(D + 2) * u - T(3) * q);
  return k;
}

// fixed-order block sum of M values (warp sums in the working precision,
// warp totals and everything after in FP64); the block's sums go to
// part[blockIdx.x] and the last block to finish returns true with every
// block's partial summed (in block order) into out[0..M) of every thread.
__device__ __forceinline__ float warp_sum_t(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum_t(double v) { return warp_sum(v); }

template <int M, class T>
__device__ bool block_partials(T (&v)[M], double* __restrict__ part, unsigned* __restrict__ ticket, double* out) {
  __shared__ double sm[8][M];
  __shared__ double res[M];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < M; ++q) {
    const T x = warp_sum_t(v[q]);
    if (lane == 0) sm[w][q] = (double)x;
  }
  __syncthreads();
  if (threadIdx.x < M) {
    double s = 0.0;
    for (int k = 0; k < nw; ++k) s += sm[k][threadIdx.x];
    part[(size_t)blockIdx.x * kAdjPartials + threadIdx.x] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  // every thread sums a fixed stride of the block partials, then a fixed tree
  double a[M];
#pragma unroll
  for (int q = 0; q < M; ++q) a[q] = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
#pragma unroll
    for (int q = 0; q < M; ++q) a[q] += __ldcg(part + (size_t)b * kAdjPartials + q);
#pragma unroll
  for (int q = 0; q < M; ++q) {
    const double x = warp_sum(a[q]);
    if (lane == 0) sm[w][q] = x;
  }
  __syncthreads();
  if (threadIdx.x < M) {
    double s = 0.0;
    for (int k = 0; k < nw; ++k) s += sm[k][threadIdx.x];
    res[threadIdx.x] = s;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < M; ++q) out[q] = res[q];
  if (threadIdx.x == 0) *ticket = 0u;
  return true;
}

template <class T> __device__ __forceinline__ T dlog(T x);
template <> __device__ __forceinline__ float dlog<float>(float x) { return logf(x); }
template <> __device__ __forceinline__ double dlog<double>(double x) { return log(x); }

// T = 1/rho_t^2 and rho_t from h (h = tau rho_t^(-1/d))
template <int D, class T>
__device__ __forceinline__ T rho_t_of_h(T h, T inv_tau) {
  const T t = T(1) / (h * inv_tau);
  return D == 2 ? t * t : t * t * t;
}

// ------------------------------------------------------------------------
// k_bwd_out: y = x + d, then the box clamp and each shape projection in order
// (Eq. displacement_surface). The adjoint of y is the transpose of that chain
// of Jacobians applied to the adjoint of x' (identity where no constraint
// acted; clamped / pushed-out coordinates get zero; a sphere projection
// c + R (y - c)/|y - c| has Jacobian R/|y - c| (I - n n^T)).
// ------------------------------------------------------------------------
template <int D, class T>
__global__ void __launch_bounds__(256) k_bwd_out(int n, const StepCtl* __restrict__ ctl,
                                                 const LL4* __restrict__ X0, const LL4* __restrict__ X1,
                                                 const uint32_t* __restrict__ p0, const uint32_t* __restrict__ p1,
                                                 const V4<T>* __restrict__ acc, const V4<T>* __restrict__ visc,
                                                 const Scalars* __restrict__ scal, Frame<T> F, Geom<T> geo,
                                                 AdjBufs<T> B) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  T v[1] = {T(0)};
  if (i < n) {
    const int buf = ctl->buf;
    const LL4 X = (buf ? X1 : X0)[i];
    const uint32_t id = (buf ? p1 : p0)[i];
    const T dt1 = (T)scal->dt1, dt2 = (T)scal->dt2;
    const V4<T> a = acc[i], at = visc[i];
    const T vt[3] = {T(0.5) * dt1 * a.x, T(0.5) * dt1 * a.y, T(0.5) * dt1 * a.z};
    const T att[3] = {at.x, at.y, at.z};
    T g[3] = {0, 0, 0};
    for (int k = 0; k < D; ++k) g[k] = (T)B.gin[(size_t)id * D + k];
    // forward, as pass B: integer drift with the box clamp, then the shapes
    const long long Xc[3] = {X.x, X.y, X.z};
    bool clamped[3] = {false, false, false};
    T z[kMaxShapes + 1][3];
    for (int k = 0; k < 3; ++k) z[0][k] = T(0);
    for (int k = 0; k < D; ++k) {
      const T dk = (vt[k] + T(0.5) * dt2 * att[k]) * dt2;
      long long u = Xc[k] + state_units(dk * F.inv_q64t);
      if (u < 0) {
        u = 0;
        clamped[k] = true;
      }
      if (u > F.xmax[k]) {
        u = F.xmax[k];
        clamped[k] = true;
      }
      z[0][k] = F.lo[k] + (T)u * F.q64t;
    }
    for (int s = 0; s < geo.n_shapes; ++s) {
      for (int k = 0; k < 3; ++k) z[s + 1][k] = z[s][k];
      project_shape(geo, s, z[s + 1], D);
    }
    // reverse
    for (int s = geo.n_shapes - 1; s >= 0; --s) {
      const T* x = z[s];
      if (!(constraint_phi(geo, s, x, D) < T(0))) continue;
      if (geo.kind[s] == 0) {
        T dv[3] = {0, 0, 0}, r2 = 0;
        for (int k = 0; k < D; ++k) {
          dv[k] = x[k] - geo.center[s][k];
          r2 += dv[k] * dv[k];
        }
        const T r = dsqrt(r2);
        if (r == T(0)) {
          for (int k = 0; k < D; ++k) g[k] = T(0);
          continue;
        }
        T ng = 0;
        for (int k = 0; k < D; ++k) ng += dv[k] * g[k];
        ng /= r;
        for (int k = 0; k < D; ++k) g[k] = geo.size[s][0] / r * (g[k] - dv[k] / r * ng);
      } else if (geo.keep_inside[s]) {
        for (int k = 0; k < D; ++k) {
          const T lo = geo.center[s][k] - geo.size[s][k], hi = geo.center[s][k] + geo.size[s][k];
          if (x[k] < lo || x[k] > hi) g[k] = T(0);
        }
      } else {
        int best = 0;
        T bestd = T(1e30);
        for (int k = 0; k < D; ++k) {
          const T dlo = x[k] - (geo.center[s][k] - geo.size[s][k]);
          const T dhi = (geo.center[s][k] + geo.size[s][k]) - x[k];
          if (dlo < bestd) { bestd = dlo; best = k; }
          if (dhi < bestd) { bestd = dhi; best = k; }
        }
        g[best] = T(0);
      }
    }
    for (int k = 0; k < D; ++k)
      if (clamped[k]) g[k] = T(0);
    B.xb[i] = V4<double>{(double)g[0], (double)g[1], (double)g[2], 0.0};
    const T c = T(0.5) * dt2 * dt2;
    B.atb[i] = V4<T>{c * g[0], c * g[1], c * g[2], T(0)};
    T pv = 0;
    for (int k = 0; k < D; ++k) pv += g[k] * (vt[k] + dt2 * att[k]);
    v[0] = pv;
  }
  double out[1];
  if (block_partials<1>(v, B.part, B.ticket, out) && threadIdx.x == 0) B.acc[kAdjDt2b] = out[0];
}

// ------------------------------------------------------------------------
// k_bwd_visc: viscous pairs (this step's force pairs) and the local eta map.
// Three gathers per pair (view, a, adjoint of a~): FP32 builds are held to 64
// registers so that four blocks per SM keep enough loads in flight.
// ------------------------------------------------------------------------
template <int D, class T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2) k_bwd_visc(int n, const StepCtl* __restrict__ ctl,
                                                  const typename ViewOf<T>::type* __restrict__ v0,
                                                  const typename ViewOf<T>::type* __restrict__ v1,
                                                  const uint32_t* __restrict__ plist,
                                                  const uint32_t* __restrict__ pcount,
                                                  const V4<T>* __restrict__ acc, const Scalars* __restrict__ scal,
                                                  Frame<T> F, Phys<T> P, int recomputed_dt, AdjBufs<T> B) {
  using VT = typename ViewOf<T>::type;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  T v[1] = {T(0)};
  if (i < n) {
    const VT* __restrict__ view = ctl->vp ? v1 : v0;
    const VT vi = view[i];
    const T qv = F.qv, hv = view_h(vi), hi = hv * qv;
    const T half_kappa = T(0.5) * P.kappa;
    const T dt1 = (T)scal->dt1, dt2 = (T)scal->dt2;
    const V4<T> ai = acc[i];
    const T rti = rho_t_of_h<D, T>(hi, P.inv_tau), Ti = inv_rho_t2<D, T>(hi, P.inv_tau);
    const T etai = dt1 * ai.w;
    const V4<T> atbi = B.atb[i];
    const V4<double> ybar = B.xb[i];
    T vx = 0, vy = 0, vz = 0;        // adjoint of v~_i from the pairs
    T xx = 0, xy = 0, xz = 0;        // adjoint of x_i from the pairs
    T hbar = 0, Tbar = 0, etab = 0;
    const int cnt = (int)pcount[i];
    struct Rec {
      V4<T> a, atb;
    };
    for_list_x(plist, view, n, i, cnt, [&](int j) { return Rec{acc[j], B.atb[j]}; },
               [&](uint32_t e, const VT& vj, const Rec& rj) {
      const int j = (int)(e >> 8);
      const T dx = vd<false>(F, vi.x, vj.x), dy = vd<false>(F, vi.y, vj.y);
      const T dz = D == 3 ? vd<false>(F, vi.z, vj.z) : T(0);
      const T r2 = dx * dx + dy * dy + dz * dz;
      const T hvj = view_h(vj);
      const T Hv = half_kappa * (hv + hvj);
      if (!(r2 < Hv * Hv) || j == i) return;
      const T irv = drsqrt<T>(r2);  // 1/r, view units
      const T r = r2 * irv * qv, ir = irv * F.inv_qv, ex = dx * qv, ey = dy * qv, ez = dz * qv;
      const ForceD<D, T> f = force_fn<D, T>(r, Hv * qv, P.alpha);
      const V4<T>& aj = rj.a;
      const V4<T>& atbj = rj.atb;
      const T Tj = inv_rho_t2<D, T>(hvj * qv, P.inv_tau);
      const T etaj = dt1 * aj.w;
      const T es = etai + etaj;
      const T ies = es > T(0) ? drcp<T>(es) : T(0);
      const T hm = T(2) * etai * etaj * ies;
      const T dhm = T(2) * etaj * etaj * ies * ies;
      const T Ts = Ti + Tj;
      const T K = hm * Ts * f.F;
      const T gx = atbi.x - atbj.x, gy = atbi.y - atbj.y, gz = atbi.z - atbj.z;
      vx += K * gx;
      vy += K * gy;
      vz += K * gz;
      const T hd = T(0.5) * dt1;
      const T Kb = gx * hd * (ai.x - aj.x) + gy * hd * (ai.y - aj.y) + gz * hd * (ai.z - aj.z);
      etab += Kb * Ts * f.F * dhm;
      Tbar += Kb * hm * f.F;
      const T Fb = Kb * hm * Ts;
      const T cr = Fb * f.Fr * ir;
      xx += cr * ex;
      xy += cr * ey;
      xz += cr * ez;
      hbar += Fb * f.FH * half_kappa;
    });
    // adjoint of v~_i: the drift, the pairs, and eta_i = rho_t,i 0.1 kappa h_i |v~_i|
    T vbx = vx + dt2 * (T)ybar.x, vby = vy + dt2 * (T)ybar.y, vbz = vz + dt2 * (T)ybar.z;
    const T hd = T(0.5) * dt1;
    const T vn = hd * dsqrt(ai.x * ai.x + ai.y * ai.y + ai.z * ai.z);
    T rtbar = 0;
    if (vn > T(0)) {
      const T kk = T(0.1) * P.kappa;
      rtbar += etab * kk * hi * vn;
      hbar += etab * kk * rti * vn;
      const T c = etab * kk * rti * hi / vn;
      vbx += c * hd * ai.x;
      vby += c * hd * ai.y;
      vbz += c * hd * ai.z;
    }
    // v~ = dt1 a / 2
    B.ab[i] = V4<T>{hd * vbx, hd * vby, hd * vbz, T(0)};
    v[0] = T(0.5) * (ai.x * vbx + ai.y * vby + ai.z * vbz);
    B.xb[i] = V4<double>{ybar.x + xx, ybar.y + xy, ybar.z + xz, 0.0};
    B.hb[i] = hbar;
    B.Tb[i] = Tbar;
    B.rtb[i] = rtbar;
  }
  double out[1];
  if (block_partials<1>(v, B.part, B.ticket, out) && threadIdx.x == 0) {
    B.acc[kAdjDt1b] = out[0];
    // recomputed sizes: dt1 = 0.25 sqrt(m), dt2 = 0.2 sqrt(m), m = r_c,k/|a_k|
    const double m = scal->min_rc_a;
    const double mb = (recomputed_dt && m > 0.0 && m < DBL_MAX) ? (0.125 * out[0] + 0.1 * B.acc[kAdjDt2b]) / sqrt(m)
                                                                : 0.0;
    B.acc[kAdjMbar] = mb;
    // the argmin particle k of m takes m's adjoint through a_k and h_k (every
    // block has written its adjoints: this is the last block to finish)
    const long long k = scal->argmin;
    if (k >= 0 && mb != 0.0) {
      const VT* __restrict__ view = ctl->vp ? v1 : v0;
      const double h = (double)view_h(view[k]) * (double)F.qv;
      const V4<T> a = acc[k];
      const double ax = a.x, ay = a.y, az = a.z;
      const double an = sqrt(ax * ax + ay * ay + az * az);
      const double c = -mb * (double)P.kappa * h / (an * an * an);
      const T* abp = (const T*)&B.ab[k];
      B.ab[k] = V4<T>{(T)(__ldcg(abp + 0) + (T)(c * ax)), (T)(__ldcg(abp + 1) + (T)(c * ay)),
                      (T)(__ldcg(abp + 2) + (T)(c * az)), __ldcg(abp + 3)};
      B.hb[k] = __ldcg(&B.hb[k]) + (T)(mb * (double)P.kappa / an);
    }
  }
}

// gradient of the signed inside distance of shape s (the branch its value takes)
template <class T>
__device__ __forceinline__ void inside_distance_grad(const Geom<T>& g, int s, const T* x, int dim, T* gr) {
  for (int k = 0; k < 3; ++k) gr[k] = T(0);
  if (g.kind[s] == 2) {  // not reached: the reverse pass refuses background-mesh geometry
    bg_interp(g, g.bg_phi, x, dim, gr);
    return;
  }
  if (g.kind[s] == 0) {
    T r2 = 0;
    for (int k = 0; k < dim; ++k) r2 += (x[k] - g.center[s][k]) * (x[k] - g.center[s][k]);
    const T r = dsqrt(r2);
    if (r > T(0))
      for (int k = 0; k < dim; ++k) gr[k] = -(x[k] - g.center[s][k]) / r;
    return;
  }
  T out2 = 0, qmax = T(-1e30), q[3] = {0, 0, 0};
  int kmax = 0;
  for (int k = 0; k < dim; ++k) {
    q[k] = fabs(x[k] - g.center[s][k]) - g.size[s][k];
    if (q[k] > T(0)) out2 += q[k] * q[k];
    if (q[k] > qmax) {
      qmax = q[k];
      kmax = k;
    }
  }
  if (out2 > T(0)) {
    const T o = dsqrt(out2);
    for (int k = 0; k < dim; ++k)
      if (q[k] > T(0)) gr[k] = -q[k] * (x[k] >= g.center[s][k] ? T(1) : T(-1)) / o;
  } else if (qmax < T(0)) {
    gr[kmax] = -(x[kmax] >= g.center[s][kmax] ? T(1) : T(-1));
  }
}

// rho_t(x) = rho_scale s(x)^-d P(x): value, gradient in x, derivatives in the
// polynomial coefficients
template <int D, class T>
__device__ __forceinline__ T rho_t_grad(const Geom<T>& g, const T* x, T* grad, T* dc) {
  const T s = spacing_of(g, x);
  const T base = g.rho_scale * (D == 2 ? T(1) / (s * s) : T(1) / (s * s * s));
  T gs[3] = {0, 0, 0};
  if (g.field_kind == 3) {
    bg_interp(g, g.bg_s, x, D, gs);
  } else if (g.field_kind != 0) {
    const T dist = shape_inside(g, g.dist_shape, x, D);
    T gd[3];
    inside_distance_grad(g, g.dist_shape, x, D, gd);
    const T sg = dist >= T(0) ? T(1) : T(-1);
    const T slope = spacing_slope(g, dist);
    for (int k = 0; k < D; ++k) gs[k] = slope * sg * gd[k];
  }
  T Pf = 1, gP[3] = {0, 0, 0};
  for (int m = 0; m < 8; ++m) dc[m] = T(0);
  if (g.n_poly > 0) {
    T t[3] = {0, 0, 0}, tt[3] = {0, 0, 0};
    for (int k = 0; k < D; ++k) {
      t[k] = T(2) * (x[k] - g.lo[k]) / g.ext[k] - T(1);
      tt[k] = T(2) / g.ext[k];
    }
    T b[8], bx[8], by[8], bz[8];
    const T X = t[0], Y = t[1], Z = t[2];
    if (D == 2) {
      const T b_[8] = {X, Y, X * X, X * Y, Y * Y, X * X * X, X * X * Y, X * Y * Y};
      const T x_[8] = {1, 0, 2 * X, Y, 0, 3 * X * X, 2 * X * Y, Y * Y};
      const T y_[8] = {0, 1, 0, X, 2 * Y, 0, X * X, 2 * X * Y};
      for (int m = 0; m < 8; ++m) {
        b[m] = b_[m];
        bx[m] = x_[m];
        by[m] = y_[m];
        bz[m] = T(0);
      }
    } else {
      const T b_[8] = {X, Y, Z, X * X, Y * Y, Z * Z, X * Y, Y * Z};
      const T x_[8] = {1, 0, 0, 2 * X, 0, 0, Y, 0};
      const T y_[8] = {0, 1, 0, 0, 2 * Y, 0, X, Z};
      const T z_[8] = {0, 0, 1, 0, 0, 2 * Z, 0, Y};
      for (int m = 0; m < 8; ++m) {
        b[m] = b_[m];
        bx[m] = x_[m];
        by[m] = y_[m];
        bz[m] = z_[m];
      }
    }
    for (int m = 0; m < g.n_poly; ++m) {
      Pf += g.poly[m] * b[m];
      dc[m] = base * b[m];
      gP[0] += g.poly[m] * bx[m] * tt[0];
      gP[1] += g.poly[m] * by[m] * tt[1];
      gP[2] += g.poly[m] * bz[m] * tt[2];
    }
  }
  const T rt = base * Pf;
  for (int k = 0; k < 3; ++k) grad[k] = T(0);
  for (int k = 0; k < D; ++k) grad[k] = rt * (-T(D) * gs[k] / s) + base * gP[k];
  return rt;
}

// adjoint of the target field at a particle: rho_t(x), h = tau rho_t^(-1/d)
// and T = rho_t^-2 carry the adjoints rtb, hb, Tb; returns the adjoint of x
// (xg) and the coefficient derivatives times that adjoint (dc)
template <int D, class T>
__device__ __forceinline__ void field_adjoint(const Frame<T>& F, const Geom<T>& geo, const LL4& X, T h, T rtb, T hb,
                                              T Tb, T* xg, T* dc) {
  T x[3], grad[3];
  abs_pos<D, T>(F, X, x);
  const T rt = rho_t_grad<D, T>(geo, x, grad, dc);
  const T irt = drcp<T>(rt);
  const T tot = rtb + hb * (-h * irt / T(D)) + Tb * (T(-2) * irt * irt * irt);
  for (int k = 0; k < 3; ++k) xg[k] = tot * grad[k];
  for (int m = 0; m < 8; ++m) dc[m] *= tot;
}

// ------------------------------------------------------------------------
// k_bwd_force: pressure and surface-tension pairs, then the equation of state
// Q = p/rho^2 = P0 (rho/rho_t)^gamma / rho^2 (P0 T in the gamma = 2 form).
// ------------------------------------------------------------------------
template <int D, class T, bool GENERAL>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? SPH_BWD_FORCE_MIN_BLOCKS : 2) k_bwd_force(int n, const StepCtl* __restrict__ ctl,
                                                   const typename ViewOf<T>::type* __restrict__ v0,
                                                   const typename ViewOf<T>::type* __restrict__ v1,
                                                   const uint32_t* __restrict__ m0, const uint32_t* __restrict__ m1,
                                                   const uint32_t* __restrict__ plist,
                                                   const uint32_t* __restrict__ pcount,
                                                   const T* __restrict__ rho, const T* __restrict__ pc,
                                                   const Scalars* __restrict__ scal, Frame<T> F, Phys<T> P,
                                                   const LL4* __restrict__ X0, const LL4* __restrict__ X1,
                                                   const uint32_t* __restrict__ p0, const uint32_t* __restrict__ p1,
                                                   Geom<T> geo, AdjBufs<T> B) {
  using VT = typename ViewOf<T>::type;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  // sigma(t), P0, gamma; without a density adjoint (gamma = 2 form) also the
  // target-field step of k_bwd_local: the 8 coefficient derivatives
  T v[11] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  if (i < n) {
    const VT* __restrict__ view = ctl->vp ? v1 : v0;
    const VT vi = view[i];
    const uint32_t ci = (ctl->buf ? m1 : m0)[i] & 0xFFu;
    const T qv = F.qv, hv = view_h(vi), hi = hv * qv;
    const T half_kappa = T(0.5) * P.kappa;
    const T sigma = (T)scal->sigma, P0 = P.P0;
    const T rti = rho_t_of_h<D, T>(hi, P.inv_tau), Ti = inv_rho_t2<D, T>(hi, P.inv_tau);
    const T Qi = GENERAL ? pc[i] : P0 * Ti;
    const V4<T> abi = B.ab[i];
    T xx = 0, xy = 0, xz = 0, hbar = 0, Tbar = 0, Qbar = 0;
    T sb = 0, pb = 0;
    const int cnt = (int)pcount[i];
    for_list_x(plist, view, n, i, cnt, [&](int j) { return B.ab[j]; }, [&](uint32_t e, const VT& vj, const V4<T>& abj) {
      const int j = (int)(e >> 8);
      const T dx = vd<false>(F, vi.x, vj.x), dy = vd<false>(F, vi.y, vj.y);
      const T dz = D == 3 ? vd<false>(F, vi.z, vj.z) : T(0);
      const T r2 = dx * dx + dy * dy + dz * dz;
      const T hvj = view_h(vj);
      const T Hv = half_kappa * (hv + hvj);
      if (!(r2 < Hv * Hv) || j == i) return;
      const T irv = drsqrt<T>(r2);  // 1/r, view units
      const T r = r2 * irv * qv, ir = irv * F.inv_qv, ex = dx * qv, ey = dy * qv, ez = dz * qv;
      const ForceD<D, T> f = force_fn<D, T>(r, Hv * qv, P.alpha);
      const T Tj = inv_rho_t2<D, T>(hvj * qv, P.inv_tau);
      const T Qj = GENERAL ? pc[j] : P0 * Tj;
      const bool other = (e & 0xFFu) != ci;
      const T beta = other ? sigma : T(0);
      const T Ts = Ti + Tj;
      const T coef = Qi + Qj + beta * P0 * Ts;
      const T S = -coef * f.F;
      const T gx = abi.x - abj.x, gy = abi.y - abj.y, gz = abi.z - abj.z;
      xx += S * gx;
      xy += S * gy;
      xz += S * gz;
      const T Sb = gx * ex + gy * ey + gz * ez;
      const T cb = -Sb * f.F;
      Qbar += cb;
      Tbar += cb * beta * P0;
      // each unordered pair is visited from both ends
      if (other) sb += T(0.5) * cb * P0 * Ts;
      pb += T(0.5) * cb * beta * Ts;
      const T Fb = -Sb * coef;
      const T cr = Fb * f.Fr * ir;
      xx += cr * ex;
      xy += cr * ey;
      xz += cr * ez;
      hbar += Fb * f.FH * half_kappa;
    });
    // equation of state
    const T rh = rho[i];
    const T lr = dlog<T>(rh / rti);
    const T gb = Qbar * Qi * lr;
    T rhob = 0, rtbar = 0;
    if (GENERAL) {
      rhob = Qbar * (P.gamma - T(2)) * Qi / rh;
      rtbar = -P.gamma * Qbar * Qi / rti;
      if (P0 != T(0)) pb += Qbar * Qi / P0;
    } else {
      Tbar += Qbar * P0;
      pb += Qbar * Ti;
    }
    V4<double> xb = B.xb[i];
    v[0] = sb;
    v[1] = pb;
    v[2] = gb;
    if (GENERAL) {
      xb.x += xx;
      xb.y += xy;
      xb.z += xz;
      B.xb[i] = xb;
      B.hb[i] += hbar;
      B.Tb[i] += Tbar;
      B.rtb[i] += rtbar;
      B.rhob[i] = rhob;
    } else {
      const int buf = ctl->buf;
      T xg[3], dc[8];
      field_adjoint<D, T>(F, geo, (buf ? X1 : X0)[i], hi, B.rtb[i] + rtbar, B.hb[i] + hbar, B.Tb[i] + Tbar, xg, dc);
      const uint32_t id = (buf ? p1 : p0)[i];
      B.gout[(size_t)id * D + 0] = xb.x + (double)(xx + xg[0]);
      B.gout[(size_t)id * D + 1] = xb.y + (double)(xy + xg[1]);
      if (D == 3) B.gout[(size_t)id * D + 2] = xb.z + (double)(xz + xg[2]);
      for (int m = 0; m < 8; ++m) v[3 + m] = dc[m];
    }
  }
  double out[11];
  if (block_partials<11>(v, B.part, B.ticket, out) && threadIdx.x == 0) {
    if (!GENERAL)
      for (int m = 0; m < 8; ++m) B.acc[kAdjPoly + m] += out[3 + m];
    // sigma(t) = sigma0 ramp(t) (Eq. sph_st_sigma) at the step pass A ran
    StepCtl c1 = *ctl;
    c1.sigma0 = 1.0;
    const double ramp = sigma_of(c1, scal->step_of_stats);
    B.acc[kAdjSigma0] += out[0] * ramp;
    B.acc[kAdjP0] += out[1];
    B.acc[kAdjGamma] += out[2];
  }
}

// ------------------------------------------------------------------------
// k_bwd_local: density pairs (DENS: rho has an adjoint; the list is symmetric,
// so i finds every j whose support holds i), then the target field:
// rho_t(x_i), h_i = tau rho_t^(-1/d), T_i = rho_t^-2. Writes the adjoint of x
// by particle id and adds the coefficient derivatives.
// ------------------------------------------------------------------------
template <int D, class T, bool DENS>
__global__ void __launch_bounds__(256) k_bwd_local(int n, const StepCtl* __restrict__ ctl,
                                                   const typename ViewOf<T>::type* __restrict__ v0,
                                                   const typename ViewOf<T>::type* __restrict__ v1,
                                                   const LL4* __restrict__ X0, const LL4* __restrict__ X1,
                                                   const uint32_t* __restrict__ p0, const uint32_t* __restrict__ p1,
                                                   const uint32_t* __restrict__ list,
                                                   const uint32_t* __restrict__ lcount, int cap, Frame<T> F,
                                                   Phys<T> P, Geom<T> geo, AdjBufs<T> B) {
  using VT = typename ViewOf<T>::type;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  T v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (i < n) {
    const VT* __restrict__ view = ctl->vp ? v1 : v0;
    const int buf = ctl->buf;
    const VT vi = view[i];
    const T qv = F.qv, hv = view_h(vi), hi = hv * qv;
    T hbar = B.hb[i];
    T xx = 0, xy = 0, xz = 0;
    if (DENS) {
      const T rbi = B.rhob[i];
      const T Hi = P.kappa * hi;
      for_skin_list(list, view, n, i, lcount[i], cap, [&](uint32_t e, const VT& vj) {
        const int j = (int)(e >> 8);
        const T dx = vd<false>(F, vi.x, vj.x), dy = vd<false>(F, vi.y, vj.y);
        const T dz = D == 3 ? vd<false>(F, vi.z, vj.z) : T(0);
        const T r = dsqrt(dx * dx + dy * dy + dz * dz) * qv;
        const KernelD<D, T> ki = wendland<D, T>(r, Hi, P.alpha);
        hbar += rbi * ki.WH * P.kappa;
        if (j == i || !(r > T(0))) return;
        const T Hj = P.kappa * view_h(vj) * qv;
        const KernelD<D, T> kj = wendland<D, T>(r, Hj, P.alpha);
        const T c = (rbi * ki.Wr + B.rhob[j] * kj.Wr) / r;
        xx += c * dx * qv;
        xy += c * dy * qv;
        xz += c * dz * qv;
      });
    }
    T xg[3], dc[8];
    field_adjoint<D, T>(F, geo, (buf ? X1 : X0)[i], hi, B.rtb[i], hbar, B.Tb[i], xg, dc);
    V4<double> xb = B.xb[i];
    xb.x += (double)(xx + xg[0]);
    xb.y += (double)(xy + xg[1]);
    xb.z += (double)(xz + xg[2]);
    const uint32_t id = (buf ? p1 : p0)[i];
    B.gout[(size_t)id * D + 0] = xb.x;
    B.gout[(size_t)id * D + 1] = xb.y;
    if (D == 3) B.gout[(size_t)id * D + 2] = xb.z;
    for (int m = 0; m < 8; ++m) v[m] = dc[m];
  }
  double out[8];
  if (block_partials<8>(v, B.part, B.ticket, out) && threadIdx.x < 8) B.acc[kAdjPoly + threadIdx.x] += out[threadIdx.x];
}

// ------------------------------------------------------------------------
// k_obj: L = sum_i (rho_i/rho_t,i - 1)^2 + lambda sum_{i<j, C_i != C_j} W(r_ij, kappa h_ij)
// at the current state, and the seeds of its reverse pass (adjoints of rho,
// rho_t, h and, from the interface term and the caller's seed, of x).
// ------------------------------------------------------------------------
template <int D, class T>
__global__ void __launch_bounds__(256) k_obj(int n, const StepCtl* __restrict__ ctl,
                                             const typename ViewOf<T>::type* __restrict__ v0,
                                             const typename ViewOf<T>::type* __restrict__ v1,
                                             const uint32_t* __restrict__ m0, const uint32_t* __restrict__ m1,
                                             const uint32_t* __restrict__ p0, const uint32_t* __restrict__ p1,
                                             const uint32_t* __restrict__ list, const uint32_t* __restrict__ lcount,
                                             int cap, Frame<T> F, Phys<T> P, T wd, T lambda, AdjBufs<T> B) {
  using VT = typename ViewOf<T>::type;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  T v[2] = {T(0), T(0)};
  if (i < n) {
    const VT* __restrict__ view = ctl->vp ? v1 : v0;
    const int buf = ctl->buf;
    const VT vi = view[i];
    const uint32_t ci = (buf ? m1 : m0)[i] & 0xFFu;
    const T qv = F.qv, hv = view_h(vi), hi = hv * qv;
    const T Hi = P.kappa * hi, half_kappa = T(0.5) * P.kappa;
    T rho = 0, xx = 0, xy = 0, xz = 0, hbar = 0, wi = 0;
    for_skin_list(list, view, n, i, lcount[i], cap, [&](uint32_t e, const VT& vj) {
      const int j = (int)(e >> 8);
      const T dx = vd<false>(F, vi.x, vj.x), dy = vd<false>(F, vi.y, vj.y);
      const T dz = D == 3 ? vd<false>(F, vi.z, vj.z) : T(0);
      const T r2 = dx * dx + dy * dy + dz * dz;
      const T r = dsqrt(r2) * qv;
      rho += wendland<D, T>(r, Hi, P.alpha).W;
      const T hvj = view_h(vj);
      const T Hv = half_kappa * (hv + hvj);
      if (j == i || (e & 0xFFu) == ci || !(r2 < Hv * Hv)) return;
      const KernelD<D, T> k = wendland<D, T>(r, Hv * qv, P.alpha);
      wi += T(0.5) * k.W;  // each unordered pair from both ends
      const T c = lambda * k.Wr / r;
      xx += c * dx * qv;
      xy += c * dy * qv;
      xz += c * dz * qv;
      hbar += lambda * k.WH * half_kappa;
    });
    const T rt = rho_t_of_h<D, T>(hi, P.inv_tau);
    const T e = rho / rt - T(1);
    v[0] = e * e;
    v[1] = wi;
    B.rhob[i] = wd * T(2) * e / rt;
    B.rtb[i] = wd * T(-2) * e * rho / (rt * rt);
    B.hb[i] = hbar;
    B.Tb[i] = T(0);
    const uint32_t id = (buf ? p1 : p0)[i];
    double s[3] = {0, 0, 0};
    if (B.gin)
      for (int k = 0; k < D; ++k) s[k] = B.gin[(size_t)id * D + k];
    B.xb[i] = V4<double>{s[0] + xx, s[1] + xy, s[2] + xz, 0.0};
  }
  double out[2];
  if (block_partials<2>(v, B.part, B.ticket, out) && threadIdx.x == 0)
    B.acc[kAdjL] = (double)wd * out[0] + (double)lambda * out[1];
}

// ------------------------------------------------------------------ tape --
// After pass A of a taped step: the state it used (current order), its
// control block and its scalars go to one slot of the tape, so that the
// reverse pass of that step needs no list rebuild and no forward recompute.
template <class VT>
__global__ void __launch_bounds__(256) k_tape_snapshot(int n, const StepCtl* __restrict__ ctl,
                                                       const Scalars* __restrict__ scal,
                                                       const LL4* __restrict__ X0, const LL4* __restrict__ X1,
                                                       const uint32_t* __restrict__ m0,
                                                       const uint32_t* __restrict__ m1,
                                                       const uint32_t* __restrict__ p0,
                                                       const uint32_t* __restrict__ p1, const VT* __restrict__ v0,
                                                       const VT* __restrict__ v1, LL4* __restrict__ oX,
                                                       uint32_t* __restrict__ oM, uint32_t* __restrict__ oP,
                                                       VT* __restrict__ oV, StepCtl* __restrict__ octl,
                                                       Scalars* __restrict__ oscal) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int buf = ctl->buf, vp = ctl->vp;
  if (i == 0) {
    *octl = *ctl;
    *oscal = *scal;
  }
  if (i >= n) return;
  oX[i] = (buf ? X1 : X0)[i];
  oM[i] = (buf ? m1 : m0)[i];
  oP[i] = (buf ? p1 : p0)[i];
  oV[i] = (vp ? v1 : v0)[i];
}

// ---------------------------------------------------------------- launch --
template <int D, class T>
cudaError_t launch_bwd_step(const DevState& S, const Frame<T>& F, const Phys<T>& P, const Geom<T>& geo,
                            const AdjBufs<T>& B, int recomputed_dt, int general_eos, cudaStream_t st) {
  using VT = typename ViewOf<T>::type;
  const int tb = 256, gb = grid_for(S.n, tb);
  if (S.n <= 0) return cudaSuccess;
  const VT* w0 = (const VT*)S.view[0];
  const VT* w1 = (const VT*)S.view[1];
  const V4<T>* acc = (const V4<T>*)S.acc4;
  k_bwd_out<D, T><<<gb, tb, 0, st>>>(S.n, S.ctl, (const LL4*)S.X[0], (const LL4*)S.X[1], S.pid[0], S.pid[1], acc,
                                     (const V4<T>*)S.visc, S.scal, F, geo, B);
  k_bwd_visc<D, T><<<gb, tb, 0, st>>>(S.n, S.ctl, w0, w1, S.plist, S.pcount, acc, S.scal, F, P, recomputed_dt, B);
  if (general_eos)
    k_bwd_force<D, T, true><<<gb, tb, 0, st>>>(S.n, S.ctl, w0, w1, S.meta[0], S.meta[1], S.plist, S.pcount,
                                               (const T*)S.rho, (const T*)S.pc, S.scal, F, P, (const LL4*)S.X[0],
                                               (const LL4*)S.X[1], S.pid[0], S.pid[1], geo, B);
  else  // the gamma = 2 form has no density adjoint: the target-field step is fused in
    k_bwd_force<D, T, false><<<gb, tb, 0, st>>>(S.n, S.ctl, w0, w1, S.meta[0], S.meta[1], S.plist, S.pcount,
                                                (const T*)S.rho, (const T*)S.pc, S.scal, F, P, (const LL4*)S.X[0],
                                                (const LL4*)S.X[1], S.pid[0], S.pid[1], geo, B);
  if (general_eos)
    k_bwd_local<D, T, true><<<gb, tb, 0, st>>>(S.n, S.ctl, w0, w1, (const LL4*)S.X[0], (const LL4*)S.X[1],
                                               S.pid[0], S.pid[1], S.list, S.lcount, S.cap, F, P, geo, B);
  return cudaGetLastError();
}

template <int D, class T>
cudaError_t launch_objective(const DevState& S, const Frame<T>& F, const Phys<T>& P, const Geom<T>& geo,
                             const AdjBufs<T>& B, double wd, double lambda, cudaStream_t st) {
  using VT = typename ViewOf<T>::type;
  const int tb = 256, gb = grid_for(S.n, tb);
  if (S.n <= 0) return cudaSuccess;
  const VT* w0 = (const VT*)S.view[0];
  const VT* w1 = (const VT*)S.view[1];
  k_obj<D, T><<<gb, tb, 0, st>>>(S.n, S.ctl, w0, w1, S.meta[0], S.meta[1], S.pid[0], S.pid[1], S.list, S.lcount,
                                 S.cap, F, P, (T)wd, (T)lambda, B);
  k_bwd_local<D, T, true><<<gb, tb, 0, st>>>(S.n, S.ctl, w0, w1, (const LL4*)S.X[0], (const LL4*)S.X[1], S.pid[0],
                                             S.pid[1], S.list, S.lcount, S.cap, F, P, geo, B);
  return cudaGetLastError();
}

template <int D, class T>
cudaError_t launch_tape_snapshot(const DevState& S, const DevState& tape, cudaStream_t st) {
  using VT = typename ViewOf<T>::type;
  const int tb = 256, gb = grid_for(S.n > 0 ? S.n : 1, tb);
  k_tape_snapshot<VT><<<gb, tb, 0, st>>>(S.n, S.ctl, S.scal, (const LL4*)S.X[0], (const LL4*)S.X[1], S.meta[0],
                                         S.meta[1], S.pid[0], S.pid[1], (const VT*)S.view[0], (const VT*)S.view[1],
                                         (LL4*)tape.X[0], tape.meta[0], tape.pid[0], (VT*)tape.view[0], tape.ctl,
                                         tape.scal);
  return cudaGetLastError();
}

#define SPH_INSTANTIATE_ADJOINT(D, T)                                                                            \
  template cudaError_t launch_tape_snapshot<D, T>(const DevState&, const DevState&, cudaStream_t);              \
  template cudaError_t launch_bwd_step<D, T>(const DevState&, const Frame<T>&, const Phys<T>&,                  \
                                             const Geom<T>&, const AdjBufs<T>&, int, int,                        \
                                             cudaStream_t);                                                      \
  template cudaError_t launch_objective<D, T>(const DevState&, const Frame<T>&, const Phys<T>&,                 \
                                              const Geom<T>&, const AdjBufs<T>&, double, double, cudaStream_t);

}  // namespace sph
