// Relaxation-step kernels (Algorithm 1, lines 6-16), templated on the
// dimension D and the working precision T (float with split-precision
// positions, or double). Instantiated per dimension in sph_step_2d.cu /
// sph_step_3d.cu.
//
// Positions are never stored as absolute coordinates: a particle is an integer
// cell (level from its smoothing length, coordinates in that level's grid) plus
// an offset inside the cell. Pair vectors are formed as (offset difference) +
// (cell difference) * cell edge, so their rounding error is relative to the
// cell size, not to the domain size.
#pragma once

#include <cfloat>

#include "sph_internal.h"

namespace sph {

// ------------------------------------------------------------------------
// Candidate enumeration. For target i (level li, cell (cx,cy,cz), offsets o)
// visit every particle j that can satisfy r_ij < kappa max(h_i, h_ij). The
// levels searched cover h_j in h_i +- lip_h R; in each level the ball of
// radius R is cut into rows of cells along x, each row a contiguous range of
// the cell-sorted arrays, trimmed to the ball's x-extent at the row.
// ------------------------------------------------------------------------
template <int D, class T, class F>
__device__ __forceinline__ void for_each_candidate(const Grid<T>& G, const V4<T>* __restrict__ pos4,
                                                   const uint32_t* __restrict__ meta,
                                                   const uint32_t* __restrict__ cstart, int li,
                                                   int cx, int cy, int cz, T ox, T oy, T oz, T hi,
                                                   T R, F&& body) {
  const T R2 = R * R;
  const T slack = hi * T(1e-5);
  const int l0 = level_of_h(G, hi - slack - G.lip_h * R);
  const int l1 = level_of_h(G, hi + slack + G.lip_h * R);
  for (int l = l0; l <= l1; ++l) {
    int cxl = cx, cyl = cy, czl = cz;
    T fx = ox, fy = oy, fz = oz;
    change_level(G, li, l, cxl, fx);
    change_level(G, li, l, cyl, fy);
    if (D == 3) change_level(G, li, l, czl, fz);
    const T c = G.cell[l], ic = G.inv_cell[l];
    const int nx = G.nx[l], ny = G.ny[l], nz = G.nz[l];
    const uint32_t base = G.base[l];
    int zlo = 0, zhi = 0;
    if (D == 3) {
      zlo = (int)dfloor((fz - R) * ic);
      zhi = (int)dfloor((fz + R) * ic);
    }
    const int ylo = (int)dfloor((fy - R) * ic), yhi = (int)dfloor((fy + R) * ic);
    for (int dz = zlo; dz <= zhi; ++dz) {
      const int czz = czl + dz;
      if (D == 3 && (czz < 0 || czz >= nz)) continue;
      T zrel = 0, dzp = 0;
      if (D == 3) {
        zrel = fz - small_int_to_fp<T>(dz) * c;
        dzp = zrel < T(0) ? -zrel : (zrel > c ? zrel - c : T(0));
      }
      for (int dy = ylo; dy <= yhi; ++dy) {
        const int cyy = cyl + dy;
        if (cyy < 0 || cyy >= ny) continue;
        const T yrel = fy - small_int_to_fp<T>(dy) * c;
        const T dyp = yrel < T(0) ? -yrel : (yrel > c ? yrel - c : T(0));
        const T dp2 = dyp * dyp + dzp * dzp;
        if (dp2 >= R2) continue;
        const T half = dsqrt(R2 - dp2);
        int x0 = cxl + (int)dfloor((fx - half) * ic);
        int x1 = cxl + (int)dfloor((fx + half) * ic);
        x0 = x0 < 0 ? 0 : x0;
        x1 = x1 > nx - 1 ? nx - 1 : x1;
        if (x0 > x1) continue;
        const uint32_t krow = base + (uint32_t)nx * ((uint32_t)cyy + (uint32_t)ny * (uint32_t)(D == 3 ? czz : 0));
        const int jb = (int)cstart[krow + x0], je = (int)cstart[krow + x1 + 1];
        for (int j = jb; j < je; ++j) {
          const V4<T> pj = pos4[j];
          const uint32_t mj = meta[j];
          const T dx = (fx - pj.x) - small_int_to_fp<T>((int)(mj >> 8) - cxl) * c;
          const T ddy = yrel - pj.y;
          const T ddz = D == 3 ? zrel - pj.z : T(0);
          const T r2 = dx * dx + ddy * ddy + ddz * ddz;
          body(j, dx, ddy, ddz, r2, pj, mj);
        }
      }
    }
  }
}

// decode target i: level and cell coordinates from its key and meta word
template <int D, class T>
__device__ __forceinline__ void decode_cell(const Grid<T>& G, uint32_t key, uint32_t meta, int& l, int& cx,
                                            int& cy, int& cz) {
  l = level_of_key(G, key);
  const uint32_t loc = key - G.base[l];
  cx = (int)(meta >> 8);
  const uint32_t row = loc / (uint32_t)G.nx[l];
  if (D == 3) {
    cy = (int)(row % (uint32_t)G.ny[l]);
    cz = (int)(row / (uint32_t)G.ny[l]);
  } else {
    cy = (int)row;
    cz = 0;
  }
}

template <class T> __device__ __forceinline__ T pair_r(T r2);
template <> __device__ __forceinline__ float pair_r<float>(float r2) { return r2 * rsqrtf(r2); }
template <> __device__ __forceinline__ double pair_r<double>(double r2) { return sqrt(r2); }

// ---------------------------------------------------------- reductions ----
__device__ __forceinline__ double warp_min(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ long long warp_sum(long long v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// fixed-order block reduction of a Partial (deterministic)
__device__ __forceinline__ Partial block_reduce(Partial p, Partial* sm) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  p.min_rc_a = warp_min(p.min_rc_a);
  p.max_a = warp_max(p.max_a);
  p.sum_rho = warp_sum(p.sum_rho);
  p.err_l2 = warp_sum(p.err_l2);
  p.err_max = warp_max(p.err_max);
  p.ipairs = warp_sum(p.ipairs);
  p.fpairs = warp_sum(p.fpairs);
  if (lane == 0) sm[w] = p;
  __syncthreads();
  if (w == 0) {
    Partial q;
    if (lane < nw) q = sm[lane];
    else q = Partial{DBL_MAX, 0.0, 0.0, 0.0, 0.0, 0, 0, 0.0};
    q.min_rc_a = warp_min(q.min_rc_a);
    q.max_a = warp_max(q.max_a);
    q.sum_rho = warp_sum(q.sum_rho);
    q.err_l2 = warp_sum(q.err_l2);
    q.err_max = warp_max(q.err_max);
    q.ipairs = warp_sum(q.ipairs);
    q.fpairs = warp_sum(q.fpairs);
    p = q;
  }
  __syncthreads();
  return p;  // valid in warp 0
}

// --------------------------------------------------------------------------
// Density pass (general gamma): rho_i (Eq. density_sum) and p_i / rho_i^2 with
// p = P0 (rho/rho_t)^gamma (Eq. EOS_current), needed by the neighbours' forces.
// --------------------------------------------------------------------------
template <int D, class T>
__global__ void __launch_bounds__(256) k_density(int n, const V4<T>* __restrict__ pos4,
                                                 const uint32_t* __restrict__ meta,
                                                 const uint32_t* __restrict__ key,
                                                 const uint32_t* __restrict__ cstart, Grid<T> G,
                                                 Phys<T> P, T* __restrict__ rho_out, T* __restrict__ pc_out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const V4<T> pi = pos4[i];
  const uint32_t mi = meta[i];
  int li, cx, cy, cz;
  decode_cell<D, T>(G, key[i], mi, li, cx, cy, cz);
  const T hi = pi.w;
  const T Hd = P.kappa * hi, Hd2 = Hd * Hd, invHd = T(1) / Hd;
  T acc = 0;
  for_each_candidate<D, T>(G, pos4, meta, cstart, li, cx, cy, cz, pi.x, pi.y, pi.z, hi, Hd * (T(1) + T(1e-5)),
                           [&](int j, T, T, T, T r2, const V4<T>&, uint32_t) {
                             if (r2 < Hd2) {
                               const T q = r2 > T(0) ? pair_r<T>(r2) * invHd : T(0);
                               const T u = T(1) - q, u2 = u * u;
                               acc += u2 * u2 * (T(1) + T(4) * q);
                             }
                           });
  const T rho = acc * P.alpha * (D == 2 ? invHd * invHd : invHd * invHd * invHd);
  const T irt2 = inv_rho_t2<D, T>(hi, P.inv_tau);  // 1/rho_t^2
  const T rt = T(1) / dsqrt(irt2);
  rho_out[i] = rho;
  pc_out[i] = P.P0 * (T)pow((double)(rho / rt), (double)P.gamma) / (rho * rho);
}

// --------------------------------------------------------------------------
// Pass A (Algorithm 1, lines 9-13): per target i
//   rho_i = sum_j W(r_ij, h_i)                                 (Eq. density_sum)
//   a_i   = -sum_j [(P_i + P_j) + beta_ij P0 (1/rho_t,i^2 + 1/rho_t,j^2)]
//                  dW(r_ij, h_ij)/dr e_ij                      (Eqs. sph_pressure_force_2,
//                                                                   sph_st_force, sph_st_beta)
// with P = P0/rho_t^2 at gamma = 2 (Eq. EOS_2) or p/rho^2 otherwise;
// e_ij = (r_i - r_j)/r_ij, h_ij = (h_i + h_j)/2, dW/dr e_ij = -20 alpha / H^(D+2)
// (1 - q)^3 (r_i - r_j) for the Wendland C2 kernel of support H.
// Writes a_i and g_i = 0.05 rho_t,i r_c,i |a_i| (eta_i = dt1 g_i, Eq.
// viscosity_coefficient with v~ = a dt1 / 2); FP64 block partials of
// min r_c/|a|, max |a|, sum rho, sum (rho/rho_t - 1)^2, max |rho/rho_t - 1|,
// pair counts; the last block reduces them in fixed order and sets dt1, dt2
// (Eq. time_step_size, see below).
// --------------------------------------------------------------------------
template <int D, class T, bool GENERAL, bool DBG>
__global__ void __launch_bounds__(256) k_pass_a(int n, const V4<T>* __restrict__ pos4,
                                                const uint32_t* __restrict__ meta,
                                                const uint32_t* __restrict__ key,
                                                const uint32_t* __restrict__ cstart,
                                                const uint32_t* __restrict__ pid, Grid<T> G, Phys<T> P,
                                                const T* __restrict__ pc, V4<T>* __restrict__ acc_out,
                                                T* __restrict__ rho_out, Partial* __restrict__ partials,
                                                Scalars* __restrict__ scal, StepCtl* __restrict__ ctl,
                                                unsigned* __restrict__ ticket, int* __restrict__ err,
                                                int advance, int* __restrict__ dbg_count,
                                                long long* __restrict__ dbg_sum) {
  __shared__ Partial sm[8];
  __shared__ bool last;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const long long step = ctl->step;
  const T sigma = (T)sigma_of(*ctl, step);
  Partial part{DBL_MAX, 0.0, 0.0, 0.0, 0.0, 0, 0, 0.0};
  if (i < n) {
    const V4<T> pi = pos4[i];
    const uint32_t mi = meta[i];
    const uint32_t ci = mi & 0xFFu;
    int li, cx, cy, cz;
    decode_cell<D, T>(G, key[i], mi, li, cx, cy, cz);
    const T hi = pi.w;
    const T Hd = P.kappa * hi, Hd2 = Hd * Hd, invHd = T(1) / Hd;
    const T qi = inv_rho_t2<D, T>(hi, P.inv_tau);  // 1/rho_t,i^2
    const T Pi = GENERAL ? pc[i] : P.P0 * qi;
    const T half_kappa = T(0.5) * P.kappa;
    T dsum = 0, ax = 0, ay = 0, az = 0;
    int nf = 0, ni = 0, nd = 0;
    long long sd = 0, sf = 0;
    for_each_candidate<D, T>(
        G, pos4, meta, cstart, li, cx, cy, cz, pi.x, pi.y, pi.z, hi, Hd * G.rfac,
        [&](int j, T dx, T dy, T dz, T r2, const V4<T>& pj, uint32_t mj) {
          if (!GENERAL && r2 < Hd2) {
            const T q = r2 > T(0) ? pair_r<T>(r2) * invHd : T(0);
            const T u = T(1) - q, u2 = u * u;
            dsum += u2 * u2 * (T(1) + T(4) * q);
            if (DBG) {
              ++nd;
              sd += pid[j];
            }
          }
          const T Hf = half_kappa * (hi + pj.w);
          if (r2 < Hf * Hf && j != i) {
            const T invH = drcp<T>(Hf);
            const T q = pair_r<T>(r2) * invH;
            const T u = T(1) - q;
            const T invH2 = invH * invH;
            const T w = u * u * u * (D == 2 ? invH2 * invH2 : invH2 * invH2 * invH);
            const T qj = inv_rho_t2<D, T>(pj.w, P.inv_tau);
            const T Pj = GENERAL ? pc[j] : P.P0 * qj;
            const bool other = (mj & 0xFFu) != ci;
            const T coef = (Pi + Pj) + (other ? sigma * P.P0 * (qi + qj) : T(0));
            const T s = coef * w;
            ax += s * dx;
            ay += s * dy;
            az += s * dz;
            ++nf;
            ni += other;
            if (DBG) sf += pid[j];
          }
        });
    const T rho = GENERAL ? rho_out[i] : dsum * P.alpha * (D == 2 ? invHd * invHd : invHd * invHd * invHd);
    const T k20 = T(20) * P.alpha;
    ax *= k20;
    ay *= k20;
    az *= k20;
    const T an = dsqrt(ax * ax + ay * ay + az * az);
    const T rt = T(1) / dsqrt(qi);
    const T rc = Hd;
    const T g = T(0.05) * rt * rc * an;
    acc_out[i] = V4<T>{ax, ay, az, g};
    if (!GENERAL && rho_out) rho_out[i] = rho;
    const double e = (double)rho / (double)rt - 1.0;
    part.min_rc_a = an > T(0) ? (double)rc / (double)an : DBL_MAX;
    part.max_a = (double)an;
    part.sum_rho = (double)rho;
    part.err_l2 = e * e;
    part.err_max = fabs(e);
    part.ipairs = ni;
    part.fpairs = nf;
    if (!(isfinite((double)an) && isfinite((double)rho))) atomicOr(err, kErrNonfinite);
    if (DBG) {
      const uint32_t id = pid[i];
      dbg_count[2 * id] = nd;
      dbg_count[2 * id + 1] = nf;
      dbg_sum[2 * id] = sd;
      dbg_sum[2 * id + 1] = sf;
    }
  }
  part = block_reduce(part, sm);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = part;
    __threadfence();
    unsigned t = atomicAdd(ticket, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  // last block: fixed-order reduction of every block partial
  __threadfence();
  Partial acc{DBL_MAX, 0.0, 0.0, 0.0, 0.0, 0, 0, 0.0};
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
    // L2 reads: the partials were written by other blocks of this launch
    const double* qd = (const double*)&partials[b];
    const long long* ql = (const long long*)&partials[b];
    Partial q;
    q.min_rc_a = __ldcg(qd + 0);
    q.max_a = __ldcg(qd + 1);
    q.sum_rho = __ldcg(qd + 2);
    q.err_l2 = __ldcg(qd + 3);
    q.err_max = __ldcg(qd + 4);
    q.ipairs = __ldcg(ql + 5);
    q.fpairs = __ldcg(ql + 6);
    acc.min_rc_a = fmin(acc.min_rc_a, q.min_rc_a);
    acc.max_a = fmax(acc.max_a, q.max_a);
    acc.sum_rho += q.sum_rho;
    acc.err_l2 += q.err_l2;
    acc.err_max = fmax(acc.err_max, q.err_max);
    acc.ipairs += q.ipairs;
    acc.fpairs += q.fpairs;
  }
  acc = block_reduce(acc, sm);
  if (threadIdx.x == 0) {
    // Eq. time_step_size with v_n = 0 (velocity reset, line 9): line 13 keeps
    // only the body-force term, dt1 = min_i 0.25 sqrt(r_c,i/|a_i|). With
    // v~_i = a_i dt1/2 and nu_i = 0.1 r_c,i |v~_i|, line 15's terms are
    // r_c/(40|v~|) = m/(20 dt1) and 0.125 r_c^2/nu = 2.5 m/dt1, m = min r_c/|a|
    // (all three are monotone in r_c,i/|a_i|, so their minima share the argmin).
    const double m = acc.min_rc_a;
    double dt1 = 0.0, dt2 = 0.0;
    if (m < DBL_MAX) {
      dt1 = 0.25 * sqrt(m);
      dt2 = fmin(dt1, fmin(m / (20.0 * dt1), 2.5 * m / dt1));
    }
    scal->dt1 = dt1;
    scal->dt2 = dt2;
    scal->min_rc_a = m;
    scal->max_a = acc.max_a;
    scal->sum_rho = acc.sum_rho;
    scal->err_l2 = acc.err_l2;
    scal->err_max = acc.err_max;
    scal->sigma = (double)sigma;
    scal->ipairs = acc.ipairs / 2;
    scal->fpairs = acc.fpairs / 2;
    scal->wall_moved = 0;
    scal->step_of_stats = step;
    if (advance) ctl->step = step + 1;
    *ticket = 0u;
  }
}

// --------------------------------------------------------------------------
// Pass B (Algorithm 1, lines 14-16): viscous force (Eq. sph_viscous_force with
// rho := rho_t, Eq. sph_viscous_force_2), the kicks and the drift
// (Eqs. time_int_01..03) and the level-set projection (Eq. displacement_surface).
// With v~ = a dt1/2 and eta = dt1 g:
//   a~_i = (dt1^2 / 2) B_i,
//   B_i  = sum_j HM(g_i, g_j) (1/rho_t,i^2 + 1/rho_t,j^2) (dW/dr / r)(a_i - a_j),
//   v_i  = dt1 a_i / 2 + dt2 a~_i / 2,   r_i += v_i dt2.
// Then the particle is re-expressed in its (possibly new) cell and level and
// its next sort key is written; records go to the "_u" arrays.
// --------------------------------------------------------------------------
template <int D, class T, bool RECORD>
__global__ void __launch_bounds__(256) k_pass_b(int n, const V4<T>* __restrict__ pos4,
                                                const uint32_t* __restrict__ meta,
                                                const uint32_t* __restrict__ key,
                                                const uint32_t* __restrict__ cstart,
                                                const uint32_t* __restrict__ pid_s,
                                                const V4<T>* __restrict__ acc, Grid<T> G, Phys<T> P,
                                                Geom<T> geo, const Scalars* __restrict__ scal,
                                                V4<T>* __restrict__ pos_u, uint32_t* __restrict__ meta_u,
                                                uint32_t* __restrict__ key_u, uint32_t* __restrict__ pid_u,
                                                V4<T>* __restrict__ visc_out, int* __restrict__ err,
                                                unsigned long long* __restrict__ wall_moved) {
  __shared__ int moved_sm[8];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  int moved = 0;
  if (i < n) {
    const V4<T> pi = pos4[i];
    const uint32_t mi = meta[i];
    int li, cx, cy, cz;
    decode_cell<D, T>(G, key[i], mi, li, cx, cy, cz);
    const T hi = pi.w;
    const T qi = inv_rho_t2<D, T>(hi, P.inv_tau);
    const V4<T> ai = acc[i];
    const T half_kappa = T(0.5) * P.kappa;
    T bx = 0, by = 0, bz = 0;
    for_each_candidate<D, T>(G, pos4, meta, cstart, li, cx, cy, cz, pi.x, pi.y, pi.z, hi,
                             P.kappa * hi * G.rfac,
                             [&](int j, T, T, T, T r2, const V4<T>& pj, uint32_t) {
                               const T Hf = half_kappa * (hi + pj.w);
                               if (r2 < Hf * Hf && j != i) {
                                 const V4<T> aj = acc[j];
                                 const T gs = ai.w + aj.w;
                                 const T hm = gs > T(0) ? T(2) * ai.w * aj.w * drcp<T>(gs) : T(0);
                                 const T invH = drcp<T>(Hf);
                                 const T q = pair_r<T>(r2) * invH;
                                 const T u = T(1) - q;
                                 const T invH2 = invH * invH;
                                 const T w = u * u * u * (D == 2 ? invH2 * invH2 : invH2 * invH2 * invH);
                                 const T s = hm * (qi + inv_rho_t2<D, T>(pj.w, P.inv_tau)) * w;
                                 bx += s * (ai.x - aj.x);
                                 by += s * (ai.y - aj.y);
                                 bz += s * (ai.z - aj.z);
                               }
                             });
    // dW/dr / r = -20 alpha (1-q)^3 / H^(D+2)
    const T km = T(-20) * P.alpha;
    bx *= km;
    by *= km;
    bz *= km;
    const T dt1 = (T)scal->dt1, dt2 = (T)scal->dt2;
    const T kv = T(0.5) * dt1 * dt1;  // a~ = kv B
    if (RECORD) visc_out[i] = V4<T>{kv * bx, kv * by, kv * bz, T(0)};
    T d[3];
    d[0] = (T(0.5) * dt1 * ai.x + T(0.5) * dt2 * kv * bx) * dt2;
    d[1] = (T(0.5) * dt1 * ai.y + T(0.5) * dt2 * kv * by) * dt2;
    d[2] = D == 3 ? (T(0.5) * dt1 * ai.z + T(0.5) * dt2 * kv * bz) * dt2 : T(0);
    int c[3] = {cx, cy, cz};
    T o[3] = {pi.x, pi.y, pi.z};
    const bool finite = isfinite((double)d[0]) && isfinite((double)d[1]) && isfinite((double)d[2]);
    if (!finite) atomicOr(err, kErrNonfinite);
    int l = li;
    if (finite) {
      const T cl = G.cell[l], icl = G.inv_cell[l];
      const int dims[3] = {G.nx[l], G.ny[l], G.nz[l]};
      // drift and re-normalise into the cell grid of level l
      for (int k = 0; k < D; ++k) {
        o[k] += d[k];
        const int sh = (int)dfloor(o[k] * icl);
        if (sh) {
          c[k] += sh;
          o[k] -= (T)sh * cl;
        }
      }
      // bounding box (first constraint): clamp, which is the closest point
      for (int k = 0; k < D; ++k) {
        if (c[k] < 0 || (c[k] == 0 && o[k] < T(0))) {
          c[k] = 0;
          o[k] = T(0);
          moved = 1;
        } else if (c[k] > dims[k] - 1 || (c[k] == dims[k] - 1 && o[k] > G.wall_hi[l][k])) {
          c[k] = dims[k] - 1;
          o[k] = G.wall_hi[l][k];
          moved = 1;
        }
      }
      // shape constraints, in order, at the absolute position
      T xa[3] = {0, 0, 0};
      for (int k = 0; k < D; ++k) xa[k] = G.lo[k] + (T)c[k] * cl + o[k];
      int mv = 0;
      for (int s = 0; s < geo.n_shapes; ++s) mv |= project_shape(geo, s, xa, D);
      if (mv) {
        moved = 1;
        for (int k = 0; k < D; ++k) {
          const T rel = xa[k] - G.lo[k];
          int cc = (int)dfloor(rel * icl);
          cc = cc < 0 ? 0 : (cc > dims[k] - 1 ? dims[k] - 1 : cc);
          c[k] = cc;
          o[k] = rel - (T)cc * cl;
        }
      }
      // smoothing length at the new position (Algorithm 1, line 6 of the next step)
      const T hn = h_of<D, T>(geo, xa);
      const int ln = level_of_h(G, hn);
      if (ln != l) {
        for (int k = 0; k < D; ++k) {
          change_level(G, l, ln, c[k], o[k]);
          const int dn = k == 0 ? G.nx[ln] : (k == 1 ? G.ny[ln] : G.nz[ln]);
          if (c[k] > dn - 1) {
            o[k] += (T)(c[k] - (dn - 1)) * G.cell[ln];
            c[k] = dn - 1;
          }
        }
        l = ln;
      }
      const uint32_t kk = G.base[l] + (uint32_t)c[0] +
                          (uint32_t)G.nx[l] * ((uint32_t)c[1] + (uint32_t)G.ny[l] * (uint32_t)(D == 3 ? c[2] : 0));
      pos_u[i] = V4<T>{o[0], o[1], D == 3 ? o[2] : T(0), hn};
      meta_u[i] = ((uint32_t)c[0] << 8) | (mi & 0xFFu);
      key_u[i] = kk;
    } else {
      pos_u[i] = pi;
      meta_u[i] = mi;
      key_u[i] = key[i];
    }
    pid_u[i] = pid_s[i];
  }
  // count of projected particles (integer atomics: deterministic)
  int v = moved;
  for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(0xffffffffu, v, s);
  if ((threadIdx.x & 31) == 0) moved_sm[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += moved_sm[w];
    if (t) atomicAdd(wall_moved, (unsigned long long)t);
  }
}

// --------------------------------------------------------------------------
// State in / out
// --------------------------------------------------------------------------
template <int D, class T>
__global__ void __launch_bounds__(256) k_set_state(int n, const double* __restrict__ xyz,
                                                   const uint8_t* __restrict__ col, Geom<T> geo, Grid<T> G,
                                                   Grid<double> Gd, V4<T>* __restrict__ pos_u,
                                                   uint32_t* __restrict__ meta_u, uint32_t* __restrict__ key_u,
                                                   uint32_t* __restrict__ pid_u, int* __restrict__ err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double x[3] = {0, 0, 0};
  bool ok = true;
  for (int k = 0; k < D; ++k) {
    x[k] = xyz[(size_t)i * D + k];
    ok = ok && isfinite(x[k]);
  }
  if (!ok) {
    atomicOr(err, kErrNonfinite);
    for (int k = 0; k < D; ++k) x[k] = Gd.lo[k];
  }
  T xt[3] = {0, 0, 0};
  for (int k = 0; k < D; ++k) xt[k] = (T)x[k];
  const T h = h_of<D, T>(geo, xt);
  const int l = level_of_h(G, h);
  int c[3] = {0, 0, 0};
  T o[3] = {0, 0, 0};
  const int dims[3] = {G.nx[l], G.ny[l], G.nz[l]};
  for (int k = 0; k < D; ++k) {
    const double rel = x[k] - Gd.lo[k];
    int cc = (int)floor(rel * Gd.inv_cell[l]);
    if (rel < 0.0 || cc > dims[k] - 1 || (cc == dims[k] - 1 && rel - cc * Gd.cell[l] > (double)Gd.wall_hi[l][k]))
      atomicOr(err, kErrOutOfDomain);
    cc = cc < 0 ? 0 : (cc > dims[k] - 1 ? dims[k] - 1 : cc);
    c[k] = cc;
    o[k] = (T)(rel - (double)cc * Gd.cell[l]);
  }
  pos_u[i] = V4<T>{o[0], o[1], o[2], h};
  meta_u[i] = ((uint32_t)c[0] << 8) | (uint32_t)col[i];
  key_u[i] = G.base[l] + (uint32_t)c[0] + (uint32_t)G.nx[l] * ((uint32_t)c[1] + (uint32_t)G.ny[l] * (uint32_t)c[2]);
  pid_u[i] = (uint32_t)i;
}

template <int D, class T>
__global__ void __launch_bounds__(256) k_get_positions(int n, const V4<T>* __restrict__ pos_u,
                                                       const uint32_t* __restrict__ meta_u,
                                                       const uint32_t* __restrict__ key_u,
                                                       const uint32_t* __restrict__ pid_u, Grid<double> Gd,
                                                       double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int l, cx, cy, cz;
  decode_cell<D, double>(Gd, key_u[i], meta_u[i], l, cx, cy, cz);
  const V4<T> p = pos_u[i];
  const uint32_t id = pid_u[i];
  const double cl = Gd.cell[l];
  out[(size_t)id * D + 0] = Gd.lo[0] + ((double)cx * cl + (double)p.x);
  out[(size_t)id * D + 1] = Gd.lo[1] + ((double)cy * cl + (double)p.y);
  if (D == 3) out[(size_t)id * D + 2] = Gd.lo[2] + ((double)cz * cl + (double)p.z);
}

// which: 0 rho (n), 1 acc (n x D), 2 visc (n x D); source arrays in sorted order
template <int D, class T>
__global__ void __launch_bounds__(256) k_get_fields(int n, int which, const uint32_t* __restrict__ pid_s,
                                                    const T* __restrict__ rho, const V4<T>* __restrict__ acc,
                                                    const V4<T>* __restrict__ visc, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t id = pid_s[i];
  if (which == 0) {
    out[id] = (double)rho[i];
    return;
  }
  const V4<T> v = which == 1 ? acc[i] : visc[i];
  out[(size_t)id * D + 0] = (double)v.x;
  out[(size_t)id * D + 1] = (double)v.y;
  if (D == 3) out[(size_t)id * D + 2] = (double)v.z;
}

// --------------------------------------------------------------------------
// Launchers
// --------------------------------------------------------------------------
inline int grid_for(int n, int tb) { return (n + tb - 1) / tb; }

template <int D, class T>
cudaError_t launch_pass_a(const DevState& S, const Grid<T>& G, const Phys<T>& P, PassFlags f,
                          cudaStream_t st) {
  const int tb = 256, gb = grid_for(S.n, tb);
  const V4<T>* pos = (const V4<T>*)S.pos4_s;
  T* rho = (T*)S.rho;
  T* pc = (T*)S.pc;
  if (f.general_eos) {
    k_density<D, T><<<gb, tb, 0, st>>>(S.n, pos, S.meta_s, S.key_s, S.cstart, G, P, rho, pc);
  }
#define SPH_PASS_A(GEN, DBG)                                                                          \
  k_pass_a<D, T, GEN, DBG><<<gb, tb, 0, st>>>(S.n, pos, S.meta_s, S.key_s, S.cstart, S.pid_s, G, P, pc, \
                                              (V4<T>*)S.acc4, rho, S.partials, S.scal, S.ctl,         \
                                              S.tickets, S.err, f.advance, S.dbg_count, S.dbg_sum)
  if (f.general_eos) {
    if (f.nbr_debug) SPH_PASS_A(true, true);
    else SPH_PASS_A(true, false);
  } else {
    if (f.nbr_debug) SPH_PASS_A(false, true);
    else SPH_PASS_A(false, false);
  }
#undef SPH_PASS_A
  return cudaGetLastError();
}

template <int D, class T>
cudaError_t launch_pass_b(const DevState& S, const Grid<T>& G, const Phys<T>& P, const Geom<T>& g,
                          PassFlags f, cudaStream_t st) {
  const int tb = 256, gb = grid_for(S.n, tb);
  unsigned long long* wm = (unsigned long long*)&S.scal->wall_moved;
  if (f.record)
    k_pass_b<D, T, true><<<gb, tb, 0, st>>>(S.n, (const V4<T>*)S.pos4_s, S.meta_s, S.key_s, S.cstart,
                                            S.pid_s, (const V4<T>*)S.acc4, G, P, g, S.scal,
                                            (V4<T>*)S.pos4_u, S.meta_u, S.key_u, S.pid_u, (V4<T>*)S.visc,
                                            S.err, wm);
  else
    k_pass_b<D, T, false><<<gb, tb, 0, st>>>(S.n, (const V4<T>*)S.pos4_s, S.meta_s, S.key_s, S.cstart,
                                             S.pid_s, (const V4<T>*)S.acc4, G, P, g, S.scal,
                                             (V4<T>*)S.pos4_u, S.meta_u, S.key_u, S.pid_u, (V4<T>*)S.visc,
                                             S.err, wm);
  return cudaGetLastError();
}

template <int D, class T>
cudaError_t launch_set_state(const DevState& S, const Grid<T>& G, const Grid<double>& Gd, const Geom<T>& g,
                             const double* xyz, const uint8_t* col, cudaStream_t st) {
  const int tb = 256, gb = grid_for(S.n, tb);
  if (S.n > 0)
    k_set_state<D, T><<<gb, tb, 0, st>>>(S.n, xyz, col, g, G, Gd, (V4<T>*)S.pos4_u, S.meta_u, S.key_u, S.pid_u,
                                         S.err);
  return cudaGetLastError();
}

template <int D, class T>
cudaError_t launch_get_positions(const DevState& S, const Grid<double>& Gd, double* out, cudaStream_t st) {
  const int tb = 256, gb = grid_for(S.n, tb);
  if (S.n > 0)
    k_get_positions<D, T><<<gb, tb, 0, st>>>(S.n, (const V4<T>*)S.pos4_u, S.meta_u, S.key_u, S.pid_u, Gd, out);
  return cudaGetLastError();
}

template <int D, class T>
cudaError_t launch_get_fields(const DevState& S, int which, double* out, cudaStream_t st) {
  const int tb = 256, gb = grid_for(S.n, tb);
  if (S.n > 0)
    k_get_fields<D, T><<<gb, tb, 0, st>>>(S.n, which, S.pid_s, (const T*)S.rho, (const V4<T>*)S.acc4,
                                          (const V4<T>*)S.visc, out);
  return cudaGetLastError();
}

#define SPH_INSTANTIATE_STEP(D, T)                                                                        \
  template cudaError_t launch_pass_a<D, T>(const DevState&, const Grid<T>&, const Phys<T>&, PassFlags,   \
                                           cudaStream_t);                                                \
  template cudaError_t launch_pass_b<D, T>(const DevState&, const Grid<T>&, const Phys<T>&,              \
                                           const Geom<T>&, PassFlags, cudaStream_t);                     \
  template cudaError_t launch_set_state<D, T>(const DevState&, const Grid<T>&, const Grid<double>&,      \
                                              const Geom<T>&, const double*, const uint8_t*, cudaStream_t); \
  template cudaError_t launch_get_positions<D, T>(const DevState&, const Grid<double>&, double*,         \
                                                  cudaStream_t);                                         \
  template cudaError_t launch_get_fields<D, T>(const DevState&, int, double*, cudaStream_t);

}  // namespace sph
