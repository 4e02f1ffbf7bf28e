// Host-side set-up shared by the handle API and the allocation-free entry
// point: validation, parameter blocks in working precision, the Lipschitz
// bound of h and the multi-resolution grid.
#pragma once

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <string>
#include <type_traits>

#include "../../include/sphmesh.h"
#include "sph_internal.h"

namespace sph {

template <class T>
inline void fill_geom(const sph_domain& d, const sph_field& f, double hfac, double rho_scale, Geom<T>& g) {
  memset(&g, 0, sizeof g);
  g.dim = d.dim;
  g.n_shapes = d.n_shapes;
  g.field_kind = f.kind;
  g.dist_shape = f.dist_shape;
  g.n_poly = f.n_poly;
  for (int k = 0; k < 3; ++k) {
    g.lo[k] = (T)d.lo[k];
    g.hi[k] = (T)d.hi[k];
    g.ext[k] = (T)(d.hi[k] - d.lo[k]);
  }
  for (int s = 0; s < d.n_shapes; ++s) {
    g.kind[s] = d.shapes[s].kind;
    g.keep_inside[s] = d.shapes[s].keep_inside;
    for (int k = 0; k < 3; ++k) {
      g.center[s][k] = (T)d.shapes[s].center[k];
      g.size[s][k] = (T)d.shapes[s].size[k];
    }
  }
  g.s0 = (T)f.s0;
  g.a = (T)f.a;
  g.b = (T)f.b;
  for (int k = 0; k < 8; ++k) g.poly[k] = (T)f.poly[k];
  g.hfac = (T)hfac;
  g.rho_scale = (T)rho_scale;
}

template <class T>
inline void fill_phys(int dim, const sph_params& par, Phys<T>& P) {
  P.P0 = (T)par.P0;
  P.gamma = (T)par.gamma;
  P.kappa = (T)par.kappa;
  P.inv_tau = (T)(1.0 / par.tau);
  P.alpha = (T)(dim == 2 ? 7.0 / M_PI : 21.0 / (2.0 * M_PI));
}

// Upper bound of |grad s|: distance functions are 1-Lipschitz and tanh' <= 1.
inline double field_slope(const sph_field& f) {
  if (f.kind == SPH_FIELD_LINEAR_DISTANCE) return fabs(f.b);
  if (f.kind == SPH_FIELD_TANH_DISTANCE) return fabs(f.b) * f.s0;
  return 0.0;
}

// Upper bound of |grad h| over the box for h = hfac s (1+P)^(-1/d):
// |grad s| <= gslope (field_slope, with the background mesh's bounds); |P| <= sum|c_k| = S on
// x~ in [-1,1]^d; |dP/dx| <= 3 sqrt(d) S * 2/min(ext) (each monomial has
// |d/dx~| <= 3 there).
inline double lipschitz_h(const sph_domain& dom, const sph_field& f, double hfac, double smax, double gslope) {
  const int d = dom.dim;
  double S = 0.0;
  for (int k = 0; k < f.n_poly; ++k) S += fabs(f.poly[k]);
  double ext_min = DBL_MAX;
  for (int k = 0; k < d; ++k) ext_min = std::min(ext_min, dom.hi[k] - dom.lo[k]);
  const double gb = gslope;
  const double fmin = 1.0 - S;
  const double gradP = 3.0 * sqrt((double)d) * S * 2.0 / ext_min;
  const double L = hfac * (gb * pow(fmin, -1.0 / d) + smax / d * pow(fmin, -1.0 / d - 1.0) * gradP);
  return L * 1.05;
}

// Host description of the multi-resolution grid. Integer positions: one state
// unit q64 = 2^-62 L (L the power of two at or above the largest box extent),
// so coordinates stay below 2^62; the level-0 cell edge is 2^cshift units.
struct HostGrid {
  int n_levels = 1, dim = 2, cshift = 0;
  int nx[kMaxLevels], ny[kMaxLevels], nz[kMaxLevels];
  uint32_t base[kMaxLevels + 1];
  double cell[kMaxLevels];  // cell edge per level (physical)
  double q64, h0, lip_h, rfac;
};

// the grid for kernels in working precision T (cell edges in view units)
template <class T>
inline void convert_grid(const HostGrid& H, double view_unit, Grid<T>& G) {
  memset(&G, 0, sizeof G);
  G.n_levels = H.n_levels;
  G.dim = H.dim;
  G.cshift = H.cshift;
  for (int l = 0; l < H.n_levels; ++l) {
    G.nx[l] = H.nx[l];
    G.ny[l] = H.ny[l];
    G.nz[l] = H.nz[l];
    G.cellv[l] = (T)(H.cell[l] / view_unit);
  }
  for (int l = 0; l <= H.n_levels; ++l) G.base[l] = H.base[l];
  G.inv_h0 = (T)(1.0 / H.h0);
  G.lip_h = (T)H.lip_h;
  G.rfac = (T)H.rfac;
}

// Multi-resolution grid for smoothing lengths in [hmin, hmax]: level l has
// cells of edge c0 2^l, c0 the power-of-two multiple of the state unit nearest
// to cell_factor kappa h0 (h0 = 0.98 hmin), doubled until the grid has fewer
// than 2^28 cells. Returns an error message or "".
inline std::string grid_setup(const sph_domain& dom, double kappa, double cell_factor, double hmin, double hmax,
                              double lip_h, HostGrid& G) {
  const int d = dom.dim;
  const double cf = cell_factor > 0 ? cell_factor : 1.0;
  const double h0 = hmin * 0.98;
  if (!(h0 > 0)) return "target field gives a non-positive smoothing length";
  if (kappa * lip_h >= 0.75) return "target field varies too fast (kappa |grad h| >= 0.75)";
  double ext = 0.0;
  for (int k = 0; k < d; ++k) ext = std::max(ext, dom.hi[k] - dom.lo[k]);
  const double q64 = std::ldexp(std::exp2(std::ceil(std::log2(ext))), -62);
  int L = 1;
  while (L < kMaxLevels && h0 * std::ldexp(1.0, L) <= hmax) ++L;
  int m = (int)std::lround(std::log2(cf * kappa * h0 / q64));
  m = std::max(m, kViewBits + 1);
  for (; m < 62; ++m) {
    const double c0 = std::ldexp(q64, m);
    uint64_t total = 0;
    G = HostGrid{};
    for (int l = 0; l < L; ++l) {
      const double c = std::ldexp(c0, l);
      int dims[3] = {1, 1, 1};
      for (int k = 0; k < d; ++k) dims[k] = std::max(1, (int)std::min(std::ceil((dom.hi[k] - dom.lo[k]) / c), 1e9));
      G.nx[l] = dims[0];
      G.ny[l] = dims[1];
      G.nz[l] = dims[2];
      G.cell[l] = c;
      G.base[l] = (uint32_t)std::min<uint64_t>(total, 0xFFFFFFFFu);
      total += (uint64_t)dims[0] * dims[1] * dims[2];
    }
    if (total < (1ull << 28)) {
      G.base[L] = (uint32_t)total;
      G.n_levels = L;
      G.dim = d;
      G.cshift = m;
      G.q64 = q64;
      G.h0 = h0;
      G.lip_h = lip_h;
      // r < kappa h_j <= kappa (h_i + lip_h r)  =>  r < kappa h_i / (1 - kappa lip_h)
      G.rfac = (1.0 + 1e-5) / (1.0 - kappa * lip_h);
      return "";
    }
  }
  return "cell grid too large";
}

// Position frames. The integer state unit q64 divides the level-0 cell edge by
// 2^kCellShift, so cell coordinates are shifts. The FP32 view drops sv low bits
// so that every pair the passes look at spans less than 2^22 view units.
struct Frames {
  Frame<float> f;
  Frame<double> d;
  Grid<float> gf;
  Grid<double> gd;
};

inline void make_frames(const sph_domain& dom, double kappa, double skin, const HostGrid& hg, Frames& out) {
  const int dim = dom.dim;
  const double c0 = hg.cell[0];
  const double q64 = hg.q64;
  const int sv = hg.cshift - kViewBits;
  auto fill = [&](auto& F) {
    using T = std::remove_reference_t<decltype(F.qv)>;
    memset(&F, 0, sizeof F);
    F.q64 = q64;
    F.inv_q64 = 1.0 / q64;
    for (int k = 0; k < 3; ++k) {
      F.lod[k] = dom.lo[k];
      F.lo[k] = (T)dom.lo[k];
      F.xmax[k] = k < dim ? (long long)std::llround((dom.hi[k] - dom.lo[k]) / q64) : 0;
    }
    F.q64t = (T)q64;
    F.inv_q64t = (T)(1.0 / q64);
    F.s2v = std::ldexp(1.0, -hg.cshift);
    F.skin = (T)(skin * kappa);
  };
  fill(out.f);
  fill(out.d);
  // view unit = c0 for both precisions (lengths of order one in the pair math)
  out.f.qv = (float)c0;
  out.f.inv_qv = (float)(1.0 / c0);
  out.d.qv = c0;
  out.d.inv_qv = 1.0 / c0;
  out.f.sv = out.d.sv = sv;
  // 1.5 * 2^(23 - kCoarseBits): its low mantissa bit is one coarse view integer
  const float bias = (float)std::ldexp(1.5, 23 - kCoarseBits);
  int bits;
  memcpy(&bits, &bias, sizeof bits);
  out.f.mbits = bits;
  out.f.mbias = bias;
  out.f.vscale = (float)std::ldexp(1.0, -kViewBits);
  convert_grid<float>(hg, c0, out.gf);
  convert_grid<double>(hg, c0, out.gd);
}

inline sph_status validate(const sph_domain* dom, const sph_field* f, int64_t n, int32_t ncol, const sph_params* p,
                    std::string& why, const sph_background* bg = nullptr) {
  if (!dom || !f || !p) { why = "null argument"; return SPH_ERR_INVALID_ARG; }
  if (dom->dim != 2 && dom->dim != 3) { why = "dim must be 2 or 3"; return SPH_ERR_INVALID_ARG; }
  if (dom->n_shapes < 0 || dom->n_shapes > kMaxShapes) { why = "n_shapes out of range"; return SPH_ERR_INVALID_ARG; }
  for (int k = 0; k < dom->dim; ++k)
    if (!(dom->hi[k] > dom->lo[k])) { why = "empty box"; return SPH_ERR_INVALID_ARG; }
  for (int s = 0; s < dom->n_shapes; ++s) {
    const sph_shape& sh = dom->shapes[s];
    if (sh.kind == SPH_SHAPE_GRID && !(bg && bg->phi)) { why = "grid shape without a background level set"; return SPH_ERR_INVALID_ARG; }
    if (sh.kind != SPH_SHAPE_SPHERE && sh.kind != SPH_SHAPE_BOX && sh.kind != SPH_SHAPE_GRID) { why = "bad shape kind"; return SPH_ERR_INVALID_ARG; }
    if (!(sh.size[0] > 0)) { why = "bad shape size"; return SPH_ERR_INVALID_ARG; }
  }
  if (n < 0 || n > (int64_t)(1u << 30)) { why = "particle count out of range"; return SPH_ERR_INVALID_ARG; }
  if (ncol < 1 || ncol > 256) { why = "n_colors must be in 1..256"; return SPH_ERR_INVALID_ARG; }
  if (f->kind == SPH_FIELD_UNIFORM) {
    if (!(f->s0 > 0)) { why = "s0 must be > 0"; return SPH_ERR_INVALID_ARG; }
  } else if (f->kind == SPH_FIELD_LINEAR_DISTANCE || f->kind == SPH_FIELD_TANH_DISTANCE) {
    if (!(f->a > 0) || !(f->b >= 0) || f->dist_shape < 0 || f->dist_shape >= dom->n_shapes) {
      why = "bad distance field";
      return SPH_ERR_INVALID_ARG;
    }
    if (f->kind == SPH_FIELD_TANH_DISTANCE && !(f->s0 > 0)) {
      why = "tanh field needs s0 > 0 (reciprocal length)";
      return SPH_ERR_INVALID_ARG;
    }
  } else if (f->kind == SPH_FIELD_BACKGROUND) {
    if (!(bg && bg->spacing)) { why = "background field without background spacing"; return SPH_ERR_INVALID_ARG; }
  } else { why = "bad field kind"; return SPH_ERR_INVALID_ARG; }
  if (bg) {
    int64_t nodes = 1;
    for (int k = 0; k < 3; ++k) {
      const int need = k < dom->dim ? 2 : 1;
      if (bg->dims[k] < need || (k >= dom->dim && bg->dims[k] != 1)) { why = "background mesh dims"; return SPH_ERR_INVALID_ARG; }
      nodes *= bg->dims[k];
      if (k < dom->dim && !(bg->lo[k] <= dom->lo[k] && bg->hi[k] >= dom->hi[k] && bg->hi[k] > bg->lo[k])) {
        why = "background mesh must contain the domain box";
        return SPH_ERR_INVALID_ARG;
      }
    }
    if (nodes > (int64_t)1 << 28) { why = "background mesh too large"; return SPH_ERR_INVALID_ARG; }
    if (bg->spacing)
      for (int64_t q = 0; q < nodes; ++q)
        if (!(bg->spacing[q] > 0) || !std::isfinite(bg->spacing[q])) { why = "background spacing must be > 0"; return SPH_ERR_INVALID_ARG; }
    if (bg->phi)
      for (int64_t q = 0; q < nodes; ++q)
        if (!std::isfinite(bg->phi[q])) { why = "background level set must be finite"; return SPH_ERR_INVALID_ARG; }
  }
  if (f->n_poly < 0 || f->n_poly > 8) { why = "n_poly out of range"; return SPH_ERR_INVALID_ARG; }
  double S = 0;
  for (int k = 0; k < f->n_poly; ++k) S += fabs(f->poly[k]);
  if (!(S < 1.0)) { why = "sum |poly| must be < 1"; return SPH_ERR_INVALID_ARG; }
  if (!(f->rho_scale >= 0)) { why = "rho_scale must be >= 0"; return SPH_ERR_INVALID_ARG; }
  if (!(p->P0 > 0) || !(p->gamma > 0) || !(p->sigma0 >= 0) || !(p->tau > 0) || !(p->kappa > 0)) {
    why = "P0, gamma, tau, kappa must be > 0 and sigma0 >= 0";
    return SPH_ERR_INVALID_ARG;
  }
  if (p->precision != SPH_PREC_FP32_SPLIT && p->precision != SPH_PREC_FP64) { why = "bad precision"; return SPH_ERR_INVALID_ARG; }
  if (p->kernel_id != 0) { why = "only kernel_id 0 (Wendland C2) exists"; return SPH_ERR_INVALID_ARG; }
  return SPH_OK;
}


}  // namespace sph
