/*
 * FP64 CPU oracle of the multi-phase SPH relaxation step (arXiv 1906.07925).
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * CPU-baseline leg of the bench, never by the product path.
 *
 * Each function cites the passage it follows. Where the paper is silent or
 * self-contradictory the reading taken is stated at the point of use.
 */
#include "sph_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PI 3.14159265358979323846

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Kernel. The paper uses "a smooth isotropic kernel" (Sec. 3.3) without     */
/* printing it. Reading: Wendland C2, W = alpha_d (1-q)^4 (1+4q), q = r/H,    */
/* alpha_2 = 7/(pi H^2), alpha_3 = 21/(2 pi H^3); zero for q >= 1.           */
/* ------------------------------------------------------------------------ */
static double wendland_alpha(double H, int dim) {
  return dim == 2 ? 7.0 / (PI * H * H) : 21.0 / (2.0 * PI * H * H * H);
}

double orc_W(double r, double H, int dim) {
  double q = r / H;
  if (q >= 1.0) return 0.0;
  double u = 1.0 - q;
  return wendland_alpha(H, dim) * u * u * u * u * (1.0 + 4.0 * q);
}

/* dW/dr = alpha_d / H * d/dq[(1-q)^4 (1+4q)] = alpha_d / H * (-20 q (1-q)^3). */
double orc_dW(double r, double H, int dim) {
  double q = r / H;
  if (q >= 1.0) return 0.0;
  double u = 1.0 - q;
  return wendland_alpha(H, dim) / H * (-20.0 * q * u * u * u);
}

/* (dW/dr) / r, written out so that it is defined at r = 0 as its limit:
 * dW/dr = -20 alpha q u^3 / H is linear in r there, so the ratio tends to
 * -20 alpha / H^2 (coincident particles). */
double orc_dW_over_r(double r, double H, int dim) {
  double q = r / H;
  if (q >= 1.0) return 0.0;
  double u = 1.0 - q;
  return wendland_alpha(H, dim) / (H * H) * (-20.0 * u * u * u);
}

/* ------------------------------------------------------------------------ */
/* Geometry: level set phi, positive in the mesh region (Sec. 3.1,           */
/* Eq. level_set_function). The region is the box [lo,hi] intersected with  */
/* each shape constraint; phi is the minimum of the constraint distances.    */
/* ------------------------------------------------------------------------ */

/* Interpolation on the Cartesian background mesh (Sec. 3.1: the level set is
 * discretised on it; Sec. 3.2: the target density is interpolated from it at
 * the particle positions). Reading: multilinear interpolation of the node
 * values (bilinear in 2D, trilinear in 3D) in the cell that holds x, x clamped
 * into the mesh box; grad receives the gradient of the interpolant there. */
static double bg_interp(const orc_problem* p, const double* v, const double* x, double* grad) {
  int d = p->dim, i0[3] = {0, 0, 0};
  double f[3] = {0, 0, 0}, h[3] = {1, 1, 1};
  for (int k = 0; k < d; ++k) {
    int n = p->bg_dims[k];
    h[k] = (p->bg_hi[k] - p->bg_lo[k]) / (n - 1);
    double t = (x[k] - p->bg_lo[k]) / h[k];
    if (t < 0.0) t = 0.0;
    if (t > n - 1) t = n - 1;
    int i = (int)floor(t);
    if (i > n - 2) i = n - 2;
    i0[k] = i;
    f[k] = t - i;
  }
  double val = 0.0, g[3] = {0, 0, 0};
  int corners = 1 << d;
  for (int c = 0; c < corners; ++c) {
    int idx[3] = {0, 0, 0};
    double w = 1.0, dw[3] = {1, 1, 1};
    for (int k = 0; k < d; ++k) {
      int b = (c >> k) & 1;
      idx[k] = i0[k] + b;
      double wk = b ? f[k] : 1.0 - f[k];
      double dk = (b ? 1.0 : -1.0) / h[k];
      for (int m = 0; m < d; ++m) dw[m] *= (m == k) ? dk : wk;
      w *= wk;
    }
    double node = v[idx[0] + (int64_t)p->bg_dims[0] * (idx[1] + (int64_t)p->bg_dims[1] * idx[2])];
    val += w * node;
    for (int m = 0; m < d; ++m) g[m] += dw[m] * node;
  }
  if (grad)
    for (int k = 0; k < 3; ++k) grad[k] = k < d ? g[k] : 0.0;
  return val;
}

/* signed distance, positive inside the shape */
static double shape_inside_distance(const orc_problem* p, const orc_shape* s, const double* x, int dim) {
  if (s->kind == ORC_GRID) return bg_interp(p, p->bg_phi, x, NULL);
  if (s->kind == ORC_SPHERE) {
    double r2 = 0.0;
    for (int k = 0; k < dim; ++k) r2 += (x[k] - s->center[k]) * (x[k] - s->center[k]);
    return s->size[0] - sqrt(r2);
  }
  double outside2 = 0.0, qmax = -INFINITY;
  for (int k = 0; k < dim; ++k) {
    double q = fabs(x[k] - s->center[k]) - s->size[k];
    if (q > 0) outside2 += q * q;
    if (q > qmax) qmax = q;
  }
  double inside = qmax < 0 ? qmax : 0.0;
  return -(sqrt(outside2) + inside);
}

static double constraint_phi(const orc_problem* p, const orc_shape* s, const double* x, int dim) {
  double v = shape_inside_distance(p, s, x, dim);
  return s->keep_inside ? v : -v;
}

static orc_shape box_shape(const orc_problem* p) {
  orc_shape b;
  b.kind = ORC_BOX;
  b.keep_inside = 1;
  for (int k = 0; k < 3; ++k) {
    b.center[k] = 0.5 * (p->lo[k] + p->hi[k]);
    b.size[k] = 0.5 * (p->hi[k] - p->lo[k]);
  }
  return b;
}

double orc_phi(const orc_problem* p, const double* x) {
  orc_shape b = box_shape(p);
  double phi = constraint_phi(p, &b, x, p->dim);
  for (int s = 0; s < p->n_shapes; ++s) {
    double v = constraint_phi(p, &p->shapes[s], x, p->dim);
    if (v < phi) phi = v;
  }
  return phi;
}

/* Eq. displacement_surface, r <- r - phi N with N = grad(phi), for a particle
 * that left the region (phi < 0). For an exact distance function this moves the
 * point to the closest point of the violated constraint's surface:
 *  - box kept inside: clamp to the box;
 *  - box kept outside: push out through the nearest face;
 *  - sphere (either side): c + R (x - c)/|x - c|.
 *  - background-mesh level set: N = grad(phi) / |grad(phi)|^2 of the
 *    interpolant (Newton's step towards phi = 0, the printed step when |grad
 *    phi| = 1), taken three times from the point that violated it.
 * Reading: constraints are applied in order, the bounding box first. */
static int project_one(const orc_problem* p, const orc_shape* s, double* x, int dim) {
  double phi = constraint_phi(p, s, x, dim);
  if (!(phi < 0.0)) return 0;
  if (s->kind == ORC_GRID) {
    double sg = s->keep_inside ? 1.0 : -1.0;
    for (int it = 0; it < 3; ++it) {
      double g[3];
      double v = sg * bg_interp(p, p->bg_phi, x, g);
      double g2 = 0.0;
      for (int k = 0; k < dim; ++k) g2 += g[k] * g[k];
      if (!(g2 > 0.0)) break;
      for (int k = 0; k < dim; ++k) x[k] -= v * sg * g[k] / g2;
    }
    return 1;
  }
  if (s->kind == ORC_SPHERE) {
    double d[3] = {0, 0, 0}, r2 = 0.0;
    for (int k = 0; k < dim; ++k) { d[k] = x[k] - s->center[k]; r2 += d[k] * d[k]; }
    double r = sqrt(r2);
    if (r == 0.0) { d[0] = 1.0; r = 1.0; }
    for (int k = 0; k < dim; ++k) x[k] = s->center[k] + s->size[0] * d[k] / r;
    return 1;
  }
  if (s->keep_inside) {
    for (int k = 0; k < dim; ++k) {
      double lo = s->center[k] - s->size[k], hi = s->center[k] + s->size[k];
      if (x[k] < lo) x[k] = lo;
      if (x[k] > hi) x[k] = hi;
    }
    return 1;
  }
  /* inside a box that must be kept outside: leave through the nearest face */
  int best = 0; double bestd = INFINITY, sign = 1.0;
  for (int k = 0; k < dim; ++k) {
    double dlo = x[k] - (s->center[k] - s->size[k]);
    double dhi = (s->center[k] + s->size[k]) - x[k];
    if (dlo < bestd) { bestd = dlo; best = k; sign = -1.0; }
    if (dhi < bestd) { bestd = dhi; best = k; sign = 1.0; }
  }
  x[best] = s->center[best] + sign * s->size[best];
  return 1;
}

/* Feature-surface particles (Sec. 3.5). Reading: a surface particle belongs to
 * the constraint surface nearest to it (the constraint value of smallest
 * magnitude, the bounding box first on ties); N is that constraint's unit
 * normal (the gradient of its signed distance, pointing into the region). */
static const orc_shape* nearest_constraint(const orc_problem* p, const double* x, orc_shape* box, double* phi) {
  *box = box_shape(p);
  const orc_shape* best = box;
  double bv = constraint_phi(p, box, x, p->dim);
  for (int s = 0; s < p->n_shapes; ++s) {
    double v = constraint_phi(p, &p->shapes[s], x, p->dim);
    if (fabs(v) < fabs(bv)) { bv = v; best = &p->shapes[s]; }
  }
  *phi = bv;
  return best;
}

static void inside_distance_grad(const orc_problem* p, const orc_shape* s, const double* x, int dim, double* g);

/* gradient of a constraint's value (the signed distance with the region positive) */
static void constraint_grad(const orc_problem* p, const orc_shape* s, const double* x, int dim, double* g) {
  inside_distance_grad(p, s, x, dim, g);
  if (!s->keep_inside)
    for (int k = 0; k < 3; ++k) g[k] = -g[k];
}

/* unit normal N(r_i) of the surface a feature-surface particle belongs to;
 * zero where the gradient vanishes */
static void surface_normal(const orc_problem* p, const double* x, double* N) {
  orc_shape box;
  double phi;
  const orc_shape* s = nearest_constraint(p, x, &box, &phi);
  constraint_grad(p, s, x, p->dim, N);
  double n2 = 0.0;
  for (int k = 0; k < p->dim; ++k) n2 += N[k] * N[k];
  double inv = n2 > 0.0 ? 1.0 / sqrt(n2) : 0.0;
  for (int k = 0; k < 3; ++k) N[k] *= inv;
}

/* Eq. force_surface: drop the normal component, F <- F - (N . F) N */
static void tangential(const double* N, double* F, int dim) {
  double dn = 0.0;
  for (int k = 0; k < dim; ++k) dn += N[k] * F[k];
  for (int k = 0; k < dim; ++k) F[k] -= dn * N[k];
}

/* Eq. displacement_surface for a feature-surface particle, applied after every
 * drift whatever the sign of phi: r <- r - phi N onto the nearest constraint
 * surface (the closest point for the exact distance functions of the sphere
 * and the box; three Newton steps for the background level set). */
static void project_to_surface(const orc_problem* p, double* x) {
  orc_shape box;
  double phi;
  const orc_shape* s = nearest_constraint(p, x, &box, &phi);
  int d = p->dim;
  if (s->kind == ORC_GRID) {
    double sg = s->keep_inside ? 1.0 : -1.0;
    for (int it = 0; it < 3; ++it) {
      double g[3];
      double v = sg * bg_interp(p, p->bg_phi, x, g);
      double g2 = 0.0;
      for (int k = 0; k < d; ++k) g2 += g[k] * g[k];
      if (!(g2 > 0.0)) break;
      for (int k = 0; k < d; ++k) x[k] -= v * sg * g[k] / g2;
    }
    return;
  }
  double g[3];
  constraint_grad(p, s, x, d, g);
  for (int k = 0; k < d; ++k) x[k] -= phi * g[k];
}

int orc_project(const orc_problem* p, double* x) {
  orc_shape b = box_shape(p);
  int moved = project_one(p, &b, x, p->dim);
  for (int s = 0; s < p->n_shapes; ++s) moved |= project_one(p, &p->shapes[s], x, p->dim);
  return moved;
}

/* ------------------------------------------------------------------------ */
/* Target information (Sec. 2.3, Eq. rho_target_function; Sec. 3.2).         */
/* rho_t = rho_scale * s(x)^-d * (1 + sum_k poly_k b_k(x~)), where s is the   */
/* user spacing shape (uniform s0, or a + b * distance to a shape surface).   */
/* ------------------------------------------------------------------------ */
static double poly_factor(const orc_problem* p, const double* x) {
  if (p->n_poly <= 0) return 1.0;
  double t[3];
  for (int k = 0; k < p->dim; ++k) t[k] = 2.0 * (x[k] - p->lo[k]) / (p->hi[k] - p->lo[k]) - 1.0;
  double b[8];
  if (p->dim == 2) {
    double X = t[0], Y = t[1];
    b[0] = X; b[1] = Y; b[2] = X * X; b[3] = X * Y; b[4] = Y * Y;
    b[5] = X * X * X; b[6] = X * X * Y; b[7] = X * Y * Y;
  } else {
    double X = t[0], Y = t[1], Z = t[2];
    b[0] = X; b[1] = Y; b[2] = Z; b[3] = X * X; b[4] = Y * Y; b[5] = Z * Z;
    b[6] = X * Y; b[7] = Y * Z;
  }
  double f = 1.0;
  for (int k = 0; k < p->n_poly && k < 8; ++k) f += p->poly[k] * b[k];
  return f;
}

/* Target spacing s(x). The circle case of Sec. 4.1 prescribes the target
 * size h_min + tanh(2.5 phi / 43) / tanh(2.5) (h_max - h_min), phi the
 * distance to the circle: kind ORC_FIELD_TANH_DISTANCE with a = h_min,
 * b = (h_max - h_min) / tanh(2.5) and s0 = 2.5 / 43. */
static double spacing(const orc_problem* p, const double* x) {
  if (p->field_kind == ORC_FIELD_UNIFORM) return p->s0;
  if (p->field_kind == ORC_FIELD_BACKGROUND) return bg_interp(p, p->bg_s, x, NULL);
  double dist = fabs(shape_inside_distance(p, &p->shapes[p->dist_shape], x, p->dim));
  if (p->field_kind == ORC_FIELD_TANH_DISTANCE) return p->a + p->b * tanh(p->s0 * dist);
  return p->a + p->b * dist;
}

/* ds/d|dist| of the distance fields */
static double spacing_slope(const orc_problem* p, double dist) {
  if (p->field_kind == ORC_FIELD_TANH_DISTANCE) {
    double t = tanh(p->s0 * fabs(dist));
    return p->b * p->s0 * (1.0 - t * t);
  }
  return p->b;
}

double orc_rho_t(const orc_problem* p, const double* x) {
  double s = spacing(p, x);
  return p->rho_scale * pow(s, -(double)p->dim) * poly_factor(p, x);
}

/* Eq. scale_SPH_particle with m_i = 1 (Eq. mass_SPH_particle). */
double orc_h(const orc_problem* p, const double* x) {
  return p->tau * pow(1.0 / orc_rho_t(p, x), 1.0 / p->dim);
}

/* Eq. sph_st_sigma (the printed ramp, read with t in steps): sigma0 up to t0,
 * sigma0 (1 - (t0 - t)/(t0 - t1)) on (t0, t1], 0 afterwards. */
double orc_sigma(const orc_problem* p, double t) {
  if (p->t0 < 0.0 || t <= p->t0) return p->sigma0;
  if (t <= p->t1) return p->sigma0 * (1.0 - (p->t0 - t) / (p->t0 - p->t1));
  return 0.0;
}

/* Eq. total_mass_2: M_v = integral of rho_t over the positive phase. */
double orc_total_mass(const orc_problem* p, int res) {
  int d = p->dim;
  double step[3], cellvol = 1.0;
  for (int k = 0; k < d; ++k) { step[k] = (p->hi[k] - p->lo[k]) / res; cellvol *= step[k]; }
  int64_t total = 1;
  for (int k = 0; k < d; ++k) total *= res;
  double sum = 0.0;
#pragma omp parallel for reduction(+ : sum) schedule(static)
  for (int64_t c = 0; c < total; ++c) {
    double x[3] = {0, 0, 0};
    int64_t r = c;
    for (int k = 0; k < d; ++k) { x[k] = p->lo[k] + ((double)(r % res) + 0.5) * step[k]; r /= res; }
    if (orc_phi(p, x) > 0.0) sum += orc_rho_t(p, x);
  }
  return sum * cellvol;
}

/* ------------------------------------------------------------------------ */
/* Neighbour search (the neighbour sets of Algorithm 1).                     */
/* Density set of i: all j (self included) with r_ij < kappa h_i            */
/*   (Eq. density_sum gathers with h_i).                                     */
/* Force set of i: all j != i with r_ij < kappa h_ij, h_ij = (h_i + h_j)/2   */
/*   (Eq. sph_pressure_force_2).                                            */
/* The union is found by brute force or a uniform grid; lists are ascending. */
/* ------------------------------------------------------------------------ */
typedef struct {
  int64_t* dstart; int32_t* dlist;  /* CSR density sets */
  int64_t* fstart; int32_t* flist;  /* CSR force sets */
} nbr_sets;

static double dist2(const double* a, const double* b, int d) {
  double s = 0.0;
  for (int k = 0; k < d; ++k) s += (a[k] - b[k]) * (a[k] - b[k]);
  return s;
}

typedef struct {
  int d; double lo[3]; double c; int64_t nc[3];
  int64_t* start; int32_t* items;
} ugrid;

static int64_t cell_coord(double x, double lo, double c, int64_t nc) {
  int64_t v = (int64_t)floor((x - lo) / c);
  if (v < 0) v = 0;
  if (v >= nc) v = nc - 1;
  return v;
}

static int ugrid_build(ugrid* g, const orc_problem* p, int64_t n, const double* pos, double c) {
  int d = p->dim;
  g->d = d; g->c = c;
  int64_t total = 1;
  for (int k = 0; k < 3; ++k) {
    g->lo[k] = p->lo[k];
    g->nc[k] = 1;
    if (k < d) {
      g->nc[k] = (int64_t)ceil((p->hi[k] - p->lo[k]) / c);
      if (g->nc[k] < 1) g->nc[k] = 1;
    }
    total *= g->nc[k];
  }
  g->start = (int64_t*)calloc((size_t)total + 1, sizeof(int64_t));
  g->items = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  int64_t* cell = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  if (!g->start || !g->items || !cell) { free(cell); return -1; }
  for (int64_t i = 0; i < n; ++i) {
    int64_t id = 0, mul = 1;
    for (int k = 0; k < d; ++k) { id += cell_coord(pos[i * d + k], g->lo[k], c, g->nc[k]) * mul; mul *= g->nc[k]; }
    cell[i] = id;
    g->start[id + 1]++;
  }
  for (int64_t t = 0; t < total; ++t) g->start[t + 1] += g->start[t];
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)total);
  if (!fill) { free(cell); return -1; }
  memcpy(fill, g->start, sizeof(int64_t) * (size_t)total);
  for (int64_t i = 0; i < n; ++i) g->items[fill[cell[i]]++] = (int32_t)i;  /* ascending i per cell */
  free(fill); free(cell);
  return 0;
}

static void ugrid_free(ugrid* g) { free(g->start); free(g->items); }

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

/* candidates of i: every j whose distance could satisfy either criterion
 * (r_ij < kappa max(h_i, h_ij) <= kappa (h_i + hmax)/2) */
static int32_t gather_candidates(const ugrid* g, const double* pos, int64_t i, double R, int32_t* out, int64_t cap) {
  int d = g->d;
  int64_t lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  for (int k = 0; k < d; ++k) {
    lo[k] = cell_coord(pos[i * d + k] - R, g->lo[k], g->c, g->nc[k]);
    hi[k] = cell_coord(pos[i * d + k] + R, g->lo[k], g->c, g->nc[k]);
  }
  int64_t cnt = 0;
  for (int64_t cz = lo[2]; cz <= hi[2]; ++cz)
    for (int64_t cy = lo[1]; cy <= hi[1]; ++cy)
      for (int64_t cx = lo[0]; cx <= hi[0]; ++cx) {
        int64_t id = cx + g->nc[0] * (cy + g->nc[1] * cz);
        for (int64_t t = g->start[id]; t < g->start[id + 1]; ++t) {
          if (cnt < cap) out[cnt] = g->items[t];
          cnt++;
        }
      }
  return (int32_t)cnt;
}

static int build_sets(const orc_problem* p, int64_t n, const double* pos, const double* h,
                      int mode, nbr_sets* S) {
  int d = p->dim;
  double kappa = p->kappa;
  double hmax = 0.0, hmin = INFINITY;
  for (int64_t i = 0; i < n; ++i) { if (h[i] > hmax) hmax = h[i]; if (h[i] < hmin) hmin = h[i]; }
  ugrid g; memset(&g, 0, sizeof g);
  if (mode == 1 && n > 0) {
    /* cells of the smallest support; each i scans the cells within its reach */
    double c = kappa * hmin;
    double ext = 0.0;
    for (int k = 0; k < d; ++k) if (p->hi[k] - p->lo[k] > ext) ext = p->hi[k] - p->lo[k];
    /* keep the grid at most ~16M cells */
    if (d == 3 && c < ext / 256.0) c = ext / 256.0;
    if (d == 2 && c < ext / 4096.0) c = ext / 4096.0;
    if (ugrid_build(&g, p, n, pos, c) != 0) return -1;
  }
  S->dstart = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  S->fstart = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  if (!S->dstart || !S->fstart) return -1;
  int32_t* dcount = (int32_t*)calloc((size_t)n + 1, sizeof(int32_t));
  int32_t* fcount = (int32_t*)calloc((size_t)n + 1, sizeof(int32_t));
  int err = 0;
  /* pass 1: counts; pass 2: fill */
  for (int pass = 0; pass < 2 && !err; ++pass) {
#pragma omp parallel
    {
      int64_t cap = 1024;
      int32_t* cand = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
#pragma omp for schedule(dynamic, 256)
      for (int64_t i = 0; i < n; ++i) {
        const double* xi = pos + i * d;
        double Rd = kappa * h[i];
        int64_t nd = 0, nf = 0;
        int32_t m;
        if (mode == 1) {
          double R = kappa * 0.5 * (h[i] + hmax);
          if (R < Rd) R = Rd;
          m = gather_candidates(&g, pos, i, R, cand, cap);
          if (m > cap) {
            cap = 2 * (int64_t)m;
            cand = (int32_t*)realloc(cand, sizeof(int32_t) * (size_t)cap);
            m = gather_candidates(&g, pos, i, R, cand, cap);
          }
          qsort(cand, (size_t)m, sizeof(int32_t), cmp_i32);
        } else {
          m = (int32_t)n;
        }
        for (int32_t t = 0; t < m; ++t) {
          int64_t j = mode == 1 ? cand[t] : t;
          double r = sqrt(dist2(xi, pos + j * d, d));
          int in_d = r < Rd;
          int in_f = (j != i) && r < kappa * 0.5 * (h[i] + h[j]);
          if (pass == 1) {
            if (in_d) S->dlist[S->dstart[i] + nd] = (int32_t)j;
            if (in_f) S->flist[S->fstart[i] + nf] = (int32_t)j;
          }
          nd += in_d; nf += in_f;
        }
        if (pass == 0) { dcount[i] = (int32_t)nd; fcount[i] = (int32_t)nf; }
      }
      free(cand);
    }
    if (pass == 0) {
      for (int64_t i = 0; i < n; ++i) {
        S->dstart[i + 1] = S->dstart[i] + dcount[i];
        S->fstart[i + 1] = S->fstart[i] + fcount[i];
      }
      S->dlist = (int32_t*)malloc(sizeof(int32_t) * (size_t)(S->dstart[n] + 1));
      S->flist = (int32_t*)malloc(sizeof(int32_t) * (size_t)(S->fstart[n] + 1));
      if (!S->dlist || !S->flist) err = 1;
    }
  }
  free(dcount); free(fcount);
  if (mode == 1 && n > 0) ugrid_free(&g);
  return err ? -1 : 0;
}

static void free_sets(nbr_sets* S) { free(S->dstart); free(S->dlist); free(S->fstart); free(S->flist); }

int orc_neighbor_sets(const orc_problem* p, int64_t n, const double* pos, int mode,
                      int32_t* dens_count, int32_t* force_count,
                      int64_t* dens_idsum, int64_t* force_idsum,
                      int64_t* dens_idxor, int64_t* force_idxor) {
  double* h = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  if (!h) return -1;
  for (int64_t i = 0; i < n; ++i) h[i] = orc_h(p, pos + i * p->dim);
  nbr_sets S; memset(&S, 0, sizeof S);
  if (build_sets(p, n, pos, h, mode, &S) != 0) { free(h); return -1; }
  for (int64_t i = 0; i < n; ++i) {
    int64_t s = 0, x = 0;
    for (int64_t t = S.dstart[i]; t < S.dstart[i + 1]; ++t) { s += S.dlist[t]; x ^= S.dlist[t]; }
    if (dens_count) dens_count[i] = (int32_t)(S.dstart[i + 1] - S.dstart[i]);
    if (dens_idsum) dens_idsum[i] = s;
    if (dens_idxor) dens_idxor[i] = x;
    s = 0; x = 0;
    for (int64_t t = S.fstart[i]; t < S.fstart[i + 1]; ++t) { s += S.flist[t]; x ^= S.flist[t]; }
    if (force_count) force_count[i] = (int32_t)(S.fstart[i + 1] - S.fstart[i]);
    if (force_idsum) force_idsum[i] = s;
    if (force_idxor) force_idxor[i] = x;
  }
  free_sets(&S); free(h);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Cell keys of the multi-resolution grid (the neighbour search of           */
/* Algorithm 1): each particle is filed at the level of its smoothing length */
/* and, within that level, in the cell that holds it.                        */
/* ------------------------------------------------------------------------ */
int orc_cell_keys(const orc_problem* p, int64_t n, const double* pos, const orc_grid* g, uint32_t* keys,
                  double* h_out) {
  const int d = p->dim;
  for (int64_t i = 0; i < n; ++i) {
    const double* x = pos + i * d;
    double h = orc_h(p, x);
    if (h_out) h_out[i] = h;
    /* level: the largest l with 2^l h0 <= h, at least 0, at most n_levels - 1 */
    int l = 0;
    while (l + 1 < g->n_levels && h >= ldexp(g->h0, l + 1)) ++l;
    int64_t c[3] = {0, 0, 0};
    for (int k = 0; k < d; ++k) {
      int64_t v = (int64_t)floor((x[k] - g->lo[k]) / g->cell[l]);
      if (v < 0) v = 0;
      if (v > g->dims[l][k] - 1) v = g->dims[l][k] - 1;
      c[k] = v;
    }
    keys[i] = g->base[l] + (uint32_t)(c[0] + (int64_t)g->dims[l][0] * (c[1] + (int64_t)g->dims[l][1] * c[2]));
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* One relaxation step (Algorithm 1).                                        */
/* ------------------------------------------------------------------------ */
static int step_core(const orc_problem* p, int64_t n, double* pos, const uint8_t* col, int64_t step,
                     int mode, const double* dt_fixed, orc_step_info* info, double* rho_out,
                     double* acc_out, double* visc_out, double* pair_abs_a, double* pair_abs_b) {
  const int d = p->dim;
  const double kappa = p->kappa, P0 = p->P0, gamma = p->gamma;
  const double sigma = orc_sigma(p, (double)step);
  orc_step_info I; memset(&I, 0, sizeof I);
  I.sigma = sigma;
  if (n <= 0) { if (info) *info = I; return 0; }

  size_t nd = (size_t)n * (size_t)d;
  double* h = (double*)malloc(sizeof(double) * (size_t)n);
  double* rt = (double*)malloc(sizeof(double) * (size_t)n);
  double* rho = (double*)malloc(sizeof(double) * (size_t)n);
  double* Pc = (double*)malloc(sizeof(double) * (size_t)n);
  double* a = (double*)malloc(sizeof(double) * nd);
  double* vt = (double*)malloc(sizeof(double) * nd);
  double* at = (double*)malloc(sizeof(double) * nd);
  double* eta = (double*)malloc(sizeof(double) * (size_t)n);
  if (!h || !rt || !rho || !Pc || !a || !vt || !at || !eta) return -1;

  /* target density and scale at r_i^n */
  for (int64_t i = 0; i < n; ++i) {
    rt[i] = orc_rho_t(p, pos + i * d);
    h[i] = p->tau * pow(1.0 / rt[i], 1.0 / d);
  }
  /* neighbour sets */
  nbr_sets S; memset(&S, 0, sizeof S);
  if (build_sets(p, n, pos, h, mode, &S) != 0) return -1;

  /* Eq. density_sum: rho_i = sum_j m_j W(r_ij, h_i), m_j = 1 */
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t t = S.dstart[i]; t < S.dstart[i + 1]; ++t) {
      int64_t j = S.dlist[t];
      s += orc_W(sqrt(dist2(pos + i * d, pos + j * d, d)), kappa * h[i], d);
    }
    rho[i] = s;
  }
  /* Pressure coefficient p_i / rho_i^2 with the EOS p = P0 (rho/rho_t)^gamma
   * (Eq. EOS_current). For gamma = 2 it is P0 / rho_t^2 and the density drops out
   * (Eq. EOS_2 / sph_pressure_force_2); the printed gamma = 2 form is used then. */
  for (int64_t i = 0; i < n; ++i) {
    if (gamma == 2.0 && !p->eos_general) Pc[i] = P0 / (rt[i] * rt[i]);
    else Pc[i] = P0 * pow(rho[i] / rt[i], gamma) / (rho[i] * rho[i]);
  }

  /* velocity reset (v_n = 0, infinite friction, Sec. 3.3);
   * a_n = -F_p + F_s (Eq. momentum_equation without F_v), with
   *   F_p,i = sum_j (P_i + P_j) dW(r_ij, h_ij)/dr e_ij          (pressure)
   *   F_s,i = -sum_j beta_ij (P0/rho_t,i^2 + P0/rho_t,j^2) dW e_ij (surface tension)
   * beta_ij = sigma(t) for distinct colours, 0 otherwise (Eq. sph_st_beta).
   * Reading: e_ij = (r_i - r_j)/r_ij (the paper defines r_ij = r_i - r_j but
   * calls e_ij "from i to j"); with dW/dr < 0 both forces then repel. */
  int64_t ipairs = 0, fpairs = 0;
#pragma omp parallel for schedule(static) reduction(+ : ipairs, fpairs)
  for (int64_t i = 0; i < n; ++i) {
    double ai[3] = {0, 0, 0}, sabs = 0.0;
    const int surf_i = p->surface && p->surface[i];
    for (int64_t t = S.fstart[i]; t < S.fstart[i + 1]; ++t) {
      int64_t j = S.flist[t];
      if (surf_i && !p->surface[j]) continue; /* Sec. 3.5: normal particles do not act on surface ones */
      double r = sqrt(dist2(pos + i * d, pos + j * d, d));
      double hij = 0.5 * (h[i] + h[j]);
      double dw = orc_dW(r, kappa * hij, d);
      double beta = (col[i] != col[j]) ? sigma : 0.0;
      double coef = (Pc[i] + Pc[j]) + beta * (P0 / (rt[i] * rt[i]) + P0 / (rt[j] * rt[j]));
      /* dW e_ij: at r = 0 (coincident particles) dW = 0 and e_ij is bounded, so the term is 0 */
      if (r > 0.0)
        for (int k = 0; k < d; ++k) ai[k] -= coef * dw * (pos[i * d + k] - pos[j * d + k]) / r;
      sabs += fabs(coef * dw);
      fpairs += 1;
      ipairs += (col[i] != col[j]);
    }
    if (surf_i) {
      double N[3];
      surface_normal(p, pos + i * d, N);
      tangential(N, ai, d);
    }
    for (int k = 0; k < d; ++k) a[i * d + k] = ai[k];
    if (pair_abs_a) pair_abs_a[i] = sabs;
  }
  I.interface_pairs = ipairs / 2;
  I.force_pairs = fpairs / 2;

  /* first time step: Eq. time_step_size with v_n = 0 leaves only the body-force term:
   * dt1 = min_i 0.25 sqrt(r_c,i / |a_i|), r_c,i = kappa h_i (global minimum).
   * Reading: if every a_i = 0 nothing moves (dt = 0). */
  double dt1 = INFINITY, mra = INFINITY, amax = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double an = 0.0;
    for (int k = 0; k < d; ++k) an += a[i * d + k] * a[i * d + k];
    an = sqrt(an);
    if (an > amax) amax = an;
    if (an > 0.0) {
      double rc = kappa * h[i];
      double t = 0.25 * sqrt(rc / an);
      if (t < dt1) dt1 = t;
      if (rc / an < mra) mra = rc / an;
    }
  }
  if (!(dt1 < INFINITY)) dt1 = 0.0;
  if (dt_fixed) dt1 = dt_fixed[0];  /* prescribed step sizes (frozen-step sensitivities) */
  /* Eq. time_int_01: v~ = v_n + a_n dt1 / 2 with v_n = 0 */
  for (size_t q = 0; q < nd; ++q) vt[q] = 0.5 * a[q] * dt1;

  /* second time step: Eq. time_step_size again with v~: the CFL term r_c/(40|v~|) and the
   * viscous term 0.125 r_c^2 / nu with nu = 0.1 r_c |v~| (Eq. viscosity_coefficient),
   * together with the body-force term of the first (reading: dt2 <= dt1). */
  double dt2 = dt1;
  for (int64_t i = 0; i < n; ++i) {
    double vn = 0.0;
    for (int k = 0; k < d; ++k) vn += vt[i * d + k] * vt[i * d + k];
    vn = sqrt(vn);
    double rc = kappa * h[i];
    double nu = 0.1 * rc * vn;
    eta[i] = rt[i] * nu; /* eta = rho nu with rho := rho_t (Eq. sph_viscous_force_2) */
    if (vn > 0.0) {
      double t1 = rc / (40.0 * vn);
      double t2 = 0.125 * rc * rc / nu;
      if (t1 < dt2) dt2 = t1;
      if (t2 < dt2) dt2 = t2;
    }
  }
  if (dt_fixed) dt2 = dt_fixed[1];

  /* viscous force: Eq. sph_viscous_force with rho := rho_t (Eq. sph_viscous_force_2):
   * a~_i = sum_j 2 eta_i eta_j/(eta_i + eta_j) (1/rho_t,i^2 + 1/rho_t,j^2)
   *        dW(r_ij, h_ij)/dr (v~_i - v~_j) / r_ij ;
   * reading: the harmonic mean is 0 when eta_i + eta_j = 0. */
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double s[3] = {0, 0, 0}, sabs = 0.0;
    const int surf_i = p->surface && p->surface[i];
    for (int64_t t = S.fstart[i]; t < S.fstart[i + 1]; ++t) {
      int64_t j = S.flist[t];
      if (surf_i && !p->surface[j]) continue;
      double r = sqrt(dist2(pos + i * d, pos + j * d, d));
      double hij = 0.5 * (h[i] + h[j]);
      double es = eta[i] + eta[j];
      double hm = es > 0.0 ? 2.0 * eta[i] * eta[j] / es : 0.0;
      double coef = hm * (1.0 / (rt[i] * rt[i]) + 1.0 / (rt[j] * rt[j])) * orc_dW_over_r(r, kappa * hij, d);
      double vi2 = 0.0, vj2 = 0.0;
      for (int k = 0; k < d; ++k) {
        double vij = vt[i * d + k] - vt[j * d + k];
        s[k] += coef * vij;
        vi2 += vt[i * d + k] * vt[i * d + k];
        vj2 += vt[j * d + k] * vt[j * d + k];
      }
      /* normaliser: magnitudes of the two velocity terms of the pair */
      sabs += fabs(coef) * (sqrt(vi2) + sqrt(vj2));
    }
    if (surf_i) {
      double N[3];
      surface_normal(p, pos + i * d, N);
      tangential(N, s, d);
    }
    for (int k = 0; k < d; ++k) at[i * d + k] = s[k];
    if (pair_abs_b) pair_abs_b[i] = sabs;
  }

  /* Eq. time_int_02 and time_int_03 with dt2, then the projection (Eq. displacement_surface). */
  int64_t moved = 0;
  for (int64_t i = 0; i < n; ++i) {
    for (int k = 0; k < d; ++k) {
      double v = vt[i * d + k] + 0.5 * at[i * d + k] * dt2;
      pos[i * d + k] += v * dt2;
    }
    if (p->surface && p->surface[i]) {
      /* the position stays in the bounding box (the state space), then goes
       * onto its surface */
      orc_shape box = box_shape(p);
      project_one(p, &box, pos + i * d, d);
      project_to_surface(p, pos + i * d);
    } else {
      moved += orc_project(p, pos + i * d);
    }
  }

  /* diagnostics */
  double srho = 0.0, el2 = 0.0, emax = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double e = rho[i] / rt[i] - 1.0;
    srho += rho[i]; el2 += e * e;
    if (fabs(e) > emax) emax = fabs(e);
  }
  I.dt1 = dt1; I.dt2 = dt2; I.min_rc_over_a = mra; I.max_a = amax;
  I.sum_rho = srho; I.err_l2 = el2; I.err_max = emax; I.wall_moved = moved;
  if (info) *info = I;
  if (rho_out) memcpy(rho_out, rho, sizeof(double) * (size_t)n);
  if (acc_out) memcpy(acc_out, a, sizeof(double) * nd);
  if (visc_out) memcpy(visc_out, at, sizeof(double) * nd);

  free_sets(&S);
  free(h); free(rt); free(rho); free(Pc); free(a); free(vt); free(at); free(eta);
  return 0;
}

int orc_step(const orc_problem* p, int64_t n, double* pos, const uint8_t* col, int64_t step,
             int mode, orc_step_info* info, double* rho_out, double* acc_out, double* visc_out,
             double* pair_abs_a, double* pair_abs_b) {
  return step_core(p, n, pos, col, step, mode, NULL, info, rho_out, acc_out, visc_out, pair_abs_a,
                   pair_abs_b);
}

int orc_step_fixed_dt(const orc_problem* p, int64_t n, double* pos, const uint8_t* col, int64_t step,
                      int mode, const double* dt, orc_step_info* info) {
  return step_core(p, n, pos, col, step, mode, dt, info, NULL, NULL, NULL, NULL, NULL);
}

/* ======================================================================== */
/* Sensitivities of a relaxation run (reverse mode, written by hand).        */
/*                                                                          */
/* The paper tunes nothing by gradient; this part differentiates the step of */
/* Algorithm 1 as the forward code above computes it, for the                */
/* objective                                                                 */
/*   L = sum_i (rho_i/rho_t,i - 1)^2 + lambda sum_{i<j, C_i != C_j} W(r_ij, kappa h_ij) */
/* after K steps, with respect to the initial positions, sigma0, gamma, P0    */
/* and the coefficients of the polynomial density factor (rho_scale fixed).  */
/* Two modes: the step sizes recomputed from the state (the min over         */
/* particles differentiated at its argmin), or prescribed ("frozen").        */
/* Pair sums are visited as unordered pairs and scattered to both ends.      */
/* ======================================================================== */

/* partial derivatives of the kernel functions (Wendland C2, support H):
 *   W = c_d H^-d f(q), f = (1-q)^4 (1+4q), f' = -20 q (1-q)^3, q = r/H
 *   dW/dH = -c_d H^-(d+1) (d f + q f')
 *   F = (dW/dr)/r = -20 c_d H^-(d+2) (1-q)^3
 *   dF/dr = 60 c_d H^-(d+3) (1-q)^2,  dF/dH = 20 c_d H^-(d+3) (1-q)^2 ((d+2)(1-q) - 3q) */
static double kernel_c(int dim) { return dim == 2 ? 7.0 / PI : 21.0 / (2.0 * PI); }

static double dW_dH(double r, double H, int dim) {
  double q = r / H;
  if (q >= 1.0) return 0.0;
  double u = 1.0 - q, f = u * u * u * u * (1.0 + 4.0 * q), fp = -20.0 * q * u * u * u;
  return -kernel_c(dim) * pow(H, -(double)(dim + 1)) * (dim * f + q * fp);
}

static void force_kernel(double r, double H, int dim, double* F, double* F_r, double* F_H) {
  double q = r / H;
  *F = *F_r = *F_H = 0.0;
  if (q >= 1.0) return;
  double u = 1.0 - q, c = kernel_c(dim);
  double Hm = pow(H, -(double)(dim + 3));
  *F = -20.0 * c * Hm * H * u * u * u;
  *F_r = 60.0 * c * Hm * u * u;
  *F_H = 20.0 * c * Hm * u * u * ((dim + 2) * u - 3.0 * q);
}

/* gradient of the signed inside distance of a shape (the branch the value takes) */
static void inside_distance_grad(const orc_problem* p, const orc_shape* s, const double* x, int dim, double* g) {
  for (int k = 0; k < 3; ++k) g[k] = 0.0;
  if (s->kind == ORC_GRID) {
    bg_interp(p, p->bg_phi, x, g);
    return;
  }
  if (s->kind == ORC_SPHERE) {
    double r2 = 0.0;
    for (int k = 0; k < dim; ++k) r2 += (x[k] - s->center[k]) * (x[k] - s->center[k]);
    double r = sqrt(r2);
    if (r > 0.0)
      for (int k = 0; k < dim; ++k) g[k] = -(x[k] - s->center[k]) / r;
    return;
  }
  double outside2 = 0.0, qmax = -INFINITY, q[3] = {0, 0, 0};
  int kmax = 0;
  for (int k = 0; k < dim; ++k) {
    q[k] = fabs(x[k] - s->center[k]) - s->size[k];
    if (q[k] > 0) outside2 += q[k] * q[k];
    if (q[k] > qmax) { qmax = q[k]; kmax = k; }
  }
  if (outside2 > 0.0) {
    double o = sqrt(outside2);
    for (int k = 0; k < dim; ++k)
      if (q[k] > 0) g[k] = -q[k] * (x[k] >= s->center[k] ? 1.0 : -1.0) / o;
  } else if (qmax < 0) {
    g[kmax] = -(x[kmax] >= s->center[kmax] ? 1.0 : -1.0);
  }
}

/* the polynomial basis b_m(x~) of the density factor and d b_m / d x_k */
static void poly_basis(const orc_problem* p, const double* x, double* b, double db[8][3]) {
  double t[3] = {0, 0, 0}, dt[3] = {0, 0, 0};
  for (int k = 0; k < p->dim; ++k) {
    t[k] = 2.0 * (x[k] - p->lo[k]) / (p->hi[k] - p->lo[k]) - 1.0;
    dt[k] = 2.0 / (p->hi[k] - p->lo[k]);
  }
  memset(db, 0, sizeof(double) * 24);
  if (p->dim == 2) {
    double X = t[0], Y = t[1];
    b[0] = X; b[1] = Y; b[2] = X * X; b[3] = X * Y; b[4] = Y * Y;
    b[5] = X * X * X; b[6] = X * X * Y; b[7] = X * Y * Y;
    double dX[8] = {1, 0, 2 * X, Y, 0, 3 * X * X, 2 * X * Y, Y * Y};
    double dY[8] = {0, 1, 0, X, 2 * Y, 0, X * X, 2 * X * Y};
    for (int m = 0; m < 8; ++m) { db[m][0] = dX[m] * dt[0]; db[m][1] = dY[m] * dt[1]; }
  } else {
    double X = t[0], Y = t[1], Z = t[2];
    b[0] = X; b[1] = Y; b[2] = Z; b[3] = X * X; b[4] = Y * Y; b[5] = Z * Z;
    b[6] = X * Y; b[7] = Y * Z;
    double dX[8] = {1, 0, 0, 2 * X, 0, 0, Y, 0};
    double dY[8] = {0, 1, 0, 0, 2 * Y, 0, X, Z};
    double dZ[8] = {0, 0, 1, 0, 0, 2 * Z, 0, Y};
    for (int m = 0; m < 8; ++m) { db[m][0] = dX[m] * dt[0]; db[m][1] = dY[m] * dt[1]; db[m][2] = dZ[m] * dt[2]; }
  }
}

/* rho_t = rho_scale s^-d P(x): its gradient in x and its derivatives in the
 * polynomial coefficients */
static double rho_t_grad(const orc_problem* p, const double* x, double* grad, double* dcoef) {
  int d = p->dim;
  double s = spacing(p, x), Pf = poly_factor(p, x);
  double base = p->rho_scale * pow(s, -(double)d);
  double rt = base * Pf;
  double gs[3] = {0, 0, 0};
  if (p->field_kind == ORC_FIELD_BACKGROUND) {
    bg_interp(p, p->bg_s, x, gs);
  } else if (p->field_kind != ORC_FIELD_UNIFORM) {
    const orc_shape* sh = &p->shapes[p->dist_shape];
    double dist = shape_inside_distance(p, sh, x, d), gd[3];
    inside_distance_grad(p, sh, x, d, gd);
    double sg = dist >= 0.0 ? 1.0 : -1.0;
    double slope = spacing_slope(p, dist);
    for (int k = 0; k < d; ++k) gs[k] = slope * sg * gd[k];
  }
  double b[8], db[8][3], gP[3] = {0, 0, 0};
  for (int m = 0; m < 8; ++m) dcoef[m] = 0.0;
  if (p->n_poly > 0) {
    poly_basis(p, x, b, db);
    for (int m = 0; m < p->n_poly && m < 8; ++m) {
      dcoef[m] = base * b[m];
      for (int k = 0; k < d; ++k) gP[k] += p->poly[m] * db[m][k];
    }
  }
  for (int k = 0; k < 3; ++k) grad[k] = 0.0;
  for (int k = 0; k < d; ++k) grad[k] = rt * (-(double)d * gs[k] / s) + base * gP[k];
  return rt;
}

/* vector-Jacobian product of orc_project at y: g holds the adjoint of the
 * projected point on entry and that of y on return. The constraints act in
 * order (box first); each violated one is a map whose Jacobian is taken at the
 * point it received. */
static void project_vjp(const orc_problem* p, const double* y, double* g) {
  int d = p->dim;
  orc_shape cons[5];
  int nc = 0;
  cons[nc++] = box_shape(p);
  for (int s = 0; s < p->n_shapes; ++s) cons[nc++] = p->shapes[s];
  double z[6][3];
  for (int k = 0; k < 3; ++k) z[0][k] = k < d ? y[k] : 0.0;
  for (int c = 0; c < nc; ++c) {
    memcpy(z[c + 1], z[c], sizeof z[c]);
    project_one(p, &cons[c], z[c + 1], d);
  }
  for (int c = nc - 1; c >= 0; --c) {
    const orc_shape* s = &cons[c];
    const double* x = z[c];
    if (!(constraint_phi(p, s, x, d) < 0.0)) continue;
    if (s->kind == ORC_SPHERE) {
      double dv[3] = {0, 0, 0}, r2 = 0.0;
      for (int k = 0; k < d; ++k) { dv[k] = x[k] - s->center[k]; r2 += dv[k] * dv[k]; }
      double r = sqrt(r2);
      if (r == 0.0) { for (int k = 0; k < d; ++k) g[k] = 0.0; continue; }
      double ng = 0.0;
      for (int k = 0; k < d; ++k) ng += dv[k] / r * g[k];
      for (int k = 0; k < d; ++k) g[k] = s->size[0] / r * (g[k] - dv[k] / r * ng);
    } else if (s->keep_inside) {
      for (int k = 0; k < d; ++k) {
        double lo = s->center[k] - s->size[k], hi = s->center[k] + s->size[k];
        if (x[k] < lo || x[k] > hi) g[k] = 0.0;
      }
    } else {
      int best = 0; double bestd = INFINITY;
      for (int k = 0; k < d; ++k) {
        double dlo = x[k] - (s->center[k] - s->size[k]);
        double dhi = (s->center[k] + s->size[k]) - x[k];
        if (dlo < bestd) { bestd = dlo; best = k; }
        if (dhi < bestd) { bestd = dhi; best = k; }
      }
      g[best] = 0.0;
    }
  }
}

/* adjoints of the per-particle target quantities -> positions and coefficients:
 * rtb (rho_t), hb (h = tau rho_t^-1/d) and Tb (T = 1/rho_t^2) at particle i */
static void local_field_vjp(const orc_problem* p, const double* x, double rtb, double hb, double Tb,
                            double* xb, double* dpoly) {
  double grad[3], dc[8];
  double rt = rho_t_grad(p, x, grad, dc);
  double h = p->tau * pow(1.0 / rt, 1.0 / p->dim);
  double T = 1.0 / (rt * rt);
  double tot = rtb + hb * (-h / (p->dim * rt)) + Tb * (-2.0 * T / rt);
  for (int k = 0; k < p->dim; ++k) xb[k] += tot * grad[k];
  for (int m = 0; m < 8; ++m) dpoly[m] += tot * dc[m];
}

typedef struct {
  double sigma0, gamma, P0, poly[8];
} param_bar;

/* density reverse: rho_i = sum_{j in D_i} W(r_ij, kappa h_i); adds to xb and hb */
static void density_vjp(const orc_problem* p, int64_t n, const double* pos, const double* h,
                        const nbr_sets* S, const double* rhob, double* xb, double* hb) {
  int d = p->dim;
  for (int64_t i = 0; i < n; ++i) {
    if (rhob[i] == 0.0) continue;
    double H = p->kappa * h[i];
    for (int64_t t = S->dstart[i]; t < S->dstart[i + 1]; ++t) {
      int64_t j = S->dlist[t];
      double r = sqrt(dist2(pos + i * d, pos + j * d, d));
      hb[i] += rhob[i] * dW_dH(r, H, d) * p->kappa;
      if (j == i || r == 0.0) continue;
      double c = rhob[i] * orc_dW(r, H, d) / r;
      for (int k = 0; k < d; ++k) {
        double e = pos[i * d + k] - pos[j * d + k];
        xb[i * d + k] += c * e;
        xb[j * d + k] -= c * e;
      }
    }
  }
}

static double ramp_of(const orc_problem* p, int64_t step) {
  orc_problem q = *p;
  q.sigma0 = 1.0;
  return orc_sigma(&q, (double)step);
}

/* One step in reverse. pos is the state the step starts from; g holds the
 * adjoint of the state it produced on entry and that of pos on return. */
static int step_vjp(const orc_problem* p, int64_t n, const double* pos, const uint8_t* col,
                    int64_t step, const double* dt_fixed, double* g, param_bar* pb) {
  const int d = p->dim;
  const double kappa = p->kappa, P0 = p->P0, gamma = p->gamma;
  const double sigma = orc_sigma(p, (double)step);
  const int dens_free = (gamma == 2.0 && !p->eos_general);
  size_t nd = (size_t)n * (size_t)d;
  double *h = calloc(n, 8), *rt = calloc(n, 8), *T = calloc(n, 8), *rho = calloc(n, 8), *Q = calloc(n, 8);
  double *a = calloc(nd, 8), *vt = calloc(nd, 8), *at = calloc(nd, 8), *eta = calloc(n, 8), *y = calloc(nd, 8);
  double *xb = calloc(nd, 8), *ab = calloc(nd, 8), *vtb = calloc(nd, 8), *atb = calloc(nd, 8);
  double *hb = calloc(n, 8), *rtb = calloc(n, 8), *Tb = calloc(n, 8), *Qb = calloc(n, 8), *etab = calloc(n, 8),
         *rhob = calloc(n, 8);
  if (!h || !rt || !T || !rho || !Q || !a || !vt || !at || !eta || !y || !xb || !ab || !vtb || !atb || !hb ||
      !rtb || !Tb || !Qb || !etab || !rhob)
    return -1;
  /* forward quantities of this step (as step_core computes them) */
  for (int64_t i = 0; i < n; ++i) {
    rt[i] = orc_rho_t(p, pos + i * d);
    h[i] = p->tau * pow(1.0 / rt[i], 1.0 / d);
    T[i] = 1.0 / (rt[i] * rt[i]);
  }
  nbr_sets S; memset(&S, 0, sizeof S);
  if (build_sets(p, n, pos, h, 1, &S) != 0) return -1;
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t t = S.dstart[i]; t < S.dstart[i + 1]; ++t) {
      int64_t j = S.dlist[t];
      s += orc_W(sqrt(dist2(pos + i * d, pos + j * d, d)), kappa * h[i], d);
    }
    rho[i] = s;
    Q[i] = dens_free ? P0 * T[i] : P0 * pow(rho[i] / rt[i], gamma) / (rho[i] * rho[i]);
  }
  for (int64_t i = 0; i < n; ++i)
    for (int64_t t = S.fstart[i]; t < S.fstart[i + 1]; ++t) {
      int64_t j = S.flist[t];
      double r = sqrt(dist2(pos + i * d, pos + j * d, d));
      double F, Fr, FH;
      force_kernel(r, kappa * 0.5 * (h[i] + h[j]), d, &F, &Fr, &FH);
      double beta = (col[i] != col[j]) ? sigma : 0.0;
      double coef = Q[i] + Q[j] + beta * P0 * (T[i] + T[j]);
      for (int k = 0; k < d; ++k) a[i * d + k] -= coef * F * (pos[i * d + k] - pos[j * d + k]);
    }
  double mmin = INFINITY; int64_t kmin = -1;
  for (int64_t i = 0; i < n; ++i) {
    double an = 0.0;
    for (int k = 0; k < d; ++k) an += a[i * d + k] * a[i * d + k];
    an = sqrt(an);
    if (an > 0.0 && kappa * h[i] / an < mmin) { mmin = kappa * h[i] / an; kmin = i; }
  }
  double dt1 = kmin >= 0 ? 0.25 * sqrt(mmin) : 0.0, dt2;
  if (dt_fixed) dt1 = dt_fixed[0];
  for (size_t q = 0; q < nd; ++q) vt[q] = 0.5 * a[q] * dt1;
  dt2 = dt1;
  for (int64_t i = 0; i < n; ++i) {
    double vn = 0.0;
    for (int k = 0; k < d; ++k) vn += vt[i * d + k] * vt[i * d + k];
    vn = sqrt(vn);
    double rc = kappa * h[i], nu = 0.1 * rc * vn;
    eta[i] = rt[i] * nu;
    if (vn > 0.0) {
      if (rc / (40.0 * vn) < dt2) dt2 = rc / (40.0 * vn);
      if (0.125 * rc * rc / nu < dt2) dt2 = 0.125 * rc * rc / nu;
    }
  }
  if (dt_fixed) dt2 = dt_fixed[1];
  for (int64_t i = 0; i < n; ++i)
    for (int64_t t = S.fstart[i]; t < S.fstart[i + 1]; ++t) {
      int64_t j = S.flist[t];
      double r = sqrt(dist2(pos + i * d, pos + j * d, d));
      double F, Fr, FH;
      force_kernel(r, kappa * 0.5 * (h[i] + h[j]), d, &F, &Fr, &FH);
      double es = eta[i] + eta[j], hm = es > 0.0 ? 2.0 * eta[i] * eta[j] / es : 0.0;
      double K = hm * (T[i] + T[j]) * F;
      for (int k = 0; k < d; ++k) at[i * d + k] += K * (vt[i * d + k] - vt[j * d + k]);
    }
  for (size_t q = 0; q < nd; ++q) y[q] = pos[q] + dt2 * (vt[q] + 0.5 * dt2 * at[q]);

  /* reverse: projection, drift and kicks (Eqs. time_int_01..03) */
  double dt1b = 0.0, dt2b = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double gi[3] = {0, 0, 0};
    for (int k = 0; k < d; ++k) gi[k] = g[i * d + k];
    project_vjp(p, y + i * d, gi);
    for (int k = 0; k < d; ++k) {
      size_t q = (size_t)i * d + k;
      xb[q] += gi[k];
      vtb[q] += dt2 * gi[k];
      atb[q] += 0.5 * dt2 * dt2 * gi[k];
      dt2b += gi[k] * (vt[q] + dt2 * at[q]);
    }
  }
  /* viscous pairs: a~_i = sum_j K_ij (v~_i - v~_j), K = hm (T_i + T_j) F */
  for (int64_t i = 0; i < n; ++i)
    for (int64_t t = S.fstart[i]; t < S.fstart[i + 1]; ++t) {
      int64_t j = S.flist[t];
      if (j < i) continue;
      double e[3] = {0, 0, 0};
      for (int k = 0; k < d; ++k) e[k] = pos[i * d + k] - pos[j * d + k];
      double r = sqrt(dist2(pos + i * d, pos + j * d, d));
      double F, Fr, FH;
      force_kernel(r, kappa * 0.5 * (h[i] + h[j]), d, &F, &Fr, &FH);
      double es = eta[i] + eta[j], hm = es > 0.0 ? 2.0 * eta[i] * eta[j] / es : 0.0;
      double dhi = es > 0.0 ? 2.0 * eta[j] * eta[j] / (es * es) : 0.0;
      double dhj = es > 0.0 ? 2.0 * eta[i] * eta[i] / (es * es) : 0.0;
      double Ts = T[i] + T[j], K = hm * Ts * F, Kb = 0.0;
      for (int k = 0; k < d; ++k) {
        double dab = atb[i * d + k] - atb[j * d + k];
        vtb[i * d + k] += K * dab;
        vtb[j * d + k] -= K * dab;
        Kb += dab * (vt[i * d + k] - vt[j * d + k]);
      }
      etab[i] += Kb * Ts * F * dhi;
      etab[j] += Kb * Ts * F * dhj;
      Tb[i] += Kb * hm * F;
      Tb[j] += Kb * hm * F;
      double Fb = Kb * hm * Ts;
      for (int k = 0; k < d; ++k) {
        xb[i * d + k] += Fb * Fr * e[k] / r;
        xb[j * d + k] -= Fb * Fr * e[k] / r;
      }
      hb[i] += Fb * FH * 0.5 * kappa;
      hb[j] += Fb * FH * 0.5 * kappa;
    }
  /* eta_i = rho_t,i 0.1 kappa h_i |v~_i|; v~ = a dt1/2 */
  for (int64_t i = 0; i < n; ++i) {
    double vn = 0.0;
    for (int k = 0; k < d; ++k) vn += vt[i * d + k] * vt[i * d + k];
    vn = sqrt(vn);
    if (vn > 0.0) {
      rtb[i] += etab[i] * 0.1 * kappa * h[i] * vn;
      hb[i] += etab[i] * 0.1 * rt[i] * kappa * vn;
      for (int k = 0; k < d; ++k) vtb[i * d + k] += etab[i] * 0.1 * rt[i] * kappa * h[i] * vt[i * d + k] / vn;
    }
    for (int k = 0; k < d; ++k) {
      ab[i * d + k] += 0.5 * dt1 * vtb[i * d + k];
      dt1b += 0.5 * a[i * d + k] * vtb[i * d + k];
    }
  }
  /* recomputed step sizes: dt1 = 0.25 sqrt(m), dt2 = 0.2 sqrt(m) (both minima
   * sit at the argmin of m = r_c,k/|a_k|) */
  if (!dt_fixed && kmin >= 0) {
    double mb = dt1b * 0.125 / sqrt(mmin) + dt2b * 0.1 / sqrt(mmin);
    double an = 0.0;
    for (int k = 0; k < d; ++k) an += a[kmin * d + k] * a[kmin * d + k];
    an = sqrt(an);
    hb[kmin] += mb * kappa / an;
    for (int k = 0; k < d; ++k) ab[kmin * d + k] -= mb * kappa * h[kmin] * a[kmin * d + k] / (an * an * an);
  }
  /* pressure and surface-tension pairs: a_i = sum_j S_ij (x_i - x_j), S = -coef F */
  double sigb = 0.0;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t t = S.fstart[i]; t < S.fstart[i + 1]; ++t) {
      int64_t j = S.flist[t];
      if (j < i) continue;
      double e[3] = {0, 0, 0};
      for (int k = 0; k < d; ++k) e[k] = pos[i * d + k] - pos[j * d + k];
      double r = sqrt(dist2(pos + i * d, pos + j * d, d));
      double F, Fr, FH;
      force_kernel(r, kappa * 0.5 * (h[i] + h[j]), d, &F, &Fr, &FH);
      int other = col[i] != col[j];
      double beta = other ? sigma : 0.0;
      double coef = Q[i] + Q[j] + beta * P0 * (T[i] + T[j]);
      double Sij = -coef * F, Sb = 0.0;
      for (int k = 0; k < d; ++k) {
        double dab = ab[i * d + k] - ab[j * d + k];
        xb[i * d + k] += Sij * dab;
        xb[j * d + k] -= Sij * dab;
        Sb += dab * e[k];
      }
      double cb = -Sb * F;
      Qb[i] += cb; Qb[j] += cb;
      Tb[i] += cb * beta * P0; Tb[j] += cb * beta * P0;
      if (other) sigb += cb * P0 * (T[i] + T[j]);
      pb->P0 += cb * beta * (T[i] + T[j]);
      double Fb = -Sb * coef;
      for (int k = 0; k < d; ++k) {
        xb[i * d + k] += Fb * Fr * e[k] / r;
        xb[j * d + k] -= Fb * Fr * e[k] / r;
      }
      hb[i] += Fb * FH * 0.5 * kappa;
      hb[j] += Fb * FH * 0.5 * kappa;
    }
  pb->sigma0 += sigb * ramp_of(p, step);
  /* equation of state: Q = p/rho^2 = P0 (rho/rho_t)^gamma / rho^2 (P0 T at gamma = 2) */
  for (int64_t i = 0; i < n; ++i) {
    double lr = log(rho[i] / rt[i]);
    pb->gamma += Qb[i] * Q[i] * lr;
    if (dens_free) {
      Tb[i] += Qb[i] * P0;
      pb->P0 += Qb[i] * T[i];
    } else {
      rhob[i] += Qb[i] * (gamma - 2.0) * Q[i] / rho[i];
      rtb[i] += -gamma * Qb[i] * Q[i] / rt[i];
      pb->P0 += Qb[i] * pow(rho[i] / rt[i], gamma) / (rho[i] * rho[i]);
    }
  }
  density_vjp(p, n, pos, h, &S, rhob, xb, hb);
  for (int64_t i = 0; i < n; ++i) local_field_vjp(p, pos + i * d, rtb[i], hb[i], Tb[i], xb + i * d, pb->poly);
  memcpy(g, xb, sizeof(double) * nd);
  free_sets(&S);
  free(h); free(rt); free(T); free(rho); free(Q); free(a); free(vt); free(at); free(eta); free(y);
  free(xb); free(ab); free(vtb); free(atb); free(hb); free(rtb); free(Tb); free(Qb); free(etab); free(rhob);
  return 0;
}

/* objective at pos; with g non-NULL also adds dL/dpos to g and dL/dcoef to dpoly */
static int objective_core(const orc_problem* p, int64_t n, const double* pos, const uint8_t* col,
                          double lambda, double* L, double* g, double* dpoly) {
  const int d = p->dim;
  const double kappa = p->kappa;
  double *h = calloc(n, 8), *rt = calloc(n, 8), *rhob = calloc(n, 8), *hb = calloc(n, 8), *rtb = calloc(n, 8);
  if (!h || !rt || !rhob || !hb || !rtb) return -1;
  for (int64_t i = 0; i < n; ++i) {
    rt[i] = orc_rho_t(p, pos + i * d);
    h[i] = p->tau * pow(1.0 / rt[i], 1.0 / d);
  }
  nbr_sets S; memset(&S, 0, sizeof S);
  if (build_sets(p, n, pos, h, 1, &S) != 0) return -1;
  double Ld = 0.0, Li = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double rho = 0.0;
    for (int64_t t = S.dstart[i]; t < S.dstart[i + 1]; ++t)
      rho += orc_W(sqrt(dist2(pos + i * d, pos + S.dlist[t] * d, d)), kappa * h[i], d);
    double e = rho / rt[i] - 1.0;
    Ld += e * e;
    rhob[i] = 2.0 * e / rt[i];
    rtb[i] = -2.0 * e * rho / (rt[i] * rt[i]);
  }
  for (int64_t i = 0; i < n; ++i)
    for (int64_t t = S.fstart[i]; t < S.fstart[i + 1]; ++t) {
      int64_t j = S.flist[t];
      if (j < i || col[i] == col[j]) continue;
      double r = sqrt(dist2(pos + i * d, pos + j * d, d));
      double H = kappa * 0.5 * (h[i] + h[j]);
      Li += orc_W(r, H, d);
      if (!g) continue;
      double c = lambda * orc_dW(r, H, d) / r;
      for (int k = 0; k < d; ++k) {
        double e = pos[i * d + k] - pos[j * d + k];
        g[i * d + k] += c * e;
        g[j * d + k] -= c * e;
      }
      double wh = lambda * dW_dH(r, H, d) * 0.5 * kappa;
      hb[i] += wh; hb[j] += wh;
    }
  *L = Ld + lambda * Li;
  if (g) {
    density_vjp(p, n, pos, h, &S, rhob, g, hb);
    for (int64_t i = 0; i < n; ++i) local_field_vjp(p, pos + i * d, rtb[i], hb[i], 0.0, g + i * d, dpoly);
  }
  free_sets(&S);
  free(h); free(rt); free(rhob); free(hb); free(rtb);
  return 0;
}

int orc_objective(const orc_problem* p, int64_t n, const double* pos, const uint8_t* col, double lambda,
                  double* L) {
  return objective_core(p, n, pos, col, lambda, L, NULL, NULL);
}

int orc_backward(const orc_problem* p, int64_t n, const double* pos0, const uint8_t* col, int64_t step0,
                 int32_t K, const double* dt_in, double* dt_out, double lambda, const double* seed,
                 double* L, double* dpos0, double* grads) {
  const int d = p->dim;
  /* the reverse pass covers analytic shapes only (no background-mesh level set) */
  for (int s = 0; s < p->n_shapes; ++s)
    if (p->shapes[s].kind == ORC_GRID) return -1;
  if (p->surface) return -1; /* nor feature-surface particles */
  size_t nd = (size_t)n * (size_t)d;
  double* traj = (double*)malloc(sizeof(double) * nd * (size_t)(K + 1));
  if (!traj) return -1;
  memcpy(traj, pos0, sizeof(double) * nd);
  for (int32_t s = 0; s < K; ++s) {
    double* x = traj + nd * (size_t)(s + 1);
    memcpy(x, traj + nd * (size_t)s, sizeof(double) * nd);
    orc_step_info info;
    if (step_core(p, n, x, col, step0 + s, 1, dt_in ? dt_in + 2 * s : NULL, &info, NULL, NULL, NULL, NULL,
                  NULL) != 0) { free(traj); return -1; }
    if (dt_out) { dt_out[2 * s] = info.dt1; dt_out[2 * s + 1] = info.dt2; }
  }
  param_bar pb; memset(&pb, 0, sizeof pb);
  memset(dpos0, 0, sizeof(double) * nd);
  if (objective_core(p, n, traj + nd * (size_t)K, col, lambda, L, dpos0, pb.poly) != 0) { free(traj); return -1; }
  if (seed)
    for (size_t q = 0; q < nd; ++q) dpos0[q] += seed[q];
  for (int32_t s = K - 1; s >= 0; --s)
    if (step_vjp(p, n, traj + nd * (size_t)s, col, step0 + s, dt_in ? dt_in + 2 * s : NULL, dpos0, &pb) != 0) {
      free(traj); return -1;
    }
  grads[0] = pb.sigma0; grads[1] = pb.gamma; grads[2] = pb.P0;
  for (int m = 0; m < 8; ++m) grads[3 + m] = pb.poly[m];
  free(traj);
  return 0;
}
