/*
 * FP64 CPU oracle of the multi-phase SPH relaxation step of
 * "A Consistent Parallel Isotropic Unstructured Mesh Generation Method based on
 * Multi-phase SPH" (arXiv 1906.07925).
 *
 * TEST INFRASTRUCTURE ONLY. This is the plain, slow reference the CUDA path is
 * checked against. Only the tests, the smoke check and the CPU-baseline leg of
 * the bench may load it. It shares no code, header or constant table with the
 * CUDA library: every formula here is written out from the paper.
 *
 * Conventions
 *  - positions are row-major (n x dim) doubles; colours are uint8;
 *  - unit particle mass (Eq. mass_SPH_particle);
 *  - h_i = tau * (1/rho_t,i)^(1/d) (Eq. scale_SPH_particle), support H = kappa*h;
 *  - every per-particle sum runs over neighbours in ascending particle index.
 */
#ifndef SPH_ORACLE_H
#define SPH_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_SPHERE 0
#define ORC_BOX 1
#define ORC_GRID 2  /* the level set sampled on the background mesh (bg_phi) */
#define ORC_FIELD_UNIFORM 0
#define ORC_FIELD_LINEAR_DISTANCE 1
#define ORC_FIELD_TANH_DISTANCE 2  /* s = a + b tanh(s0 |dist|): the circle case of Sec. 4.1 */
#define ORC_FIELD_BACKGROUND 3     /* s sampled on the background mesh (bg_s) */

typedef struct {
  int32_t kind;        /* ORC_SPHERE or ORC_BOX */
  int32_t keep_inside; /* 1: the mesh region is inside the shape */
  double center[3];
  double size[3];      /* sphere: size[0] = radius; box: half extents */
} orc_shape;

typedef struct {
  int32_t dim;
  int32_t n_shapes;
  double lo[3], hi[3];
  orc_shape shapes[4];
  int32_t field_kind;
  int32_t dist_shape;
  double s0, a, b;
  int32_t n_poly;
  int32_t eos_general;  /* 1: use p/rho^2 even at gamma = 2 (for the gamma = 2 identity check) */
  double poly[8];
  double rho_scale;
  double P0, gamma, sigma0, tau, kappa;
  double t0, t1;       /* surface-tension ramp window in steps; t0 < 0: none */
  /* Cartesian background mesh (Sec. 3.1, 3.2): node values at
   * bg_lo + i (bg_hi - bg_lo) / (bg_dims - 1), x fastest; bg_dims[2] = 1 in 2D.
   * bg_phi: level set (positive in the region) for ORC_GRID shapes; bg_s:
   * target spacing for ORC_FIELD_BACKGROUND. NULL when unused. */
  int32_t bg_dims[3];
  int32_t bg_pad;
  double bg_lo[3], bg_hi[3];
  const double* bg_phi;
  const double* bg_s;
  /* feature-surface particles (Sec. 3.5): surface[i] != 0 marks particle i
   * (index order of the positions passed to a step); NULL: none */
  const uint8_t* surface;
} orc_problem;

typedef struct {
  double sigma;            /* surface-tension coefficient used in this step */
  double dt1, dt2;         /* first and second time-step sizes */
  double min_rc_over_a;    /* min_i r_c,i / |a_i| (inf if all a = 0) */
  double max_a;            /* max_i |a_i| */
  double sum_rho;          /* sum_i rho_i */
  double err_l2;           /* sum_i (rho_i/rho_t,i - 1)^2 */
  double err_max;          /* max_i |rho_i/rho_t,i - 1| */
  int64_t interface_pairs; /* unordered force pairs with distinct colours */
  int64_t force_pairs;     /* unordered force pairs */
  int64_t wall_moved;      /* particles moved by the level-set projection */
} orc_step_info;

/* Wendland C2 kernel and its radial derivative, support H (reading of the
 * unspecified "smooth isotropic kernel"). */
double orc_W(double r, double H, int dim);
double orc_dW(double r, double H, int dim);
/* (dW/dr)/r, continued at r = 0 by its limit -20 alpha_d / H^2 (coincident
 * particles); the factor of the viscous pair term (Eq. sph_viscous_force). */
double orc_dW_over_r(double r, double H, int dim);

/* Level set (positive in the mesh region, Sec. 3.1) and the projection of
 * Eq. displacement_surface, applied to each violated constraint in order. */
double orc_phi(const orc_problem* p, const double* x);
int orc_project(const orc_problem* p, double* x);

/* Target fields at x (Sec. 2.3 / 3.2). */
double orc_rho_t(const orc_problem* p, const double* x);
double orc_h(const orc_problem* p, const double* x);

/* Surface-tension coefficient at step t (Eq. sph_st_sigma). */
double orc_sigma(const orc_problem* p, double t);

/* M_v = integral of rho_t over the positive phase (Eq. total_mass_2), midpoint
 * rule with res cells per axis. */
double orc_total_mass(const orc_problem* p, int res);

/* Neighbour sets. mode 0: brute force O(n^2); mode 1: uniform grid.
 * Per particle: density-set size (r_ij < kappa h_i, self included), force-set
 * size (j != i, r_ij < kappa h_ij), and the sums / xors of the member indices. */
int orc_neighbor_sets(const orc_problem* p, int64_t n, const double* pos, int mode,
                      int32_t* dens_count, int32_t* force_count,
                      int64_t* dens_idsum, int64_t* force_idsum,
                      int64_t* dens_idxor, int64_t* force_idxor);

/* Multi-resolution cell grid of the neighbour search (Algorithm 1 builds a
 * neighbour list every step; this is the cell structure it is built from):
 * level l has cells of edge cell[l] = cell[0] 2^l and dims[l] cells per axis
 * from lo; keys of level l start at base[l] (base[n_levels] = total cells). */
typedef struct {
  int32_t n_levels;
  int32_t dim;
  double lo[3];
  double h0;          /* a particle with h < 2 h0 lives at level 0 */
  double cell[8];
  int32_t dims[8][3];
  uint32_t base[9];
} orc_grid;

/* Cell key of every particle: level l = floor(log2(h_i/h0)) clamped to
 * [0, n_levels - 1], cell coordinates c_k = floor((x_k - lo_k)/cell[l]) clamped
 * to [0, dims[l][k] - 1], key = base[l] + c_x + dims_x (c_y + dims_y c_z).
 * h_out (n, may be NULL) receives h_i. Returns 0. */
int orc_cell_keys(const orc_problem* p, int64_t n, const double* pos, const orc_grid* g, uint32_t* keys,
                  double* h_out);

/* One relaxation step (Algorithm 1) advancing pos in place.
 * Any of the per-particle outputs may be NULL:
 *   rho (n), acc (n*dim) = a_n, visc (n*dim) = a~, pair_abs_a (n) = sum_j of
 *   |pair term| of a_i, pair_abs_b (n) = sum_j |coefficient of a~ pair term| *
 *   (|v~_i| + |v~_j|) (normalisers of the parity tolerance). Returns 0 on success. */
int orc_step(const orc_problem* p, int64_t n, double* pos, const uint8_t* col, int64_t step,
             int mode, orc_step_info* info, double* rho, double* acc, double* visc,
             double* pair_abs_a, double* pair_abs_b);

/* orc_step with prescribed step sizes dt = {dt1, dt2} instead of the ones
 * Eq. time_step_size gives (for finite-difference checks of frozen-step
 * sensitivities). */
int orc_step_fixed_dt(const orc_problem* p, int64_t n, double* pos, const uint8_t* col, int64_t step,
                      int mode, const double* dt, orc_step_info* info);

/* Objective of the sensitivity runs (not in the paper): the density error and
 * an interface energy,
 *   L = sum_i (rho_i/rho_t,i - 1)^2 + lambda sum_{i<j, C_i != C_j} W(r_ij, kappa h_ij). */
int orc_objective(const orc_problem* p, int64_t n, const double* pos, const uint8_t* col, double lambda,
                  double* L);

/* K steps from pos0 (step counter step0), then L at the end state, then the
 * hand-written reverse pass. dt_in (2K: dt1, dt2 per step) prescribes the step
 * sizes ("frozen"); NULL recomputes them from the state and differentiates
 * that choice too. dt_out (2K, may be NULL) receives the sizes used. seed
 * (n*dim, may be NULL) is added to dL/dx_K. Outputs: L, dpos0 = dL/dx_0
 * (n*dim), grads = {dL/dsigma0, dL/dgamma, dL/dP0, dL/dpoly[0..7]} (11), with
 * rho_scale held fixed. */
int orc_backward(const orc_problem* p, int64_t n, const double* pos0, const uint8_t* col, int64_t step0,
                 int32_t K, const double* dt_in, double* dt_out, double lambda, const double* seed,
                 double* L, double* dpos0, double* grads);

/* Number of OpenMP threads the oracle uses. */
int orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
