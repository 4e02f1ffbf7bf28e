/*
 * sphmesh — GB300 (sm_103a) multi-phase SPH particle relaxation.
 *
 * C ABI of the relaxation step of "A Consistent Parallel Isotropic Unstructured
 * Mesh Generation Method based on Multi-phase SPH" (Ji, Fu, Hu, Adams,
 * arXiv 1906.07925): coloured particles relax toward a target density field;
 * the pressure force of a tailored EOS regularises the point distribution and an
 * inter-colour surface-tension force keeps the colours (sub-domains) compact.
 *
 * Every call here runs on the GPU through hand-written CUDA kernels; there is
 * no CPU fallback. Plain pointers and sizes only.
 *
 * Ownership. A handle owns its device buffers. They are obtained at creation
 * through the caller's allocator (sph_alloc; NULL: cudaMallocAsync on the
 * given stream) and returned through it in sph_destroy. Device work is issued
 * on the stream given at creation. No global state: handles are independent,
 * but one handle must not be used from two threads at once.
 *
 * Errors. Every call returns sph_status. Device-side problems (non-finite
 * force, a particle outside the grid, a sampling budget exhausted) are latched
 * in a device error word; calls that synchronise (sph_get_*, sph_sync) report
 * them. sph_last_error() gives a message for the last failing call.
 *
 * Layouts. Positions cross the boundary as row-major n x dim doubles in
 * original particle order (particle id = row), colours as n uint8, whatever
 * order the library keeps internally. A pointer argument named *_dev is device
 * memory when the accompanying `on_device` flag is 1, host memory otherwise.
 */
#ifndef SPHMESH_H
#define SPHMESH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SPH_OK = 0,
  SPH_ERR_INVALID_ARG = 1,   /* bad argument; nothing was changed */
  SPH_ERR_OOM = 2,           /* the allocator returned NULL */
  SPH_ERR_CUDA = 3,          /* a CUDA runtime call failed */
  SPH_ERR_NONFINITE = 4,     /* a density, force or position became NaN/Inf */
  SPH_ERR_OUT_OF_DOMAIN = 5, /* a particle left the grid (after projection) */
  SPH_ERR_CELL_OVERFLOW = 6, /* the cell grid would exceed its index range */
  SPH_ERR_TIMEOUT = 7,       /* a bounded device loop gave up */
  SPH_ERR_STATE = 8          /* call not valid in the handle's current state */
} sph_status;

/* Level-set constraints (Sec. 3.1, Eq. level_set_function). The mesh region
 * (phi > 0) is the box [lo, hi] intersected with every shape constraint. */
enum { SPH_SHAPE_SPHERE = 0, SPH_SHAPE_BOX = 1, SPH_SHAPE_GRID = 2 };

typedef struct {
  int32_t kind;        /* SPH_SHAPE_SPHERE, SPH_SHAPE_BOX, or SPH_SHAPE_GRID (the level set of
                          the background mesh, sph_create_background; center and size
                          unused, size[0] > 0) */
  int32_t keep_inside; /* 1: region inside the shape; 0: outside (a hole) */
  double center[3];
  double size[3];      /* sphere: size[0] = radius; box: half extents */
} sph_shape;

typedef struct {
  int32_t dim;         /* 2 or 3 */
  int32_t n_shapes;    /* 0..4 */
  double lo[3], hi[3]; /* bounding box (third component ignored in 2D) */
  sph_shape shapes[4];
} sph_domain;

/* Target density (Sec. 2.3, Eq. rho_target_function):
 *   rho_t(x) = rho_scale * s(x)^-d * (1 + sum_k poly[k] b_k(x~)),
 * s = s0 (SPH_FIELD_UNIFORM), a + b * |distance to shapes[dist_shape]|
 * (SPH_FIELD_LINEAR_DISTANCE) or a + b * tanh(s0 * |distance to
 * shapes[dist_shape]|) (SPH_FIELD_TANH_DISTANCE, s0 a reciprocal length: the
 * target size of the paper's circle case, Sec. 4.1, is
 * h_min + tanh(2.5 phi / 43) / tanh(2.5) (h_max - h_min), i.e. a = h_min,
 * b = (h_max - h_min) / tanh(2.5), s0 = 2.5 / 43), or the node values of a
 * background mesh interpolated at x (SPH_FIELD_BACKGROUND, sph_create_background);
 * x~ = 2 (x - lo)/(hi - lo) - 1 and b_k are
 *   2D: x, y, x^2, xy, y^2, x^3, x^2 y, x y^2;  3D: x, y, z, x^2, y^2, z^2, xy, yz.
 * rho_scale = 0 asks sph_create to choose it so that the total mass
 * M_v = integral of rho_t over the region (Eq. total_mass_2) equals the
 * particle count (unit mass, Eq. mass_SPH_particle). sum_k |poly[k]| < 1. */
enum { SPH_FIELD_UNIFORM = 0, SPH_FIELD_LINEAR_DISTANCE = 1, SPH_FIELD_TANH_DISTANCE = 2,
       SPH_FIELD_BACKGROUND = 3 /* s interpolated from the background mesh (sph_create_background) */ };

typedef struct {
  int32_t kind;
  int32_t dist_shape;
  double s0, a, b;
  int32_t n_poly;      /* 0..8 */
  int32_t reserved;
  double poly[8];
  double rho_scale;
} sph_field;

enum { SPH_PREC_FP32_SPLIT = 0, SPH_PREC_FP64 = 1 };

typedef struct {
  double P0;           /* EOS reference pressure (Eq. EOS_current) */
  double gamma;        /* EOS exponent; 2 gives the density-free force (Eq. EOS_2) */
  double sigma0;       /* initial surface-tension coefficient, 3 (Eq. sph_st_sigma) */
  double tau;          /* h = tau (m/rho_t)^(1/d) (Eq. scale_SPH_particle) */
  double kappa;        /* kernel support = kappa * h */
  int32_t precision;   /* SPH_PREC_FP32_SPLIT (FP32 offsets from cell origins) or SPH_PREC_FP64 */
  int32_t kernel_id;   /* 0: Wendland C2 (the only one) */
  uint64_t seed;       /* seed of the initial sampling (Philox4x32-10) */
  double cell_factor;  /* finest cell edge / smallest support; 0 -> 1.0 */
  int32_t block_size;  /* threads per block of the pair passes: 0 (256), 128 or 256 */
  int32_t use_graph;   /* 1: sph_step replays a captured CUDA graph of one step */
  int32_t record_fields; /* 1: keep rho, a_n and a~ of the last step for sph_get_field */
  int32_t list_capacity; /* neighbour-list entries per particle; 0 -> auto */
  double skin;           /* neighbour-list skin as a fraction of the support kappa h;
                            0 -> 0.15 in 3D, 0.2 in 2D; the list is rebuilt when a particle has moved
                            half its skin (results do not depend on it) */
} sph_params;

typedef struct {
  /* returns device memory of `bytes` bytes (16-byte aligned) or NULL */
  void* (*alloc)(size_t bytes, void* ctx);
  void (*free)(void* ptr, size_t bytes, void* ctx);
  void* ctx;
} sph_alloc;

typedef struct {
  int64_t step;            /* steps taken so far */
  double sigma;            /* surface-tension coefficient used in the last step */
  double dt1, dt2;         /* the two time-step sizes of the last step (Eq. time_step_size) */
  double min_rc_over_a;    /* min_i r_c,i/|a_i| of the last step */
  double max_a;            /* max_i |a_i| */
  double sum_rho;          /* sum_i rho_i (FP64 reduction) */
  double err_l2;           /* sum_i (rho_i/rho_t,i - 1)^2 */
  double err_max;          /* max_i |rho_i/rho_t,i - 1| */
  int64_t interface_pairs; /* unordered neighbour pairs with distinct colours */
  int64_t force_pairs;     /* unordered neighbour pairs (r_ij < kappa h_ij) */
  int64_t wall_moved;      /* particles moved by the level-set projection */
  double rho_scale;        /* rho_scale in use */
  int32_t error_flags;     /* latched device error bits (1 << sph_status) */
  int32_t n_levels;        /* cell levels of the multi-resolution grid */
  int64_t list_entries;    /* neighbour-list entries scanned by the last step (sum over i) */
  int64_t list_rebuilds;   /* neighbour-list builds so far */
  int32_t list_max;        /* longest list of the last build (> list_capacity: overflow) */
  int32_t list_capacity;   /* entries per particle the lists hold */
  double ramp_t0, ramp_t1; /* surface-tension ramp window in steps (-1: none yet) */
} sph_stats;

typedef struct {
  int32_t n_levels;
  int32_t dim;
  double lo[3];
  double h0;               /* smoothing length at the bottom of level 0 */
  double lip_h;            /* Lipschitz bound of h used to pick searched levels */
  double cell[8];          /* cell edge of each level (level l: cell[0] * 2^l) */
  int32_t dims[8][3];      /* cells per axis of each level */
  uint32_t base[9];        /* first cell key of each level; base[n_levels] = total */
} sph_grid_info;

typedef struct sph_handle sph_handle;

/* Create a relaxation instance: validate, fix rho_scale (Eq. total_mass_2),
 * draw n_particles positions with density proportional to rho_t in the region
 * and colour each by the nearest of n_colors generators drawn uniformly in the
 * region (the Voronoi initialisation of Sec. 4.2), build the multi-resolution
 * grid. n_colors in 1..256. `stream` is a cudaStream_t (NULL: legacy default).
 * Errors: INVALID_ARG, OOM, CUDA, CELL_OVERFLOW. */
sph_status sph_create(const sph_domain* dom, const sph_field* field, int64_t n_particles,
                      int32_t n_colors, const sph_params* params, const sph_alloc* alloc,
                      void* stream, sph_handle** out);

/* Feature-surface particles (Sec. 3.5): flags[id] != 0 (host, n bytes, by
 * particle id; NULL clears every flag) marks particle id as a surface
 * particle. A surface particle takes forces (pressure, surface tension,
 * viscous) from other surface particles only, drops their component along the
 * surface normal N (Eq. force_surface), and after every drift is moved onto the
 * surface it belongs to, r <- r - phi N (Eq. displacement_surface). Reading:
 * it belongs to the nearest constraint surface (the constraint value of
 * smallest magnitude, the bounding box first on ties) and N is that
 * constraint's unit normal into the region; the position is kept in the
 * bounding box first. Normal particles treat surface particles as ordinary
 * neighbours. sph_set_state and sph_load clear the flags; sph_backward refuses
 * a handle with flagged particles (INVALID_ARG). With rho_scale = 0 the field
 * is normalised to all n particles: pass rho_scale for the volume particles
 * alone (the paper's M_v) when using surface particles. Synchronises. */
sph_status sph_set_surface(sph_handle* h, const uint8_t* flags);

/* Cartesian background mesh (Sec. 3.1: the level set is discretised on a
 * Cartesian background mesh; Sec. 3.2: the target information is computed on
 * it and interpolated at the particle positions). Node (i, j, k) sits at
 * lo + (i, j, k) (hi - lo) / (dims - 1); values are stored x fastest. Values
 * are interpolated multilinearly (bilinear in 2D, trilinear in 3D) in the cell
 * that holds the point, points clamped into the mesh box. A level-set
 * constraint (SPH_SHAPE_GRID) violated by a particle is corrected by three
 * Newton steps x <- x - phi grad(phi) / |grad(phi)|^2 of the interpolant (the
 * printed Eq. displacement_surface when phi is a distance function). */
typedef struct {
  int32_t dims[3];       /* nodes per axis, >= 2 (dims[2] = 1 in 2D); product <= 2^28 */
  int32_t reserved;
  double lo[3], hi[3];   /* mesh box; must contain the domain box */
  const double* phi;     /* host: level set at the nodes, positive in the region (NULL: none) */
  const double* spacing; /* host: target spacing s > 0 at the nodes (NULL: none) */
} sph_background;

/* sph_create with a background mesh: shapes of kind SPH_SHAPE_GRID use bg->phi
 * and a field of kind SPH_FIELD_BACKGROUND uses bg->spacing (the distance
 * fields may also name a SPH_SHAPE_GRID shape). The node arrays are copied to
 * the device; the caller may free them when the call returns. sph_backward
 * refuses a handle with a SPH_SHAPE_GRID constraint (INVALID_ARG); the batch
 * API takes no background mesh. Errors as sph_create, and INVALID_ARG for an
 * inconsistent mesh. */
sph_status sph_create_background(const sph_domain* dom, const sph_field* field, const sph_background* bg,
                                 int64_t n_particles, int32_t n_colors, const sph_params* params,
                                 const sph_alloc* alloc, void* stream, sph_handle** out);

/* Replace the particle state (Algorithm 1 state = positions + colours; velocity
 * is zeroed every step, Sec. 3.3). xyz: n x dim doubles, col: n uint8 (colour <
 * 256), both in particle-id order, on the device if on_device else on the host.
 * Resets the step counter. Errors: INVALID_ARG, CUDA. */
sph_status sph_set_state(sph_handle* h, const double* xyz, const uint8_t* col, int32_t on_device);

/* Launch configuration (no counterpart in the paper: it changes how the work
 * is spread over the GPU, not what is computed). pass_threads: threads per
 * block of the two pair passes, 128 or 256 (0: keep; 256 at creation unless
 * params.block_size says 128); cell_factor: finest cell edge over the
 * smallest support, > 0 (0: keep), which rebuilds the multi-resolution grid;
 * stage_views: 1 runs the density/force pass (Algorithm 1's neighbour loop,
 * Sec. 3.3) staged, 0 unstaged, -1 keeps the setting. Staged, each list
 * rebuild also finds, per block of 256 particles (in cell order), the
 * distinct neighbours of their lists (at most 2,560, else that block stays
 * unstaged) and numbers every list entry by its rank in that set; every step
 * the pass copies the block's neighbour views into shared memory once and
 * reads them there instead of gathering each pair's view from global memory.
 * It applies to FP32 handles with gamma = 2, 256 threads per block and no
 * feature-surface particles (other configurations run unstaged) and costs a
 * second list array (4 bytes x list capacity per particle) plus 40 bytes per
 * particle of neighbour sets. The block size and staging leave every result
 * bit for bit unchanged; a new cell factor changes the cell order and so the
 * order of each particle's sums (rounding only). The next step rebuilds the
 * neighbour list; captured graphs are re-captured. Synchronises. Errors:
 * INVALID_ARG (stage_views = 1 on an FP64 handle), OOM, CELL_OVERFLOW.
 * sph_get_tuning reads the configuration in use (any pointer may be NULL). */
sph_status sph_set_tuning(sph_handle* h, int32_t pass_threads, double cell_factor, int32_t stage_views);
sph_status sph_get_tuning(const sph_handle* h, int32_t* pass_threads, double* cell_factor, int32_t* stage_views);

/* Coverage of the staged pass (sph_set_tuning): blocks of 256 particles,
 * how many of them the last list rebuild staged, and the neighbour views
 * they stage in all (0 and 0 while staging is off). Synchronises. */
sph_status sph_get_stage_info(sph_handle* h, int64_t* blocks, int64_t* staged_blocks, int64_t* staged_views);

/* Advance n_steps relaxation steps (Algorithm 1): cell list,
 * density + pressure + surface-tension forces, time step, viscous force,
 * two-stage integration, level-set projection. Asynchronous on the handle's
 * stream. Errors: INVALID_ARG, CUDA, STATE. */
sph_status sph_step(sph_handle* h, int32_t n_steps);

/* Like sph_step, but with direct launches and CUDA events on the handle's
 * stream around each phase; ms_out[0..2] receive the summed device time (ms)
 * of the cell-list build, pass A (density, pressure, surface tension,
 * reductions) and pass B (viscous force, integration, projection, re-keying)
 * over the n_steps steps. Synchronises. Errors: INVALID_ARG, CUDA. */
sph_status sph_step_profiled(sph_handle* h, int32_t n_steps, float* ms_out);

/* Surface-tension schedule (Eq. sph_st_sigma): sigma = sigma0 for step <= t0,
 * linear to 0 on (t0, t1], 0 after; step counted from sph_set_state/create.
 * t0 < 0 removes the ramp. Errors: INVALID_ARG (t1 <= t0 with t0 >= 0). */
sph_status sph_ramp_surface_tension(sph_handle* h, int64_t t0_step, int64_t t1_step);

/* Start the ramp automatically when the partition has converged (Sec. 3.3,
 * "topology static for e.g. 50 iterations"): after a step whose interface-pair
 * count closes a run of `window` steps that all stayed within `tol` (relative)
 * of the count that opened the run, t0 = that step and t1 = (1 + theta) t0
 * (theta in [0.1, 0.2] in the paper). The test runs on the device inside the
 * step (no host synchronisation); sph_get_stats reports the window it chose.
 * window = 0 turns it off; sph_ramp_surface_tension also turns it off.
 * Errors: INVALID_ARG (window < 0, tol < 0, theta <= 0). Synchronises. */
sph_status sph_auto_ramp(sph_handle* h, int32_t window, double tol, double theta);

/* Current positions (n x dim doubles, particle-id order). Synchronises. */
sph_status sph_get_positions(sph_handle* h, double* out, int32_t on_device);

/* Colours (n uint8, particle-id order). Synchronises. */
sph_status sph_get_colors(sph_handle* h, uint8_t* out, int32_t on_device);

/* Reductions of the last step (FP64 on the device). Synchronises and reports
 * latched device errors. */
sph_status sph_get_stats(sph_handle* h, sph_stats* out);

/* Per-colour size of the partition. The method partitions the domain into
 * sub-domains (one per colour) that are to be of equal size (Sec. 2.1) and
 * gives each its share of the total mass (Sec. 2.3, Eq. mass_for_partition).
 * volume[c] (n_colors doubles) receives V_c = sum over the particles of
 * colour c of m_i/rho_i (unit mass, rho_i the summation density of Eq.
 * density_sum from the last step), reduced in FP64 on the device in a fixed
 * order (repeated calls give identical bits); count[c] (n_colors int64, may
 * be NULL) the number of particles of colour c, i.e. its mass. Host arrays.
 * Errors: STATE when no step was taken since the state was set (create,
 * sph_set_state, sph_load, sph_backward). Synchronises. */
sph_status sph_get_color_volumes(sph_handle* h, double* volume, int64_t* count);

/* Per-particle results of the last step, particle-id order, as doubles:
 * SPH_OUT_RHO (n): summation density (Eq. density_sum);
 * SPH_OUT_ACC (n x dim): a_n = -F_p + F_s (Eqs. sph_pressure_force_2, sph_st_force);
 * SPH_OUT_VISC (n x dim): a~ (Eq. sph_viscous_force with rho := rho_t).
 * Needs params.record_fields = 1. Errors: STATE if nothing was recorded. */
enum { SPH_OUT_RHO = 0, SPH_OUT_ACC = 1, SPH_OUT_VISC = 2 };
sph_status sph_get_field(sph_handle* h, int32_t which, double* out, int32_t on_device);

/* Neighbour sets of the current state (Algorithm 1's neighbour search), per particle id:
 * density set (r_ij < kappa h_i, self included) and force set (j != i,
 * r_ij < kappa (h_i + h_j)/2): sizes and the sum of member ids. Any output may
 * be NULL. Host arrays. Synchronises. */
sph_status sph_neighbor_sets(sph_handle* h, int32_t* dens_count, int32_t* force_count,
                             int64_t* dens_idsum, int64_t* force_idsum);

/* Cell list of the current state (the cell structure the neighbour search of
 * Algorithm 1 runs on): cell key of each particle (particle-id order; the key
 * of level l = floor(log2(h/h0)) clamped to the grid's levels, cell c =
 * floor((x - lo)/cell_l) per axis, key = base_l + c_x + dims_x (c_y + dims_y
 * c_z), see sph_get_grid) and the particle ids in sorted order (by key, equal
 * keys by particle id). Host arrays. Synchronises. */
sph_status sph_get_cell_list(sph_handle* h, uint32_t* key_by_id, uint32_t* sorted_ids);

/* Grid description (levels, cell edges, dims, key bases). */
sph_status sph_get_grid(sph_handle* h, sph_grid_info* out);

/* Wait for the handle's stream; report latched device errors. */
sph_status sph_sync(sph_handle* h);

/* Checkpoint: the full state is positions + colours + step counter + the
 * sigma schedule (velocity is not state). With buf == NULL, *nbytes receives
 * the size needed. Synchronises. Layout (host byte order): a header of 8
 * int64 {magic 0x3148534D48505300, version 1, n, dim, step counter, 0, 0, 0},
 * the ramp window {t0, t1} as 2 doubles (-1: none), n x dim doubles
 * (positions, particle-id order), n bytes (colours). sph_load checks magic,
 * version, n and dim and takes the state, the step counter and the ramp
 * window from the blob. */
sph_status sph_save(sph_handle* h, void* buf, size_t* nbytes);
sph_status sph_load(sph_handle* h, const void* buf, size_t nbytes);

/* ---------------------------------------------------------------------------
 * Sensitivities of a relaxation run (reverse mode). The paper tunes nothing by
 * gradient; this differentiates K steps of Algorithm 1 as the
 * library computes them, for the objective
 *   L = w sum_i (rho_i/rho_t,i - 1)^2 + lambda sum_{i<j, C_i != C_j} W(r_ij, kappa h_ij)
 * at the end state (rho from Eq. density_sum, W the kernel), plus seed . x_K
 * when a seed (dL/dx_K of an outer loss) is given.
 *
 * Step sizes (Eq. time_step_size): with frozen_dt = 0 they are recomputed from
 * the state and their dependence is differentiated (the global minimum at its
 * argmin particle); with frozen_dt = 1 they are constants: those of dt_in when
 * given, else those this run chose.
 *
 * Memory: the run keeps the positions (FP64, by particle id) at the start of
 * every segment of ckpt_every steps and re-runs each segment from there into a
 * tape of ckpt_every steps (each step's state, a, a~, rho and force pairs:
 * roughly 100 + 4 * list_capacity bytes per particle) just before reversing it.
 * Checkpoints, tape and five n-sized reverse-pass arrays are allocated once
 * through the handle's allocator (grown when K or ckpt_every grows) and kept
 * until sph_destroy.
 * --------------------------------------------------------------------------- */
typedef struct {
  double density_weight; /* w: weight of the density-error term */
  double lambda;       /* weight of the interface term */
  int32_t frozen_dt;   /* 1: step sizes are constants; 0: recomputed and differentiated */
  int32_t ckpt_every;  /* checkpoint interval in steps (>= 1) */
} sph_objective;

typedef struct {
  double L;            /* objective at the end state (without the seed term) */
  double d_sigma0;     /* dL/dsigma0 (through the ramp, if any) */
  double d_gamma;      /* dL/dgamma (of the general equation of state p = P0 (rho/rho_t)^gamma) */
  double d_P0;         /* dL/dP0 (0 up to rounding when step sizes are recomputed: the run is P0-free) */
  double d_poly[8];    /* dL/dpoly[m], rho_scale held fixed */
} sph_grad;

/* From the handle's current state x_0 (step counter t), run K steps, evaluate
 * L at x_K and return the gradient: dpos0 (n x dim doubles, particle-id
 * order) = dL/dx_0 and *grad. The handle is left at x_K with counter t + K, as
 * after sph_step(h, K).
 *
 * Arguments: obj (not NULL); seed (n x dim, particle-id order) or NULL;
 * dt_in (2K doubles: dt1, dt2 per step) or NULL; dt_out (2K) or NULL receives
 * the step sizes used. seed, dt_in, dt_out and dpos0 live in device memory
 * when on_device = 1, else in host memory. Errors: INVALID_ARG (K < 0,
 * ckpt_every < 1, null obj/dpos0/grad, dt_in with frozen_dt = 0), OOM, and the
 * device errors of sph_step. Synchronises. */
sph_status sph_backward(sph_handle* h, int32_t K, const sph_objective* obj, const double* seed,
                        const double* dt_in, double* dt_out, double* dpos0, int32_t on_device, sph_grad* grad);

/* ---------------------------------------------------------------------------
 * Batches of independent instances (uneven sizes, 2D and 3D mixed). One CUDA
 * graph advances every instance by one step: instance k's kernels form one
 * branch-local chain, the branches fork from and join to the batch's stream and
 * run concurrently. The paper runs one instance at a time; batching is a
 * service of the library for many small problems on one GPU.
 * --------------------------------------------------------------------------- */
typedef struct {
  sph_domain dom;
  sph_field field;
  int64_t n_particles;
  int32_t n_colors;
  int32_t reserved;
  sph_params params;   /* use_graph is ignored (the batch graph replaces it) */
} sph_instance_desc;

typedef struct sph_batch sph_batch;

/* Create n_inst instances (as sph_create each, all on `stream`; NULL: a new
 * stream). n_branches > 0 fixes the number of graph branches; 0 leaves it to
 * sph_batch_tune (or 16 at the first step). Errors as sph_create. */
sph_status sph_batch_create(const sph_instance_desc* descs, int32_t n_inst, const sph_alloc* alloc, void* stream,
                            int32_t n_branches, sph_batch** out);

/* Autotuner: time steps_each graph-launched steps of the whole batch for each
 * candidate branch count and keep the fastest (instances are dealt longest
 * first, particles x dimension cost, to the least-loaded branch); then, one
 * knob at a time from the best so far, the launch configuration of every
 * instance (sph_set_tuning): 128 or 256 threads per block of the pair passes,
 * then cell factor 0.75, 1 or 1.5, then the staged pass on or off (FP32
 * instances).
 * Each trial starts from the same state; the trial steps are undone (the
 * state and step counters are restored). Synchronises. */
sph_status sph_batch_tune(sph_batch* b, const int32_t* candidates, int32_t n_candidates, int32_t steps_each);

/* One configuration the autotuner timed (or chose): graph branches, threads
 * per block of the pair passes, cell factor, its device time per batched
 * step, and whether the pass ran staged. */
typedef struct {
  int32_t branches;
  int32_t pass_threads;
  double cell_factor;
  float ms_per_step;
  int32_t stage_views;
} sph_batch_trial;

/* The autotuner's choice and its trials in order (trials may be NULL; at most
 * cap are written; *n_trials receives their number). */
sph_status sph_batch_tuning(const sph_batch* b, sph_batch_trial* chosen, sph_batch_trial* trials, int32_t cap,
                            int32_t* n_trials);

/* n_steps steps of every instance, one graph launch per step (async). */
sph_status sph_batch_step(sph_batch* b, int32_t n_steps);

/* Reference mode: the same steps as a loop of per-instance graph launches on
 * the batch's stream (one graph per instance and step). */
sph_status sph_batch_step_each(sph_batch* b, int32_t n_steps);

/* Instance k's handle (owned by the batch: use sph_get_positions, sph_get_stats
 * etc. on it; do not destroy it). */
sph_status sph_batch_get(sph_batch* b, int32_t k, sph_handle** h);

/* Instance count, branch count in use, and the autotuner's trials (n_tuned
 * entries of branch count and ms per step; arrays may be NULL, else they hold
 * at least n_candidates + 4 entries after sph_batch_tune; sph_batch_tuning
 * gives the trials' full configurations). */
sph_status sph_batch_info(const sph_batch* b, int32_t* n_inst, int32_t* n_branches, int32_t* n_tuned,
                          int32_t* tuned_branches, float* tuned_ms);

/* Wait for the batch's stream; report latched device errors of any instance. */
sph_status sph_batch_sync(sph_batch* b);
const char* sph_batch_last_error(const sph_batch* b);
void sph_batch_destroy(sph_batch* b);

/* Message of the last failing call on this handle (never NULL). */
const char* sph_last_error(const sph_handle* h);

/* Particle count, dimension and the rho_scale in use. */
sph_status sph_get_info(const sph_handle* h, int64_t* n_particles, int32_t* dim, double* rho_scale);

/* Release every buffer through the allocator that created it. */
void sph_destroy(sph_handle* h);

/* ---------------------------------------------------------------------------
 * Allocation-free evaluation (the paper has no counterpart; this is a service
 * of the library). Some callers cannot allocate device memory at the point
 * where they need the forces: a host framework that owns every device buffer
 * and forbids allocation inside its per-step callback, a real-time loop that
 * cannot afford cudaMalloc's implicit device synchronisation, or an embedded
 * runtime without an allocator. For them this call evaluates, for a given
 * particle state and without any handle, what the first pass of a relaxation
 * step evaluates (the density, a_n = -F_p + F_s and the two time steps), using
 * scratch space in a file-scope device array of the library instead of
 * allocations. It calls no cudaMalloc, cudaFree or allocating routine.
 *
 * Limits: n <= SPH_NOALLOC_MAX_PARTICLES; the multi-resolution grid the
 * problem needs must fit in SPH_NOALLOC_MAX_CELLS cells (raise
 * params->cell_factor otherwise); FP32 split precision only; field->rho_scale
 * must be given (> 0). Anything beyond: SPH_ERR_INVALID_ARG, nothing launched.
 * The scratch array (about 35 MB) is held by every GPU that loads the library
 * until the process exits. A particle with more than 95 neighbours inside its
 * support makes the call fail with SPH_ERR_CELL_OVERFLOW.
 *
 * Arguments: dom, field, params as for sph_create (sigma = params->sigma0, no
 * ramp); xyz_dev (n x dim doubles) and col_dev (n uint8) are device inputs in
 * particle-id order; rho_dev (n), acc_dev (n x dim) and dt_dev (2: dt1, dt2)
 * are device outputs, written in particle-id order. stream: a cudaStream_t
 * (NULL: legacy default stream).
 *
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress) with that device current. Every call synchronises
 * `stream` and copies the device error word into host memory before it
 * returns, so no call may be made while `stream` (or, with stream NULL, the
 * legacy default stream) is being captured into a CUDA graph. Every call
 * reuses the same array and leaves its contents behind (the counters it needs
 * zeroed are cleared at the start of each call); calls that overlap on the GPU
 * (two streams, two threads) race on it and must be serialised by the caller.
 * Device-side errors come back through the status: SPH_ERR_NONFINITE,
 * SPH_ERR_OUT_OF_DOMAIN, SPH_ERR_CELL_OVERFLOW (more than 95 neighbours),
 * SPH_ERR_TIMEOUT, and SPH_ERR_CUDA for any other device error bit. */
#define SPH_NOALLOC_MAX_PARTICLES 32768
#define SPH_NOALLOC_MAX_CELLS (1 << 19)
sph_status sph_eval_forces_noalloc(const sph_domain* dom, const sph_field* field, const sph_params* params,
                                   int64_t n, const double* xyz_dev, const uint8_t* col_dev, double* rho_dev,
                                   double* acc_dev, double* dt_dev, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SPHMESH_H */
