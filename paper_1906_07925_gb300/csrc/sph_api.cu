// Host side of the C ABI (include/sphmesh.h): handle, validation, grid and
// frame set-up, buffer ownership through the caller's allocator, step
// orchestration (direct launches or a replayed CUDA graph of one step),
// accessors, checkpoints.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/sphmesh.h"
#include "sph_host.h"
#include "sph_internal.h"

using namespace sph;

struct sph_handle {
  int dim = 2, prec = SPH_PREC_FP32_SPLIT, ncol = 1;
  int64_t n = 0;
  sph_domain dom{};
  sph_field field{};
  sph_params par{};
  sph_alloc alloc{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  double rho_scale = 1.0, lip_h = 0.0, hmin = 0.0, hmax = 0.0;
  // background mesh (sph_create_background): device node arrays, the mesh box
  // and the interpolants' gradient bounds
  bool has_bg = false, bg_grid_shape = false;
  bool has_surface = false;  // feature-surface particles flagged (sph_set_surface)
  const double* bg_phi = nullptr;
  const double* bg_s = nullptr;
  int bg_n[3] = {1, 1, 1};
  double bg_lo[3] = {0, 0, 0}, bg_hi[3] = {0, 0, 0};
  double bg_lip_phi = 1.0, bg_lip_s = 0.0;
  HostGrid hg{};
  Grid<float> Gf{};
  Grid<double> Gdw{};
  Frame<float> Ff{};
  Frame<double> Fd{};
  Geom<float> geof{};
  Geom<double> geod{};
  Phys<float> Pf{};
  Phys<double> Pd{};
  DevState S{};
  std::vector<std::pair<void*, size_t>> blocks;
  int64_t steps = 0;
  double t0 = -1.0, t1 = -1.0;
  int auto_window = 0;  // > 0: automatic ramp start (sph_auto_ramp)
  double auto_tol = 0.0, auto_theta = 0.0;
  bool recorded = false;
  bool rho_valid = false;
  // step-size history of a running sph_backward (the control block's dt_*)
  double* dt_hist = nullptr;
  long long dt_base = 0;
  int dt_len = 0, dt_mode = 0;
  uint32_t cells_cap = 0;  // cells the cell arrays hold  // S.rho holds the summation density of the current positions' last pass A
  // per-colour volume scratch (sph_get_color_volumes; allocated on first use)
  double* cv_part = nullptr;
  unsigned long long* cv_cpart = nullptr;
  double* cv_out = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int graph_record = -1;
  // reverse-pass buffers (allocated by the first sph_backward)
  struct {
    bool ready = false;
    void *xb = nullptr, *atb = nullptr, *ab = nullptr, *hb = nullptr, *Tb = nullptr, *rtb = nullptr,
         *rhob = nullptr;
    double *part = nullptr, *acc = nullptr, *g[2] = {nullptr, nullptr};
    unsigned* ticket = nullptr;
    uint8_t* col = nullptr;  // colours by particle id
    std::vector<DevState> tape;  // taped-step slots (grown on demand, freed with the handle)
    std::vector<cudaGraphExec_t> g_rerun;     // per slot: re-run step
    std::vector<cudaGraphExec_t> g_rev[2][2];  // per step-size mode, direction (g0 -> g1, g1 -> g0) and slot
    double *ck = nullptr, *xk = nullptr, *dts = nullptr, *seed = nullptr;  // checkpoints, x_K, step sizes, seed
    size_t ck_n = 0, dts_n = 0;                                           // their capacities (grown on demand)
  } adj;
  std::string err;
};

namespace {

// ------------------------------------------------------------------ util --
void* default_alloc_fn(size_t bytes, void* ctx) {
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, (cudaStream_t)ctx) != cudaSuccess) return nullptr;
  return p;
}
void default_free_fn(void* p, size_t, void* ctx) { cudaFreeAsync(p, (cudaStream_t)ctx); }

sph_status fail(sph_handle* h, sph_status s, const std::string& msg) {
  if (h) h->err = msg;
  return s;
}

sph_status cuda_fail(sph_handle* h, cudaError_t e, const char* where) {
  return fail(h, SPH_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define SPH_CUDA(h, expr)                                    \
  do {                                                       \
    cudaError_t e_ = (expr);                                 \
    if (e_ != cudaSuccess) return cuda_fail((h), e_, #expr); \
  } while (0)

#define SPH_TRY(expr)            \
  do {                           \
    sph_status s_ = (expr);      \
    if (s_ != SPH_OK) return s_; \
  } while (0)

template <class P>
sph_status grab(sph_handle* h, P*& out, size_t count) {
  size_t bytes = std::max<size_t>(count * sizeof(P), 16);
  bytes = (bytes + 255) & ~size_t(255);
  void* p = h->alloc.alloc(bytes, h->alloc.ctx);
  if (!p) return fail(h, SPH_ERR_OOM, "allocation of " + std::to_string(bytes) + " bytes failed");
  h->blocks.emplace_back(p, bytes);
  out = (P*)p;
  return SPH_OK;
}

sph_status status_from_flags(sph_handle* h, int flags) {
  if (flags & kErrNonfinite) return fail(h, SPH_ERR_NONFINITE, "non-finite density, force or position");
  if (flags & kErrOutOfDomain) return fail(h, SPH_ERR_OUT_OF_DOMAIN, "a particle was outside the box");
  if (flags & kErrListOverflow)
    return fail(h, SPH_ERR_CELL_OVERFLOW, "a neighbour list exceeded its capacity (raise params.list_capacity)");
  if (flags & kErrTimeout) return fail(h, SPH_ERR_TIMEOUT, "a bounded device loop gave up");
  return SPH_OK;
}

// list skin (fraction of kappa h) when params.skin = 0: a longer list costs
// every step, a shorter one more frequent rebuilds. 3D: on the 8M-particle
// graded workload (20 graph-replayed steps after 5 warm-up steps) 0.15 took
// 5.94 ms per step against 6.6 / 6.33 / 6.16 ms for 0.12 / 0.2 / 0.25 (5.93
// vs 6.16 ms for 0.15 / 0.2 over 50 steps). 2D: 0.2 (the 262,144-particle
// polynomial-field workload: 20 steps in 2.77 ms against 2.82 at 0.15).
inline double default_skin(int dim) { return dim == 3 ? 0.15 : 0.2; }

// position frames and kernel grids (make_frames in sph_host.h)
void setup_frames(sph_handle* h) {
  Frames fr;
  make_frames(h->dom, h->par.kappa, h->par.skin > 0 ? h->par.skin : default_skin(h->dim), h->hg, fr);
  h->Ff = fr.f;
  h->Fd = fr.d;
  h->Gf = fr.gf;
  h->Gdw = fr.gd;
}

// expected list length for a support kappa h and a skin: the ball of radius
// kappa h (1 + skin) holds about V_d (kappa tau (1 + skin))^d particles
// Expected list length: the list radius R = kappa max(h_i, h_j)(1 + skin) is at
// most g h_i with g = kappa (1 + skin) / (1 - kappa L (1 + skin)) (h_j <= h_i + L r,
// L the field's Lipschitz bound of h), and inside that ball the number density
// (tau/h)^d is at most (tau/h_i)^d / (1 - L g)^d. The capacity is the larger of
// twice that and that plus ten standard deviations of a Poisson count (random
// initial states cluster), plus 16.
int auto_capacity(const sph_handle* h) {
  const double skin = h->par.skin > 0 ? h->par.skin : default_skin(h->dim);
  const double k1 = h->par.kappa * (1.0 + skin);
  const double L = std::min(h->lip_h, 0.5 / k1);
  const double g = k1 / (1.0 - L * k1);
  const double dens = std::pow(1.0 / std::max(1.0 - L * g, 0.25), (double)h->dim);
  const double r = h->par.tau * g * 1.05;
  const double e = (h->dim == 2 ? M_PI * r * r : 4.0 / 3.0 * M_PI * r * r * r) * dens;
  int cap = (int)std::ceil(std::max(2.0 * e, e + 10.0 * std::sqrt(e)) + 16.0);
  return (cap + 7) & ~7;
}

// FP32 handles start with the staged pass A on (sph_set_tuning switches it)
constexpr bool kStageDefault = false;

// buffers of the staged pass A (FP32 handles): the list again with ranks in
// each block's neighbour set, the sets and their counts (-1: not staged until
// the next list rebuild fills them)
sph_status ensure_stage(sph_handle* h) {
  DevState& S = h->S;
  if (S.llist) return SPH_OK;
  const size_t N = (size_t)std::max<int64_t>(h->n, 1), nb = (N + kStageBlock - 1) / kStageBlock;
  SPH_TRY(grab(h, S.llist, N * (size_t)S.cap));
  SPH_TRY(grab(h, S.scount, nb));
  SPH_TRY(grab(h, S.sj, nb * (size_t)kStageCap));
  SPH_CUDA(h, cudaMemsetAsync(S.scount, 0xFF, sizeof(int) * nb, h->stream));
  SPH_CUDA(h, h->dim == 2 ? prepare_staged_pass<2>() : prepare_staged_pass<3>());
  return SPH_OK;
}

// one relaxation step on the handle's stream; dt_fix (device, may be null)
// prescribes {dt1, dt2}, dt_rec (device, may be null) receives them. Sx (may
// be null: the handle's own) redirects buffers; with `tape`, the state pass A
// used is copied into it before pass B moves the particles.
sph_status launch_step(sph_handle* h, int record, int force_rebuild = 0, cudaEvent_t* ev = nullptr,
                       const double* dt_fix = nullptr, double* dt_rec = nullptr, const DevState* Sx = nullptr,
                       const DevState* tape = nullptr) {
  const DevState& S = Sx ? *Sx : h->S;
  PassFlags f;
  f.f32 = &h->Ff;
  f.general_eos = h->par.gamma != 2.0;
  f.record = record;
  f.dt_fix = dt_fix;
  f.dt_rec = dt_rec;
  const bool f64 = h->prec == SPH_PREC_FP64;
  f.geo = f64 ? (const void*)&h->geod : (const void*)&h->geof;
  f.surface = h->has_surface ? 1 : 0;
  cudaError_t e = cudaSuccess;
  if (ev) e = cudaEventRecord(ev[0], h->stream);
  if (e == cudaSuccess) e = launch_gate(S, force_rebuild, h->stream);
  if (e == cudaSuccess) {
    if (h->dim == 2)
      e = f64 ? launch_rebuild<2, double>(S, h->Gdw, h->Fd, h->geod, h->par.kappa, h->stream, &h->Gf, &h->Ff)
              : launch_rebuild<2, float>(S, h->Gf, h->Ff, h->geof, (float)h->par.kappa, h->stream);
    else
      e = f64 ? launch_rebuild<3, double>(S, h->Gdw, h->Fd, h->geod, h->par.kappa, h->stream, &h->Gf, &h->Ff)
              : launch_rebuild<3, float>(S, h->Gf, h->Ff, h->geof, (float)h->par.kappa, h->stream);
  }
  if (ev && e == cudaSuccess) e = cudaEventRecord(ev[1], h->stream);
  if (e == cudaSuccess) {
    if (h->dim == 2)
      e = f64 ? launch_pass_a<2, double>(S, h->Fd, h->Pd, f, h->stream)
              : launch_pass_a<2, float>(S, h->Ff, h->Pf, f, h->stream);
    else
      e = f64 ? launch_pass_a<3, double>(S, h->Fd, h->Pd, f, h->stream)
              : launch_pass_a<3, float>(S, h->Ff, h->Pf, f, h->stream);
  }
  if (tape && e == cudaSuccess) {
    if (h->dim == 2)
      e = f64 ? launch_tape_snapshot<2, double>(S, *tape, h->stream) : launch_tape_snapshot<2, float>(S, *tape, h->stream);
    else
      e = f64 ? launch_tape_snapshot<3, double>(S, *tape, h->stream) : launch_tape_snapshot<3, float>(S, *tape, h->stream);
  }
  if (ev && e == cudaSuccess) e = cudaEventRecord(ev[2], h->stream);
  if (e == cudaSuccess) {
    if (h->dim == 2)
      e = f64 ? launch_pass_b<2, double>(S, h->Fd, h->Pd, h->geod, f, h->stream)
              : launch_pass_b<2, float>(S, h->Ff, h->Pf, h->geof, f, h->stream);
    else
      e = f64 ? launch_pass_b<3, double>(S, h->Fd, h->Pd, h->geod, f, h->stream)
              : launch_pass_b<3, float>(S, h->Ff, h->Pf, h->geof, f, h->stream);
  }
  if (ev && e == cudaSuccess) e = cudaEventRecord(ev[3], h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "step kernels");
  return SPH_OK;
}

// a list rebuild plus pass A without advancing (diagnostics); the next step
// rebuilds again so that its views are fresh
sph_status launch_evaluate(sph_handle* h, int nbr_debug) {
  DevState S = h->S;
  S.scal = h->S.scal + 1;  // keep the last step's statistics
  PassFlags f;
  f.f32 = &h->Ff;
  f.general_eos = h->par.gamma != 2.0;
  f.nbr_debug = nbr_debug;
  f.advance = 0;
  const bool f64 = h->prec == SPH_PREC_FP64;
  f.geo = f64 ? (const void*)&h->geod : (const void*)&h->geof;
  f.surface = h->has_surface ? 1 : 0;
  cudaError_t e = launch_gate(S, 1, h->stream);
  if (e == cudaSuccess) {
    if (h->dim == 2)
      e = f64 ? launch_rebuild<2, double>(S, h->Gdw, h->Fd, h->geod, h->par.kappa, h->stream, &h->Gf, &h->Ff)
              : launch_rebuild<2, float>(S, h->Gf, h->Ff, h->geof, (float)h->par.kappa, h->stream);
    else
      e = f64 ? launch_rebuild<3, double>(S, h->Gdw, h->Fd, h->geod, h->par.kappa, h->stream, &h->Gf, &h->Ff)
              : launch_rebuild<3, float>(S, h->Gf, h->Ff, h->geof, (float)h->par.kappa, h->stream);
  }
  if (e == cudaSuccess) {
    if (h->dim == 2)
      e = f64 ? launch_pass_a<2, double>(S, h->Fd, h->Pd, f, h->stream)
              : launch_pass_a<2, float>(S, h->Ff, h->Pf, f, h->stream);
    else
      e = f64 ? launch_pass_a<3, double>(S, h->Fd, h->Pd, f, h->stream)
              : launch_pass_a<3, float>(S, h->Ff, h->Pf, f, h->stream);
  }
  if (e == cudaSuccess) e = launch_request_rebuild(S, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "evaluate");
  h->recorded = false;
  return SPH_OK;
}

sph_status ensure_graph(sph_handle* h, int record) {
  // the captured step depends on field recording and on whether pass A takes
  // its feature-surface variant
  const int key = record | (h->has_surface ? 2 : 0);
  if (h->gexec && h->graph_record == key) return SPH_OK;
  if (h->gexec) {
    cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
  }
  cudaGraph_t g = nullptr;
  SPH_CUDA(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  sph_status s = launch_step(h, record);
  cudaError_t e = cudaStreamEndCapture(h->stream, &g);
  if (s != SPH_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&h->gexec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
  h->graph_record = key;
  return SPH_OK;
}

// every captured graph of the handle (the step's and the reverse pass's): they
// bake launch configurations, grids and frames into their nodes
void drop_graphs(sph_handle* h) {
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  h->gexec = nullptr;
  h->graph_record = -1;
  for (auto* v : {&h->adj.g_rerun, &h->adj.g_rev[0][0], &h->adj.g_rev[0][1], &h->adj.g_rev[1][0],
                  &h->adj.g_rev[1][1]})
    for (cudaGraphExec_t& g : *v)
      if (g) {
        cudaGraphExecDestroy(g);
        g = nullptr;
      }
}

// whole control block (set-up / set_state: the next step rebuilds the list)
sph_status write_ctl_all(sph_handle* h) {
  StepCtl c{};
  c.step = h->steps;
  c.t0 = h->t0;
  c.t1 = h->t1;
  c.sigma0 = h->par.sigma0;
  c.buf = 0;
  c.vp = 0;
  c.rebuild = 0;
  c.need_rebuild = 1;
  c.rebuilds = 0;
  c.auto_on = h->auto_window > 0;
  c.auto_window = h->auto_window;
  c.auto_tol = h->auto_tol;
  c.auto_theta = h->auto_theta;
  c.auto_ref = -1;
  c.dt_hist = h->dt_hist;
  c.dt_base = h->dt_base;
  c.dt_len = h->dt_len;
  c.dt_mode = h->dt_mode;
  SPH_CUDA(h, launch_write_ctl(h->S, c, h->stream));
  return SPH_OK;
}

// the step-size history fields of the control block only (the list
// bookkeeping and the schedule stay on the device)
sph_status write_ctl_hist(sph_handle* h) {
  struct {
    double* hist;
    long long base;
    int len, mode;
  } v{h->dt_hist, h->dt_base, h->dt_len, h->dt_mode};
  static_assert(sizeof v == offsetof(StepCtl, dt_mode) + sizeof(int) - offsetof(StepCtl, dt_hist), "layout");
  SPH_CUDA(h, cudaMemcpyAsync((char*)h->S.ctl + offsetof(StepCtl, dt_hist), &v, sizeof v, cudaMemcpyHostToDevice,
                              h->stream));
  return SPH_OK;
}

// only the schedule and the counter (the list bookkeeping stays on the device);
// with the automatic ramp on, the device owns the schedule
sph_status write_ctl_sched(sph_handle* h) {
  const double sched[2] = {h->t0, h->t1};
  const long long step = h->steps;
  SPH_CUDA(h, cudaMemcpyAsync((char*)h->S.ctl + offsetof(StepCtl, step), &step, sizeof step,
                              cudaMemcpyHostToDevice, h->stream));
  if (h->auto_window <= 0)
    SPH_CUDA(h, cudaMemcpyAsync((char*)h->S.ctl + offsetof(StepCtl, t0), sched, sizeof sched,
                                cudaMemcpyHostToDevice, h->stream));
  SPH_CUDA(h, cudaStreamSynchronize(h->stream));
  return SPH_OK;
}

sph_status read_flags(sph_handle* h, int* flags) {
  SPH_CUDA(h, cudaMemcpyAsync(flags, h->S.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  SPH_CUDA(h, cudaStreamSynchronize(h->stream));
  return SPH_OK;
}

sph_status do_set_state(sph_handle* h, const double* xyz_dev, const uint8_t* col_dev) {
  DevState& S = h->S;
  h->has_surface = false;  // the meta words are rewritten from the colours
  cudaError_t e;
  const bool f64 = h->prec == SPH_PREC_FP64;
  if (h->dim == 2)
    e = f64 ? launch_set_state<2, double>(S, h->Fd, xyz_dev, col_dev, h->stream)
            : launch_set_state<2, float>(S, h->Ff, xyz_dev, col_dev, h->stream);
  else
    e = f64 ? launch_set_state<3, double>(S, h->Fd, xyz_dev, col_dev, h->stream)
            : launch_set_state<3, float>(S, h->Ff, xyz_dev, col_dev, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "set_state");
  h->steps = 0;
  h->recorded = false;
  h->rho_valid = false;
  return write_ctl_all(h);
}

// temporary device buffer through the handle's allocator, released at scope end
struct Temp {
  sph_handle* h;
  void* p = nullptr;
  size_t bytes = 0;
  Temp(sph_handle* hh, size_t b) : h(hh), bytes(std::max<size_t>(b, 16)) { p = h->alloc.alloc(bytes, h->alloc.ctx); }
  ~Temp() {
    if (p) {
      cudaStreamSynchronize(h->stream);
      h->alloc.free(p, bytes, h->alloc.ctx);
    }
  }
};

// ------------------------------------------------------- reverse pass --
// state from positions by id (device) at step counter `step`; the next gate
// rebuilds the list
sph_status set_state_at(sph_handle* h, const double* xyz_dev, const uint8_t* col_dev, int64_t step) {
  const bool f64 = h->prec == SPH_PREC_FP64;
  cudaError_t e;
  if (h->dim == 2)
    e = f64 ? launch_set_state<2, double>(h->S, h->Fd, xyz_dev, col_dev, h->stream)
            : launch_set_state<2, float>(h->S, h->Ff, xyz_dev, col_dev, h->stream);
  else
    e = f64 ? launch_set_state<3, double>(h->S, h->Fd, xyz_dev, col_dev, h->stream)
            : launch_set_state<3, float>(h->S, h->Ff, xyz_dev, col_dev, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "set_state");
  h->steps = step;
  h->recorded = false;
  h->rho_valid = false;
  return write_ctl_all(h);
}

sph_status positions_to(sph_handle* h, double* dst_dev) {
  const bool f64 = h->prec == SPH_PREC_FP64;
  cudaError_t e;
  if (h->dim == 2)
    e = f64 ? launch_get_positions<2, double>(h->S, h->Fd, dst_dev, h->stream)
            : launch_get_positions<2, float>(h->S, h->Ff, dst_dev, h->stream);
  else
    e = f64 ? launch_get_positions<3, double>(h->S, h->Fd, dst_dev, h->stream)
            : launch_get_positions<3, float>(h->S, h->Ff, dst_dev, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "get_positions");
  return SPH_OK;
}

// list rebuild at the current state (then the forward quantities of the step
// when `forward`: pass A without advancing, pass B recording a~ without moving)
sph_status reverse_setup(sph_handle* h, bool forward, const double* dt_fix) {
  DevState& S = h->S;
  PassFlags f;
  f.f32 = &h->Ff;
  f.general_eos = h->par.gamma != 2.0;
  f.record = 1;
  f.advance = 0;
  f.move = 0;
  f.dt_fix = dt_fix;
  const bool f64 = h->prec == SPH_PREC_FP64;
  // without `forward` (the objective at x_K) the list is rebuilt only if the
  // last step asked for it: otherwise it still holds every pair of x_K
  cudaError_t e = launch_gate(S, forward ? 1 : 0, h->stream);
  if (e == cudaSuccess) {
    if (h->dim == 2)
      e = f64 ? launch_rebuild<2, double>(S, h->Gdw, h->Fd, h->geod, h->par.kappa, h->stream, &h->Gf, &h->Ff)
              : launch_rebuild<2, float>(S, h->Gf, h->Ff, h->geof, (float)h->par.kappa, h->stream);
    else
      e = f64 ? launch_rebuild<3, double>(S, h->Gdw, h->Fd, h->geod, h->par.kappa, h->stream, &h->Gf, &h->Ff)
              : launch_rebuild<3, float>(S, h->Gf, h->Ff, h->geof, (float)h->par.kappa, h->stream);
  }
  if (forward && e == cudaSuccess) {
    if (h->dim == 2)
      e = f64 ? launch_pass_a<2, double>(S, h->Fd, h->Pd, f, h->stream)
              : launch_pass_a<2, float>(S, h->Ff, h->Pf, f, h->stream);
    else
      e = f64 ? launch_pass_a<3, double>(S, h->Fd, h->Pd, f, h->stream)
              : launch_pass_a<3, float>(S, h->Ff, h->Pf, f, h->stream);
  }
  if (forward && e == cudaSuccess) {
    if (h->dim == 2)
      e = f64 ? launch_pass_b<2, double>(S, h->Fd, h->Pd, h->geod, f, h->stream)
              : launch_pass_b<2, float>(S, h->Ff, h->Pf, h->geof, f, h->stream);
    else
      e = f64 ? launch_pass_b<3, double>(S, h->Fd, h->Pd, h->geod, f, h->stream)
              : launch_pass_b<3, float>(S, h->Ff, h->Pf, h->geof, f, h->stream);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "reverse set-up");
  return SPH_OK;
}

sph_status ensure_adj(sph_handle* h) {
  if (h->adj.ready) return SPH_OK;
  const size_t N = (size_t)h->n, d = (size_t)h->dim;
  const size_t t1 = h->prec == SPH_PREC_FP64 ? 8 : 4, v4 = 4 * t1;
  const size_t nb = N / 256 + 2;
  auto& a = h->adj;
  uint8_t* p = nullptr;
  SPH_TRY(grab(h, p, N * 32)); a.xb = p;
  SPH_TRY(grab(h, p, N * v4)); a.atb = p;
  SPH_TRY(grab(h, p, N * v4)); a.ab = p;
  SPH_TRY(grab(h, p, N * t1)); a.hb = p;
  SPH_TRY(grab(h, p, N * t1)); a.Tb = p;
  SPH_TRY(grab(h, p, N * t1)); a.rtb = p;
  SPH_TRY(grab(h, p, N * t1)); a.rhob = p;
  SPH_TRY(grab(h, a.part, nb * kAdjPartials));
  SPH_TRY(grab(h, a.acc, (size_t)kAdjSlots));
  SPH_TRY(grab(h, a.g[0], N * d));
  SPH_TRY(grab(h, a.g[1], N * d));
  SPH_TRY(grab(h, a.ticket, 4));
  SPH_TRY(grab(h, a.col, N));
  SPH_CUDA(h, cudaMemsetAsync(a.ticket, 0, 16, h->stream));
  a.ready = true;
  return SPH_OK;
}

template <class T>
AdjBufs<T> adj_bufs(sph_handle* h, const double* gin, double* gout) {
  AdjBufs<T> B;
  auto& a = h->adj;
  B.gin = gin;
  B.gout = gout;
  B.xb = (V4<double>*)a.xb;
  B.atb = (V4<T>*)a.atb;
  B.ab = (V4<T>*)a.ab;
  B.hb = (T*)a.hb;
  B.Tb = (T*)a.Tb;
  B.rtb = (T*)a.rtb;
  B.rhob = (T*)a.rhob;
  B.part = a.part;
  B.acc = a.acc;
  B.ticket = a.ticket;
  return B;
}

sph_status run_objective(sph_handle* h, double wd, double lambda, const double* seed, double* gout) {
  cudaError_t e;
  const bool f64 = h->prec == SPH_PREC_FP64;
  if (h->dim == 2)
    e = f64 ? launch_objective<2, double>(h->S, h->Fd, h->Pd, h->geod, adj_bufs<double>(h, seed, gout), wd,
                                          lambda, h->stream)
            : launch_objective<2, float>(h->S, h->Ff, h->Pf, h->geof, adj_bufs<float>(h, seed, gout), wd,
                                         lambda, h->stream);
  else
    e = f64 ? launch_objective<3, double>(h->S, h->Fd, h->Pd, h->geod, adj_bufs<double>(h, seed, gout), wd,
                                          lambda, h->stream)
            : launch_objective<3, float>(h->S, h->Ff, h->Pf, h->geof, adj_bufs<float>(h, seed, gout), wd,
                                         lambda, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "objective");
  return SPH_OK;
}

sph_status run_bwd_step(sph_handle* h, const DevState& S, const double* gin, double* gout, int recomputed) {
  cudaError_t e;
  const bool f64 = h->prec == SPH_PREC_FP64;
  const int gen = h->par.gamma != 2.0;
  if (h->dim == 2)
    e = f64 ? launch_bwd_step<2, double>(S, h->Fd, h->Pd, h->geod, adj_bufs<double>(h, gin, gout), recomputed, gen,
                                         h->stream)
            : launch_bwd_step<2, float>(S, h->Ff, h->Pf, h->geof, adj_bufs<float>(h, gin, gout), recomputed, gen,
                                        h->stream);
  else
    e = f64 ? launch_bwd_step<3, double>(S, h->Fd, h->Pd, h->geod, adj_bufs<double>(h, gin, gout), recomputed, gen,
                                         h->stream)
            : launch_bwd_step<3, float>(S, h->Ff, h->Pf, h->geof, adj_bufs<float>(h, gin, gout), recomputed, gen,
                                        h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "reverse step");
  return SPH_OK;
}

// Per-step record of a taped step: the state pass A used (current order), the
// step's forward results (a, g, a~, rho, p/rho^2, this step's force pairs),
// its control block and scalars, and with a general EOS its neighbour list.
// Slots are allocated once (through the handle's allocator) and reused.
sph_status ensure_tape(sph_handle* h, int slots) {
  const size_t N = (size_t)h->n, cap = (size_t)h->S.cap;
  const size_t t1 = h->prec == SPH_PREC_FP64 ? 8 : 4, v4 = 4 * t1;
  const bool gen = h->par.gamma != 2.0;
  auto& tape = h->adj.tape;
  while ((int)tape.size() < slots) {
    DevState T = h->S;
    uint8_t* p = nullptr;
    SPH_TRY(grab(h, p, N * 32)); T.X[0] = T.X[1] = p;
    SPH_TRY(grab(h, T.meta[0], N)); T.meta[1] = T.meta[0];
    SPH_TRY(grab(h, T.pid[0], N)); T.pid[1] = T.pid[0];
    SPH_TRY(grab(h, p, N * v4)); T.view[0] = T.view[1] = p;
    SPH_TRY(grab(h, T.plist, N * cap));
    SPH_TRY(grab(h, T.pcount, N));
    SPH_TRY(grab(h, p, N * v4)); T.acc4 = p;
    SPH_TRY(grab(h, p, N * v4)); T.visc = p;
    SPH_TRY(grab(h, p, N * t1)); T.rho = p;
    SPH_TRY(grab(h, p, N * t1)); T.pc = p;
    SPH_TRY(grab(h, T.ctl, 1));
    SPH_TRY(grab(h, T.scal, 1));
    if (gen) {
      SPH_TRY(grab(h, T.list, N * cap));
      SPH_TRY(grab(h, T.lcount, N));
    }
    tape.push_back(T);
    h->adj.g_rerun.push_back(nullptr);
    for (auto& m : h->adj.g_rev)
      for (auto& v : m) v.push_back(nullptr);
  }
  return SPH_OK;
}

// instantiate what `body` issues on the handle's stream as a graph
template <class Body>
sph_status capture(sph_handle* h, cudaGraphExec_t* out, Body&& body) {
  cudaGraph_t g = nullptr;
  SPH_CUDA(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  sph_status s = body();
  cudaError_t e = cudaStreamEndCapture(h->stream, &g);
  if (s != SPH_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
  return SPH_OK;
}

// one step writing its forward results into tape slot T (and the state into it)
sph_status taped_step(sph_handle* h, const DevState& T, const double* dt_fix, double* dt_rec) {
  DevState S2 = h->S;
  S2.plist = T.plist;
  S2.pcount = T.pcount;
  S2.acc4 = T.acc4;
  S2.visc = T.visc;
  S2.rho = T.rho;
  S2.pc = T.pc;
  SPH_TRY(launch_step(h, 1, 0, nullptr, dt_fix, dt_rec, &S2, &T));
  if (T.list != h->S.list) {
    SPH_CUDA(h, cudaMemcpyAsync(T.list, h->S.list, (size_t)h->n * (size_t)h->S.cap * 4, cudaMemcpyDeviceToDevice,
                                h->stream));
    SPH_CUDA(h, cudaMemcpyAsync(T.lcount, h->S.lcount, (size_t)h->n * 4, cudaMemcpyDeviceToDevice, h->stream));
  }
  return SPH_OK;
}


}  // namespace

// gradient bound of the multilinear interpolant of node values v: in a cell,
// d/dx_k is a convex combination of the cell's k-edge differences / h_k
static double bg_slope(const sph_background& b, int d, const double* v) {
  double s2 = 0.0;
  const int64_t nx = b.dims[0], ny = b.dims[1], nz = b.dims[2];
  for (int k = 0; k < d; ++k) {
    const double hk = (b.hi[k] - b.lo[k]) / (b.dims[k] - 1);
    const int64_t step = k == 0 ? 1 : (k == 1 ? nx : nx * ny);
    double m = 0.0;
    for (int64_t q = 0; q < nx * ny * nz; ++q) {
      const int64_t ik = k == 0 ? q % nx : (k == 1 ? (q / nx) % ny : q / (nx * ny));
      if (ik + 1 < b.dims[k]) m = std::max(m, fabs(v[q + step] - v[q]) / hk);
    }
    s2 += m * m;
  }
  return sqrt(s2);
}

template <class T>
static void set_bg(const sph_handle* h, Geom<T>& g) {
  g.bg_phi = h->bg_phi;
  g.bg_s = h->bg_s;
  for (int k = 0; k < 3; ++k) {
    g.bg_n[k] = h->bg_n[k];
    g.bg_lo[k] = (T)h->bg_lo[k];
    const double hk = h->bg_n[k] > 1 ? (h->bg_hi[k] - h->bg_lo[k]) / (h->bg_n[k] - 1) : 1.0;
    g.bg_h[k] = (T)hk;
    g.bg_inv_h[k] = (T)(1.0 / hk);
  }
}

// ================================================================== C ABI ==
extern "C" {

void sph_destroy(sph_handle* h);

static sph_status create_impl(sph_handle* h, const sph_domain* dom, const sph_field* field, int64_t n_particles,
                              int32_t n_colors, const sph_params* params, const sph_alloc* alloc, void* stream,
                              const sph_background* bg) {
  h->dom = *dom;
  h->field = *field;
  h->par = *params;
  h->dim = dom->dim;
  h->prec = params->precision;
  h->n = n_particles;
  h->ncol = n_colors;
  h->stream = (cudaStream_t)stream;
  if (!h->stream) {
    SPH_CUDA(h, cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    h->own_stream = true;
  }
  if (alloc && alloc->alloc && alloc->free) {
    h->alloc = *alloc;
  } else {
    h->alloc.alloc = default_alloc_fn;
    h->alloc.free = default_free_fn;
    h->alloc.ctx = (void*)h->stream;
  }
  const int d = h->dim;
  const int nn = (int)n_particles;

  // ---- background mesh: node arrays to the device ----
  if (bg) {
    h->has_bg = true;
    const size_t nodes = (size_t)bg->dims[0] * bg->dims[1] * bg->dims[2];
    for (int k = 0; k < 3; ++k) {
      h->bg_n[k] = bg->dims[k];
      h->bg_lo[k] = bg->lo[k];
      h->bg_hi[k] = bg->hi[k];
    }
    for (int s = 0; s < dom->n_shapes; ++s) h->bg_grid_shape |= dom->shapes[s].kind == SPH_SHAPE_GRID;
    if (bg->phi) {
      double* dv;
      SPH_TRY(grab(h, dv, nodes));
      SPH_CUDA(h, cudaMemcpy(dv, bg->phi, nodes * sizeof(double), cudaMemcpyHostToDevice));
      h->bg_phi = dv;
      h->bg_lip_phi = bg_slope(*bg, d, bg->phi);
    }
    if (bg->spacing) {
      double* dv;
      SPH_TRY(grab(h, dv, nodes));
      SPH_CUDA(h, cudaMemcpy(dv, bg->spacing, nodes * sizeof(double), cudaMemcpyHostToDevice));
      h->bg_s = dv;
      h->bg_lip_s = bg_slope(*bg, d, bg->spacing);
    }
  }
  // |grad s| bound: the field's slope, times the background level set's
  // gradient bound when the distance is measured to it
  double gslope = field_slope(h->field);
  if (h->field.kind == SPH_FIELD_BACKGROUND) gslope = h->bg_lip_s;
  else if (h->field.kind != SPH_FIELD_UNIFORM && dom->n_shapes > 0 &&
           dom->shapes[h->field.dist_shape].kind == SPH_SHAPE_GRID)
    gslope *= h->bg_lip_phi;

  // ---- target field: total mass (Eq. total_mass_2) and the range of h ----
  Geom<double> g1;
  fill_geom<double>(h->dom, h->field, 1.0, 1.0, g1);
  set_bg(h, g1);
  const int res = d == 2 ? 2048 : 192;
  FieldBounds fb{};
  {
    Temp scratch(h, sizeof(double) * field_bounds_scratch_doubles());
    if (!scratch.p) return fail(h, SPH_ERR_OOM, "scratch allocation failed");
    cudaError_t e = d == 2 ? field_bounds<2>(g1, res, &fb, (double*)scratch.p, h->stream)
                           : field_bounds<3>(g1, res, &fb, (double*)scratch.p, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "field_bounds");
  }
  if (!(fb.sum_w > 0)) return fail(h, SPH_ERR_INVALID_ARG, "the region is empty at the sampling resolution");
  double cellvol = 1.0;
  for (int k = 0; k < d; ++k) cellvol *= (h->dom.hi[k] - h->dom.lo[k]) / res;
  const double mass1 = fb.sum_w * cellvol;  // integral of s^-d (1+P)
  h->rho_scale = field->rho_scale > 0 ? field->rho_scale : (n_particles > 0 ? (double)n_particles / mass1 : 1.0);
  const double hfac = h->par.tau * pow(h->rho_scale, -1.0 / d);
  // sampled bounds of h, widened by the Lipschitz bound over half a sample cell
  double diag = 0.0;
  for (int k = 0; k < d; ++k) diag += pow((h->dom.hi[k] - h->dom.lo[k]) / res, 2);
  diag = sqrt(diag);
  h->lip_h = lipschitz_h(h->dom, h->field, hfac, fb.max_seff * (1.0 + 1e-6) + gslope * diag, gslope);
  h->hmin = std::max(0.5 * hfac * fb.min_seff, hfac * fb.min_seff - h->lip_h * diag);
  h->hmax = hfac * fb.max_seff + h->lip_h * diag;
  fill_geom<double>(h->dom, h->field, hfac, h->rho_scale, h->geod);
  fill_geom<float>(h->dom, h->field, hfac, h->rho_scale, h->geof);
  set_bg(h, h->geod);
  set_bg(h, h->geof);
  fill_phys(d, h->par, h->Pf);
  fill_phys(d, h->par, h->Pd);
  {
    const std::string why = grid_setup(h->dom, h->par.kappa, h->par.cell_factor, h->hmin, h->hmax, h->lip_h, h->hg);
    if (!why.empty())
      return fail(h, why == "cell grid too large" ? SPH_ERR_CELL_OVERFLOW : SPH_ERR_INVALID_ARG, why);
    h->S.total_cells = h->hg.base[h->hg.n_levels];
  }
  setup_frames(h);

  // ---- buffers ----
  DevState& S = h->S;
  S.n = nn;
  S.dim = d;
  S.fp64 = h->prec == SPH_PREC_FP64;
  S.cap = h->par.list_capacity > 0 ? h->par.list_capacity : std::min(auto_capacity(h), kMaxListCapacity);
  S.pass_threads = h->par.block_size == 128 ? 128 : 256;
  const size_t v4 = S.fp64 ? 32 : 16, t1 = S.fp64 ? 8 : 4;
  const size_t N = (size_t)std::max<int64_t>(n_particles, 1);
  uint8_t* tmpb;
  for (int b = 0; b < 2; ++b) {
    SPH_TRY(grab(h, tmpb, N * 32)); S.X[b] = tmpb;
    SPH_TRY(grab(h, S.meta[b], N));
    SPH_TRY(grab(h, S.pid[b], N));
    SPH_TRY(grab(h, tmpb, N * v4)); S.view[b] = tmpb;
  }
  SPH_TRY(grab(h, tmpb, N * v4)); S.vbuild = tmpb;
  if (h->prec == SPH_PREC_FP64) {
    SPH_TRY(grab(h, tmpb, N * 16)); S.view32 = tmpb;
  }
  SPH_TRY(grab(h, tmpb, N * v4)); S.acc4 = tmpb;
  SPH_TRY(grab(h, tmpb, N * v4)); S.visc = tmpb;
  SPH_TRY(grab(h, tmpb, N * t1)); S.rho = tmpb;
  SPH_TRY(grab(h, tmpb, N * t1)); S.pc = tmpb;
  SPH_TRY(grab(h, S.key, N));
  SPH_TRY(grab(h, S.tmp, N));
  SPH_TRY(grab(h, S.list, N * (size_t)S.cap));
  SPH_TRY(grab(h, S.lcount, N));
  SPH_TRY(grab(h, S.plist, N * (size_t)S.cap));
  SPH_TRY(grab(h, S.pcount, N));
  SPH_TRY(grab(h, S.cnt, (size_t)S.total_cells));
  h->cells_cap = S.total_cells;
  SPH_TRY(grab(h, S.cstart, (size_t)S.total_cells + 1));
  SPH_TRY(grab(h, S.scan_part, (size_t)S.total_cells / 4096 + 2));
  SPH_TRY(grab(h, S.partials, N / 128 + 2));
  SPH_TRY(grab(h, S.scal, 2));
  SPH_TRY(grab(h, S.ctl, 1));
  SPH_TRY(grab(h, S.tickets, 4));
  SPH_TRY(grab(h, S.err, 1));
  SPH_CUDA(h, cudaMemsetAsync(S.cnt, 0, sizeof(uint32_t) * S.total_cells, h->stream));
  SPH_CUDA(h, cudaMemsetAsync(S.tickets, 0, sizeof(unsigned) * 4, h->stream));
  SPH_CUDA(h, cudaMemsetAsync(S.err, 0, sizeof(int), h->stream));
  SPH_CUDA(h, cudaMemsetAsync(S.scal, 0, sizeof(Scalars) * 2, h->stream));
  SPH_CUDA(h, cudaMemsetAsync(S.lcount, 0, sizeof(uint32_t) * N, h->stream));
  if (!S.fp64 && kStageDefault) {
    SPH_TRY(ensure_stage(h));
    S.stage = 1;
  }

  // ---- initial state ----
  {
    Temp xyz(h, sizeof(double) * N * d), col(h, N), gens(h, sizeof(double) * 3 * 256);
    if (!xyz.p || !col.p || !gens.p) return fail(h, SPH_ERR_OOM, "scratch allocation failed");
    const double wmax = fb.max_w * 1.25;
    cudaError_t e = d == 2 ? sample_positions<2>(g1, nn, n_colors, params->seed, wmax, (double*)xyz.p,
                                                 (uint8_t*)col.p, (double*)gens.p, S.err, h->stream)
                           : sample_positions<3>(g1, nn, n_colors, params->seed, wmax, (double*)xyz.p,
                                                 (uint8_t*)col.p, (double*)gens.p, S.err, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "sample_positions");
    SPH_TRY(do_set_state(h, (const double*)xyz.p, (const uint8_t*)col.p));
    SPH_CUDA(h, cudaStreamSynchronize(h->stream));
  }
  int flags = 0;
  SPH_TRY(read_flags(h, &flags));
  return status_from_flags(h, flags);
}

static sph_status create_common(const sph_domain* dom, const sph_field* field, const sph_background* bg,
                                int64_t n_particles, int32_t n_colors, const sph_params* params,
                                const sph_alloc* alloc, void* stream, sph_handle** out, const char* who) {
  if (!out) return SPH_ERR_INVALID_ARG;
  *out = nullptr;
  std::string why;
  sph_status vs = validate(dom, field, n_particles, n_colors, params, why, bg);
  if (vs == SPH_OK && n_particles > (int64_t)(1 << 24)) {
    why = "at most 2^24 particles per instance";
    vs = SPH_ERR_INVALID_ARG;
  }
  if (vs == SPH_OK && (params->skin < 0 || params->list_capacity < 0 || params->list_capacity > kMaxListCapacity)) {
    why = "skin must be >= 0 and list_capacity in 0..32767";
    vs = SPH_ERR_INVALID_ARG;
  }
  if (vs == SPH_OK && params->block_size != 0 && params->block_size != 128 && params->block_size != 256) {
    why = "block_size must be 0, 128 or 256";
    vs = SPH_ERR_INVALID_ARG;
  }
  if (vs != SPH_OK) {
    fprintf(stderr, "%s: %s\n", who, why.c_str());
    return vs;
  }
  sph_handle* h = new sph_handle();
  sph_status s = create_impl(h, dom, field, n_particles, n_colors, params, alloc, stream, bg);
  if (s != SPH_OK) {
    fprintf(stderr, "%s: %s\n", who, h->err.c_str());
    sph_destroy(h);
    return s;
  }
  *out = h;
  return SPH_OK;
}

sph_status sph_create(const sph_domain* dom, const sph_field* field, int64_t n_particles, int32_t n_colors,
                      const sph_params* params, const sph_alloc* alloc, void* stream, sph_handle** out) {
  return create_common(dom, field, nullptr, n_particles, n_colors, params, alloc, stream, out, "sph_create");
}

sph_status sph_create_background(const sph_domain* dom, const sph_field* field, const sph_background* bg,
                                 int64_t n_particles, int32_t n_colors, const sph_params* params,
                                 const sph_alloc* alloc, void* stream, sph_handle** out) {
  if (!bg) return SPH_ERR_INVALID_ARG;
  return create_common(dom, field, bg, n_particles, n_colors, params, alloc, stream, out, "sph_create_background");
}

sph_status sph_set_state(sph_handle* h, const double* xyz, const uint8_t* col, int32_t on_device) {
  if (!h || (h->n > 0 && (!xyz || !col))) return fail(h, SPH_ERR_INVALID_ARG, "null state");
  const size_t N = (size_t)h->n, d = (size_t)h->dim;
  SPH_CUDA(h, cudaMemsetAsync(h->S.err, 0, sizeof(int), h->stream));
  if (on_device) {
    SPH_TRY(do_set_state(h, xyz, col));
  } else {
    Temp tx(h, sizeof(double) * N * d), tc(h, N);
    if (!tx.p || !tc.p) return fail(h, SPH_ERR_OOM, "scratch allocation failed");
    SPH_CUDA(h, cudaMemcpyAsync(tx.p, xyz, sizeof(double) * N * d, cudaMemcpyHostToDevice, h->stream));
    SPH_CUDA(h, cudaMemcpyAsync(tc.p, col, N, cudaMemcpyHostToDevice, h->stream));
    SPH_TRY(do_set_state(h, (const double*)tx.p, (const uint8_t*)tc.p));
    SPH_CUDA(h, cudaStreamSynchronize(h->stream));
  }
  int flags = 0;
  SPH_TRY(read_flags(h, &flags));
  return status_from_flags(h, flags);
}

sph_status sph_set_surface(sph_handle* h, const uint8_t* flags) {
  if (!h) return SPH_ERR_INVALID_ARG;
  const size_t N = (size_t)h->n;
  bool any = false;
  if (flags)
    for (size_t q = 0; q < N && !any; ++q) any = flags[q] != 0;
  if (N > 0) {
    Temp tf(h, any ? N : 1);
    if (!tf.p) return fail(h, SPH_ERR_OOM, "scratch allocation failed");
    if (any) SPH_CUDA(h, cudaMemcpyAsync(tf.p, flags, N, cudaMemcpyHostToDevice, h->stream));
    SPH_CUDA(h, launch_set_surface(h->S, any ? (const uint8_t*)tf.p : nullptr, h->stream));
    SPH_CUDA(h, cudaStreamSynchronize(h->stream));
  }
  h->has_surface = any;
  return SPH_OK;
}

sph_status sph_set_tuning(sph_handle* h, int32_t pass_threads, double cell_factor, int32_t stage_views) {
  if (!h) return SPH_ERR_INVALID_ARG;
  if ((pass_threads != 0 && pass_threads != 128 && pass_threads != 256) || !(cell_factor >= 0.0) ||
      cell_factor > 16.0 || stage_views < -1 || stage_views > 1)
    return fail(h, SPH_ERR_INVALID_ARG,
                "pass_threads in {0, 128, 256}, 0 <= cell_factor <= 16, stage_views in {-1, 0, 1}");
  if (stage_views == 1 && h->S.fp64)
    return fail(h, SPH_ERR_INVALID_ARG, "the staged pass exists for the FP32 split precision only");
  SPH_CUDA(h, cudaStreamSynchronize(h->stream));
  drop_graphs(h);
  if (pass_threads) h->S.pass_threads = pass_threads;
  if (stage_views == 1) SPH_TRY(ensure_stage(h));
  if (stage_views >= 0) h->S.stage = stage_views;
  const double cf_now = h->par.cell_factor > 0 ? h->par.cell_factor : 1.0;
  if (cell_factor > 0 && cell_factor != cf_now) {
    HostGrid hg;
    const std::string why = grid_setup(h->dom, h->par.kappa, cell_factor, h->hmin, h->hmax, h->lip_h, hg);
    if (!why.empty())
      return fail(h, why == "cell grid too large" ? SPH_ERR_CELL_OVERFLOW : SPH_ERR_INVALID_ARG, why);
    const uint32_t cells = hg.base[hg.n_levels];
    if (cells > h->cells_cap) {  // larger cell arrays (the old ones are released with the handle)
      uint32_t *cnt, *cstart, *part;
      SPH_TRY(grab(h, cnt, (size_t)cells));
      SPH_TRY(grab(h, cstart, (size_t)cells + 1));
      SPH_TRY(grab(h, part, (size_t)cells / 4096 + 2));
      h->S.cnt = cnt;
      h->S.cstart = cstart;
      h->S.scan_part = part;
      h->cells_cap = cells;
    }
    SPH_CUDA(h, cudaMemsetAsync(h->S.cnt, 0, sizeof(uint32_t) * cells, h->stream));
    h->hg = hg;
    h->S.total_cells = cells;
    h->par.cell_factor = cell_factor;
    setup_frames(h);
    for (DevState& T : h->adj.tape) {
      T.cnt = h->S.cnt;
      T.cstart = h->S.cstart;
      T.scan_part = h->S.scan_part;
      T.total_cells = cells;
    }
  }
  for (DevState& T : h->adj.tape) {
    T.pass_threads = h->S.pass_threads;
    T.stage = h->S.stage;
    T.llist = h->S.llist;
    T.scount = h->S.scount;
    T.sj = h->S.sj;
  }
  // the next step rebuilds the list (and, after a new grid, the views)
  SPH_CUDA(h, launch_request_rebuild(h->S, h->stream));
  SPH_CUDA(h, cudaStreamSynchronize(h->stream));
  return SPH_OK;
}

sph_status sph_get_tuning(const sph_handle* h, int32_t* pass_threads, double* cell_factor, int32_t* stage_views) {
  if (!h) return SPH_ERR_INVALID_ARG;
  if (pass_threads) *pass_threads = h->S.pass_threads;
  if (cell_factor) *cell_factor = h->par.cell_factor > 0 ? h->par.cell_factor : 1.0;
  if (stage_views) *stage_views = h->S.stage;
  return SPH_OK;
}

sph_status sph_get_stage_info(sph_handle* h, int64_t* blocks, int64_t* staged_blocks, int64_t* staged_views) {
  if (!h) return SPH_ERR_INVALID_ARG;
  const size_t nb = ((size_t)std::max<int64_t>(h->n, 1) + kStageBlock - 1) / kStageBlock;
  int64_t sb = 0, sv = 0;
  if (h->S.stage && h->S.scount) {
    std::vector<int> c(nb);
    SPH_CUDA(h, cudaMemcpyAsync(c.data(), h->S.scount, sizeof(int) * nb, cudaMemcpyDeviceToHost, h->stream));
    SPH_CUDA(h, cudaStreamSynchronize(h->stream));
    for (int v : c)
      if (v >= 0) {
        ++sb;
        sv += v;
      }
  }
  if (blocks) *blocks = (int64_t)nb;
  if (staged_blocks) *staged_blocks = sb;
  if (staged_views) *staged_views = sv;
  return SPH_OK;
}

sph_status sph_step(sph_handle* h, int32_t n_steps) {
  if (!h || n_steps < 0) return fail(h, SPH_ERR_INVALID_ARG, "bad step count");
  if (h->n == 0 || n_steps == 0) {
    h->steps += n_steps;
    return write_ctl_sched(h);
  }
  const int record = h->par.record_fields ? 1 : 0;
  if (h->par.use_graph) {
    SPH_TRY(ensure_graph(h, record));
    for (int s = 0; s < n_steps; ++s) SPH_CUDA(h, cudaGraphLaunch(h->gexec, h->stream));
  } else {
    for (int s = 0; s < n_steps; ++s) SPH_TRY(launch_step(h, record));
  }
  h->steps += n_steps;
  h->recorded = record;
  h->rho_valid = true;
  return SPH_OK;
}

sph_status sph_step_profiled(sph_handle* h, int32_t n_steps, float* ms_out) {
  if (!h || n_steps < 0 || !ms_out) return fail(h, SPH_ERR_INVALID_ARG, "bad arguments");
  ms_out[0] = ms_out[1] = ms_out[2] = 0.0f;
  if (h->n == 0 || n_steps == 0) return SPH_OK;
  const int record = h->par.record_fields ? 1 : 0;
  cudaEvent_t ev[4];
  for (auto& e : ev) SPH_CUDA(h, cudaEventCreate(&e));
  sph_status st = SPH_OK;
  for (int s = 0; s < n_steps && st == SPH_OK; ++s) {
    st = launch_step(h, record, 0, ev);
    if (st != SPH_OK) break;
    cudaError_t e = cudaEventSynchronize(ev[3]);
    float t;
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
      e = cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
      ms_out[k] += t;
    }
    if (e != cudaSuccess) st = cuda_fail(h, e, "profiled step");
    else h->steps += 1;
  }
  for (auto& e : ev) cudaEventDestroy(e);
  h->recorded = record && st == SPH_OK;
  h->rho_valid = h->rho_valid || st == SPH_OK;
  return st;
}

sph_status sph_ramp_surface_tension(sph_handle* h, int64_t t0, int64_t t1) {
  if (!h) return SPH_ERR_INVALID_ARG;
  if (t0 >= 0 && t1 <= t0) return fail(h, SPH_ERR_INVALID_ARG, "ramp needs t1 > t0");
  SPH_CUDA(h, cudaStreamSynchronize(h->stream));
  h->t0 = t0 < 0 ? -1.0 : (double)t0;
  h->t1 = t0 < 0 ? -1.0 : (double)t1;
  if (h->auto_window > 0) {  // an explicit schedule replaces the automatic one
    h->auto_window = 0;
    const int off = 0;
    SPH_CUDA(h, cudaMemcpyAsync((char*)h->S.ctl + offsetof(StepCtl, auto_on), &off, sizeof off,
                                cudaMemcpyHostToDevice, h->stream));
  }
  return write_ctl_sched(h);
}

sph_status sph_auto_ramp(sph_handle* h, int32_t window, double tol, double theta) {
  if (!h || window < 0 || !(tol >= 0.0) || !(theta > 0.0)) return fail(h, SPH_ERR_INVALID_ARG, "bad arguments");
  SPH_CUDA(h, cudaStreamSynchronize(h->stream));
  StepCtl c{};
  SPH_CUDA(h, cudaMemcpy(&c, h->S.ctl, sizeof c, cudaMemcpyDeviceToHost));
  h->auto_window = window;
  h->auto_tol = tol;
  h->auto_theta = theta;
  if (window > 0) {
    h->t0 = h->t1 = -1.0;
    c.t0 = c.t1 = -1.0;
  }
  c.auto_on = window > 0;
  c.auto_window = window;
  c.auto_tol = tol;
  c.auto_theta = theta;
  c.auto_stable = 0;
  c.auto_done = 0;
  c.auto_ref = -1;
  SPH_CUDA(h, launch_write_ctl(h->S, c, h->stream));
  SPH_CUDA(h, cudaStreamSynchronize(h->stream));
  return SPH_OK;
}

sph_status sph_get_positions(sph_handle* h, double* out, int32_t on_device) {
  if (!h || (h->n > 0 && !out)) return fail(h, SPH_ERR_INVALID_ARG, "null output");
  const size_t N = (size_t)h->n, d = (size_t)h->dim;
  double* dst = out;
  Temp t(h, on_device ? 0 : sizeof(double) * N * d);
  if (!on_device) dst = (double*)t.p;
  cudaError_t e;
  const bool f64 = h->prec == SPH_PREC_FP64;
  if (h->dim == 2)
    e = f64 ? launch_get_positions<2, double>(h->S, h->Fd, dst, h->stream)
            : launch_get_positions<2, float>(h->S, h->Ff, dst, h->stream);
  else
    e = f64 ? launch_get_positions<3, double>(h->S, h->Fd, dst, h->stream)
            : launch_get_positions<3, float>(h->S, h->Ff, dst, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "get_positions");
  if (!on_device) SPH_CUDA(h, cudaMemcpyAsync(out, dst, sizeof(double) * N * d, cudaMemcpyDeviceToHost, h->stream));
  SPH_CUDA(h, cudaStreamSynchronize(h->stream));
  int flags = 0;
  SPH_TRY(read_flags(h, &flags));
  return status_from_flags(h, flags);
}

sph_status sph_get_colors(sph_handle* h, uint8_t* out, int32_t on_device) {
  if (!h || (h->n > 0 && !out)) return fail(h, SPH_ERR_INVALID_ARG, "null output");
  const size_t N = (size_t)h->n;
  Temp t(h, on_device ? 0 : N);
  uint8_t* dst = on_device ? out : (uint8_t*)t.p;
  cudaError_t e = launch_get_colors(h->S, dst, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "get_colors");
  if (!on_device) SPH_CUDA(h, cudaMemcpyAsync(out, dst, N, cudaMemcpyDeviceToHost, h->stream));
  SPH_CUDA(h, cudaStreamSynchronize(h->stream));
  return SPH_OK;
}

sph_status sph_get_stats(sph_handle* h, sph_stats* out) {
  if (!h || !out) return fail(h, SPH_ERR_INVALID_ARG, "null output");
  Scalars sc{};
  int flags = 0;
  SPH_CUDA(h, cudaMemcpyAsync(&sc, h->S.scal, sizeof sc, cudaMemcpyDeviceToHost, h->stream));
  SPH_CUDA(h, cudaMemcpyAsync(&flags, h->S.err, sizeof flags, cudaMemcpyDeviceToHost, h->stream));
  StepCtl ctl{};
  SPH_CUDA(h, cudaMemcpyAsync(&ctl, h->S.ctl, sizeof ctl, cudaMemcpyDeviceToHost, h->stream));
  SPH_CUDA(h, cudaStreamSynchronize(h->stream));
  memset(out, 0, sizeof *out);
  out->step = h->steps;
  out->sigma = sc.sigma;
  out->dt1 = sc.dt1;
  out->dt2 = sc.dt2;
  out->min_rc_over_a = sc.min_rc_a >= DBL_MAX ? INFINITY : sc.min_rc_a;
  out->max_a = sc.max_a;
  out->sum_rho = sc.sum_rho;
  out->err_l2 = sc.err_l2;
  out->err_max = sc.err_max;
  out->interface_pairs = sc.ipairs;
  out->force_pairs = sc.fpairs;
  out->wall_moved = sc.wall_moved;
  out->rho_scale = h->rho_scale;
  out->error_flags = flags;
  out->n_levels = h->hg.n_levels;
  out->list_entries = sc.lentries;
  out->list_rebuilds = ctl.rebuilds;
  out->list_max = ctl.lmax;
  out->list_capacity = h->S.cap;
  out->ramp_t0 = ctl.t0;
  out->ramp_t1 = ctl.t1;
  if (h->auto_window > 0 && ctl.auto_done) {  // the device fixed the schedule
    h->t0 = ctl.t0;
    h->t1 = ctl.t1;
  }
  return status_from_flags(h, flags);
}

sph_status sph_get_color_volumes(sph_handle* h, double* volume, int64_t* count) {
  if (!h || !volume) return fail(h, SPH_ERR_INVALID_ARG, "null output");
  if (!h->rho_valid) return fail(h, SPH_ERR_STATE, "no step since the state was set: no densities to sum");
  const int nc = h->ncol;
  if (h->n == 0) {
    for (int c = 0; c < nc; ++c) {
      volume[c] = 0.0;
      if (count) count[c] = 0;
    }
    return SPH_OK;
  }
  if (!h->cv_out) {
    const size_t nb = (size_t)color_volume_blocks((int)h->n);
    SPH_TRY(grab(h, h->cv_part, nb * 256));
    SPH_TRY(grab(h, h->cv_cpart, nb * 256));
    SPH_TRY(grab(h, h->cv_out, 512));
  }
  long long* cnt_d = (long long*)(h->cv_out + 256);
  cudaError_t e = h->prec == SPH_PREC_FP64
                      ? launch_color_volumes<double>(h->S, h->cv_part, h->cv_cpart, h->cv_out, cnt_d, h->stream)
                      : launch_color_volumes<float>(h->S, h->cv_part, h->cv_cpart, h->cv_out, cnt_d, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "color volumes");
  double v[256];
  long long k[256];
  SPH_CUDA(h, cudaMemcpyAsync(v, h->cv_out, sizeof v, cudaMemcpyDeviceToHost, h->stream));
  SPH_CUDA(h, cudaMemcpyAsync(k, cnt_d, sizeof k, cudaMemcpyDeviceToHost, h->stream));
  SPH_CUDA(h, cudaStreamSynchronize(h->stream));
  for (int c = 0; c < nc; ++c) {
    volume[c] = v[c];
    if (count) count[c] = (int64_t)k[c];
  }
  int flags = 0;
  SPH_TRY(read_flags(h, &flags));
  return status_from_flags(h, flags);
}

sph_status sph_get_field(sph_handle* h, int32_t which, double* out, int32_t on_device) {
  if (!h || (h->n > 0 && !out) || which < 0 || which > 2) return fail(h, SPH_ERR_INVALID_ARG, "bad field request");
  if (!h->recorded) return fail(h, SPH_ERR_STATE, "no recorded step (set params.record_fields and step)");
  const size_t N = (size_t)h->n, cnt = which == 0 ? N : N * (size_t)h->dim;
  Temp t(h, on_device ? 0 : sizeof(double) * cnt);
  double* dst = on_device ? out : (double*)t.p;
  cudaError_t e;
  const bool f64 = h->prec == SPH_PREC_FP64;
  if (h->dim == 2)
    e = f64 ? launch_get_fields<2, double>(h->S, which, dst, h->stream)
            : launch_get_fields<2, float>(h->S, which, dst, h->stream);
  else
    e = f64 ? launch_get_fields<3, double>(h->S, which, dst, h->stream)
            : launch_get_fields<3, float>(h->S, which, dst, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "get_field");
  if (!on_device) SPH_CUDA(h, cudaMemcpyAsync(out, dst, sizeof(double) * cnt, cudaMemcpyDeviceToHost, h->stream));
  SPH_CUDA(h, cudaStreamSynchronize(h->stream));
  return SPH_OK;
}

sph_status sph_neighbor_sets(sph_handle* h, int32_t* dens_count, int32_t* force_count, int64_t* dens_idsum,
                             int64_t* force_idsum) {
  if (!h) return SPH_ERR_INVALID_ARG;
  const size_t N = (size_t)std::max<int64_t>(h->n, 1);
  if (!h->S.dbg_count) {
    SPH_TRY(grab(h, h->S.dbg_count, 2 * N));
    SPH_TRY(grab(h, h->S.dbg_sum, 2 * N));
  }
  if (h->n == 0) return SPH_OK;
  SPH_TRY(launch_evaluate(h, 1));
  std::vector<int32_t> cnt(2 * N);
  std::vector<long long> sum(2 * N);
  SPH_CUDA(h, cudaMemcpyAsync(cnt.data(), h->S.dbg_count, sizeof(int32_t) * 2 * N, cudaMemcpyDeviceToHost,
                              h->stream));
  SPH_CUDA(h, cudaMemcpyAsync(sum.data(), h->S.dbg_sum, sizeof(long long) * 2 * N, cudaMemcpyDeviceToHost,
                              h->stream));
  SPH_CUDA(h, cudaStreamSynchronize(h->stream));
  for (size_t i = 0; i < (size_t)h->n; ++i) {
    if (dens_count) dens_count[i] = cnt[2 * i];
    if (force_count) force_count[i] = cnt[2 * i + 1];
    if (dens_idsum) dens_idsum[i] = sum[2 * i];
    if (force_idsum) force_idsum[i] = sum[2 * i + 1];
  }
  int flags = 0;
  SPH_TRY(read_flags(h, &flags));
  return status_from_flags(h, flags);
}

sph_status sph_get_cell_list(sph_handle* h, uint32_t* key_by_id, uint32_t* sorted_ids) {
  if (!h) return SPH_ERR_INVALID_ARG;
  if (h->n == 0) return SPH_OK;
  const size_t N = (size_t)h->n;
  SPH_TRY(launch_evaluate(h, 0));
  // after the rebuild: keys were computed in the old order (buffer 1 - buf)
  StepCtl c{};
  SPH_CUDA(h, cudaMemcpyAsync(&c, h->S.ctl, sizeof c, cudaMemcpyDeviceToHost, h->stream));
  SPH_CUDA(h, cudaStreamSynchronize(h->stream));
  std::vector<uint32_t> ku(N), pu(N);
  SPH_CUDA(h, cudaMemcpyAsync(ku.data(), h->S.key, 4 * N, cudaMemcpyDeviceToHost, h->stream));
  SPH_CUDA(h, cudaMemcpyAsync(pu.data(), h->S.pid[1 - c.buf], 4 * N, cudaMemcpyDeviceToHost, h->stream));
  if (sorted_ids) SPH_CUDA(h, cudaMemcpyAsync(sorted_ids, h->S.pid[c.buf], 4 * N, cudaMemcpyDeviceToHost, h->stream));
  SPH_CUDA(h, cudaStreamSynchronize(h->stream));
  if (key_by_id)
    for (size_t i = 0; i < N; ++i) key_by_id[pu[i]] = ku[i];
  return SPH_OK;
}

sph_status sph_get_grid(sph_handle* h, sph_grid_info* out) {
  if (!h || !out) return SPH_ERR_INVALID_ARG;
  memset(out, 0, sizeof *out);
  out->n_levels = h->hg.n_levels;
  out->dim = h->dim;
  for (int k = 0; k < 3; ++k) out->lo[k] = h->dom.lo[k];
  out->h0 = h->hg.h0;
  out->lip_h = h->lip_h;
  for (int l = 0; l < h->hg.n_levels; ++l) {
    out->cell[l] = h->hg.cell[l];
    out->dims[l][0] = h->hg.nx[l];
    out->dims[l][1] = h->hg.ny[l];
    out->dims[l][2] = h->hg.nz[l];
  }
  for (int l = 0; l <= h->hg.n_levels; ++l) out->base[l] = h->hg.base[l];
  return SPH_OK;
}

sph_status sph_sync(sph_handle* h) {
  if (!h) return SPH_ERR_INVALID_ARG;
  int flags = 0;
  SPH_TRY(read_flags(h, &flags));
  return status_from_flags(h, flags);
}

// checkpoint layout: header (8 x int64: magic, version, n, dim, steps, 0, 0, 0),
// 2 doubles (t0, t1), n*dim doubles (positions), n bytes (colours)
static const int64_t kMagic = 0x3148534D48505300LL;

sph_status sph_save(sph_handle* h, void* buf, size_t* nbytes) {
  if (!h || !nbytes) return SPH_ERR_INVALID_ARG;
  const size_t N = (size_t)h->n, d = (size_t)h->dim;
  const size_t need = 8 * 8 + 2 * 8 + 8 * N * d + N;
  if (!buf) {
    *nbytes = need;
    return SPH_OK;
  }
  if (*nbytes < need) return fail(h, SPH_ERR_INVALID_ARG, "checkpoint buffer too small");
  int64_t hdr[8] = {kMagic, 1, (int64_t)N, (int64_t)d, h->steps, 0, 0, 0};
  double sched[2] = {h->t0, h->t1};
  uint8_t* p = (uint8_t*)buf;
  memcpy(p, hdr, sizeof hdr);
  memcpy(p + 64, sched, sizeof sched);
  SPH_TRY(sph_get_positions(h, (double*)(p + 80), 0));
  SPH_TRY(sph_get_colors(h, p + 80 + 8 * N * d, 0));
  *nbytes = need;
  return SPH_OK;
}

sph_status sph_load(sph_handle* h, const void* buf, size_t nbytes) {
  if (!h || !buf || nbytes < 80) return fail(h, SPH_ERR_INVALID_ARG, "bad checkpoint");
  int64_t hdr[8];
  double sched[2];
  memcpy(hdr, buf, sizeof hdr);
  memcpy(sched, (const uint8_t*)buf + 64, sizeof sched);
  const size_t N = (size_t)h->n, d = (size_t)h->dim;
  if (hdr[0] != kMagic || hdr[1] != 1 || hdr[2] != (int64_t)N || hdr[3] != (int64_t)d ||
      nbytes < 80 + 8 * N * d + N)
    return fail(h, SPH_ERR_INVALID_ARG, "checkpoint does not match this handle");
  const uint8_t* p = (const uint8_t*)buf;
  SPH_TRY(sph_set_state(h, (const double*)(p + 80), p + 80 + 8 * N * d, 0));
  h->steps = hdr[4];
  h->t0 = sched[0];
  h->t1 = sched[1];
  return write_ctl_sched(h);
}

sph_status sph_backward(sph_handle* h, int32_t K, const sph_objective* obj, const double* seed,
                        const double* dt_in, double* dt_out, double* dpos0, int32_t on_device, sph_grad* grad) {
  if (!h || !obj || !grad || (h->n > 0 && !dpos0)) return fail(h, SPH_ERR_INVALID_ARG, "null argument");
  if (K < 0 || obj->ckpt_every < 1) return fail(h, SPH_ERR_INVALID_ARG, "K < 0 or ckpt_every < 1");
  if (dt_in && !obj->frozen_dt) return fail(h, SPH_ERR_INVALID_ARG, "dt_in needs frozen_dt = 1");
  if (h->bg_grid_shape)
    return fail(h, SPH_ERR_INVALID_ARG, "the reverse pass covers analytic shapes only (no background level set)");
  if (h->has_surface)
    return fail(h, SPH_ERR_INVALID_ARG, "the reverse pass covers normal particles only (no feature-surface particles)");
  memset(grad, 0, sizeof *grad);
  const size_t N = (size_t)h->n, d = (size_t)h->dim, nd = N * d;
  const int64_t t0 = h->steps;
  if (N == 0) {
    h->steps += K;
    return write_ctl_sched(h);
  }
  SPH_TRY(ensure_adj(h));
  auto& a = h->adj;
  const int c = obj->ckpt_every;
  const int nck = K > 0 ? (K + c - 1) / c : 0;
  const size_t nseg = (size_t)std::min(c, std::max(K, 1));
  // device scratch (kept by the handle, grown on demand): checkpoints, x_K,
  // step sizes, a host-side seed
  if ((size_t)std::max(nck, 1) > a.ck_n) {
    SPH_TRY(grab(h, a.ck, nd * (size_t)std::max(nck, 1)));
    a.ck_n = (size_t)std::max(nck, 1);
  }
  if (!a.xk) {
    SPH_TRY(grab(h, a.xk, nd));
    SPH_TRY(grab(h, a.seed, nd));
  }
  if ((size_t)std::max(K, 1) > a.dts_n) {
    SPH_TRY(grab(h, a.dts, 2 * (size_t)std::max(K, 1)));
    a.dts_n = (size_t)std::max(K, 1);
  }
  double* ck = a.ck;
  double* xk = a.xk;
  double* dts = a.dts;
  const double* seed_d = seed;
  if (seed && !on_device) {
    SPH_CUDA(h, cudaMemcpyAsync(a.seed, seed, sizeof(double) * nd, cudaMemcpyHostToDevice, h->stream));
    seed_d = a.seed;
  }
  if (dt_in) {
    SPH_CUDA(h, cudaMemcpyAsync(dts, dt_in, sizeof(double) * 2 * (size_t)K,
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
  }
  SPH_CUDA(h, cudaMemsetAsync(h->S.err, 0, sizeof(int), h->stream));
  SPH_CUDA(h, cudaMemsetAsync(a.acc, 0, sizeof(double) * kAdjSlots, h->stream));
  if (launch_get_colors(h->S, a.col, h->stream) != cudaSuccess) return fail(h, SPH_ERR_CUDA, "colours");
  // The step sizes of this run go through a history the control block names:
  // every step of the forward run records the sizes it chose (or, with dt_in,
  // replays the prescribed ones), and every re-run step replays them; no
  // per-step copies. The history is switched off whichever way this returns.
  struct HistOff {
    sph_handle* h;
    ~HistOff() {
      if (h->dt_mode) {
        h->dt_mode = 0;
        h->dt_hist = nullptr;
        h->dt_len = 0;
        write_ctl_hist(h);
      }
    }
  } hist_off{h};
  h->dt_hist = dts;
  h->dt_base = t0;
  h->dt_len = K;
  h->dt_mode = dt_in ? 2 : 1;
  SPH_TRY(write_ctl_hist(h));
  // Forward run with a position checkpoint at the start of every segment. The
  // last segment is taped on the way; every other segment is re-run from its
  // checkpoint (with the recorded sizes) into the tape just before its
  // reverse sweep.
  SPH_TRY(ensure_tape(h, (int)nseg));
  const std::vector<DevState>& tape = h->adj.tape;
  const int last0 = nck > 0 ? (nck - 1) * c : 0;
  for (int s = 0; s < K; ++s) {
    if (s % c == 0) SPH_TRY(positions_to(h, ck + nd * (size_t)(s / c)));
    if (s >= last0) {
      // the graph of a taped step into slot k, shared with the re-runs (the
      // step-size history mode is read from the control block at run time)
      const int k = s - last0;
      if (!a.g_rerun[k])
        SPH_TRY(capture(h, &a.g_rerun[k], [&] { return taped_step(h, tape[k], nullptr, nullptr); }));
      SPH_CUDA(h, cudaGraphLaunch(a.g_rerun[k], h->stream));
    } else {
      SPH_TRY(ensure_graph(h, 0));  // the handle's graph of one step
      SPH_CUDA(h, cudaGraphLaunch(h->gexec, h->stream));
    }
    h->steps += 1;
  }
  h->dt_mode = 2;  // from here on every step replays the recorded sizes
  SPH_TRY(positions_to(h, xk));
  // objective at x_K: the gradient seed (g[cur])
  int cur = 0;
  SPH_TRY(reverse_setup(h, false, nullptr));
  SPH_TRY(run_objective(h, obj->density_weight, obj->lambda, seed_d, a.g[cur]));
  // reverse sweep, segment by segment; every re-run step and every reverse
  // step is one replay of a graph cached per tape slot (the buffers are fixed)
  const int fz = obj->frozen_dt ? 1 : 0;
  for (int seg = nck - 1; seg >= 0; --seg) {
    const int s0 = seg * c, s1 = std::min(K, s0 + c);
    if (seg != nck - 1) {
      SPH_TRY(set_state_at(h, ck + nd * (size_t)seg, a.col, t0 + s0));  // control block: replay
      for (int s = s0; s < s1; ++s) {
        const int k = s - s0;
        if (!a.g_rerun[k])
          SPH_TRY(capture(h, &a.g_rerun[k], [&] { return taped_step(h, tape[k], nullptr, nullptr); }));
        SPH_CUDA(h, cudaGraphLaunch(a.g_rerun[k], h->stream));
      }
    }
    for (int s = s1 - 1; s >= s0; --s) {
      const int k = s - s0;
      cudaGraphExec_t& g = a.g_rev[fz][cur][k];
      if (!g) SPH_TRY(capture(h, &g, [&] { return run_bwd_step(h, tape[k], a.g[cur], a.g[1 - cur], !fz); }));
      SPH_CUDA(h, cudaGraphLaunch(g, h->stream));
      cur = 1 - cur;
    }
  }
  // results
  double acc[kAdjSlots];
  SPH_CUDA(h, cudaMemcpyAsync(acc, a.acc, sizeof acc, cudaMemcpyDeviceToHost, h->stream));
  if (on_device) {
    SPH_CUDA(h, cudaMemcpyAsync(dpos0, a.g[cur], sizeof(double) * nd, cudaMemcpyDeviceToDevice, h->stream));
    if (dt_out && K > 0)
      SPH_CUDA(h, cudaMemcpyAsync(dt_out, dts, sizeof(double) * 2 * (size_t)K, cudaMemcpyDeviceToDevice, h->stream));
  } else {
    SPH_CUDA(h, cudaMemcpyAsync(dpos0, a.g[cur], sizeof(double) * nd, cudaMemcpyDeviceToHost, h->stream));
    if (dt_out && K > 0)
      SPH_CUDA(h, cudaMemcpyAsync(dt_out, dts, sizeof(double) * 2 * (size_t)K, cudaMemcpyDeviceToHost, h->stream));
  }
  // leave the handle at x_K (history off)
  h->dt_mode = 0;
  h->dt_hist = nullptr;
  h->dt_len = 0;
  SPH_TRY(set_state_at(h, xk, a.col, t0 + K));
  SPH_CUDA(h, cudaStreamSynchronize(h->stream));
  grad->L = acc[kAdjL];
  grad->d_sigma0 = acc[kAdjSigma0];
  grad->d_gamma = acc[kAdjGamma];
  grad->d_P0 = acc[kAdjP0];
  for (int m = 0; m < 8; ++m) grad->d_poly[m] = acc[kAdjPoly + m];
  int flags = 0;
  SPH_TRY(read_flags(h, &flags));
  return status_from_flags(h, flags);
}

// ================================================================ batch ==
// Many independent instances stepped by one CUDA graph per step. Instance k's
// step (its 12 kernels, predicated on its own list-rebuild flag) sits on
// branch b(k) of the graph; the branches fork from and join to the batch's
// stream, so instances on different branches run concurrently and fill the
// SMs that one small instance leaves idle. Instances are dealt to branches
// longest first onto the least-loaded branch (load = particles x dimension
// cost); the branch count is the autotuned parameter.
}  // extern "C"

struct sph_batch {
  std::vector<sph_handle*> inst;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<cudaStream_t> branch;
  std::vector<cudaEvent_t> ev;  // [0]: fork, [1 + b]: join of branch b
  cudaGraphExec_t gexec = nullptr;
  int n_branches = 0;
  std::vector<float> tuned_ms;  // per trial of the autotuner: its branch count and ms per step
  std::vector<int> tuned_b;
  std::vector<sph_batch_trial> trials;  // every trial with its full configuration
  sph_batch_trial chosen{};
  std::string err;
};

namespace {

double inst_cost(const sph_handle* h) { return (double)h->n * (h->dim == 3 ? 2.5 : 1.0); }

sph_status batch_fail(sph_batch* b, sph_status s, const std::string& m) {
  b->err = m;
  return s;
}

void batch_drop_graph(sph_batch* b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  b->gexec = nullptr;
}

// capture one step of every instance into a graph with nb branches
sph_status batch_capture(sph_batch* b, int nb) {
  batch_drop_graph(b);
  while ((int)b->branch.size() < nb) {
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
      return batch_fail(b, SPH_ERR_CUDA, "stream creation failed");
    b->branch.push_back(s);
  }
  while ((int)b->ev.size() < nb + 1) {
    cudaEvent_t e;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
      return batch_fail(b, SPH_ERR_CUDA, "event creation failed");
    b->ev.push_back(e);
  }
  // longest-first onto the least-loaded branch
  std::vector<int> order(b->inst.size());
  for (size_t k = 0; k < order.size(); ++k) order[k] = (int)k;
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return inst_cost(b->inst[x]) > inst_cost(b->inst[y]); });
  std::vector<double> load(nb, 0.0);
  std::vector<int> where(b->inst.size(), 0);
  for (int k : order) {
    int best = 0;
    for (int q = 1; q < nb; ++q)
      if (load[q] < load[best]) best = q;
    where[k] = best;
    load[best] += inst_cost(b->inst[k]);
  }
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return batch_fail(b, SPH_ERR_CUDA, "begin capture");
  sph_status st = SPH_OK;
  if (cudaEventRecord(b->ev[0], b->stream) != cudaSuccess) st = SPH_ERR_CUDA;
  for (int q = 0; q < nb && st == SPH_OK; ++q)
    if (cudaStreamWaitEvent(b->branch[q], b->ev[0], 0) != cudaSuccess) st = SPH_ERR_CUDA;
  // each branch issues its instances in submission order
  for (size_t k = 0; k < order.size() && st == SPH_OK; ++k) {
    sph_handle* h = b->inst[order[k]];
    cudaStream_t keep = h->stream;
    h->stream = b->branch[where[order[k]]];
    st = launch_step(h, h->par.record_fields ? 1 : 0);
    h->stream = keep;
  }
  for (int q = 0; q < nb && st == SPH_OK; ++q) {
    if (cudaEventRecord(b->ev[1 + q], b->branch[q]) != cudaSuccess ||
        cudaStreamWaitEvent(b->stream, b->ev[1 + q], 0) != cudaSuccess)
      st = SPH_ERR_CUDA;
  }
  e = cudaStreamEndCapture(b->stream, &g);
  if (st != SPH_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return batch_fail(b, SPH_ERR_CUDA, "capture of the batched step failed");
  }
  e = cudaGraphInstantiate(&b->gexec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return batch_fail(b, SPH_ERR_CUDA, "graph instantiation failed");
  b->n_branches = nb;
  return SPH_OK;
}

}  // namespace

extern "C" {

sph_status sph_batch_create(const sph_instance_desc* descs, int32_t n_inst, const sph_alloc* alloc, void* stream,
                            int32_t n_branches, sph_batch** out) {
  if (!out || !descs || n_inst <= 0 || n_branches < 0) return SPH_ERR_INVALID_ARG;
  *out = nullptr;
  sph_batch* b = new sph_batch();
  b->stream = (cudaStream_t)stream;
  if (!b->stream) {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete b;
      return SPH_ERR_CUDA;
    }
    b->own_stream = true;
  }
  for (int k = 0; k < n_inst; ++k) {
    sph_handle* h = nullptr;
    sph_params par = descs[k].params;
    par.use_graph = 0;
    sph_status s = sph_create(&descs[k].dom, &descs[k].field, descs[k].n_particles, descs[k].n_colors, &par, alloc,
                              b->stream, &h);
    if (s != SPH_OK) {
      fprintf(stderr, "sph_batch_create: instance %d failed\n", k);
      sph_batch_destroy(b);
      return s;
    }
    b->inst.push_back(h);
  }
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) {
    sph_batch_destroy(b);
    return SPH_ERR_CUDA;
  }
  if (n_branches > 0) {
    sph_status s = batch_capture(b, std::min<int>(n_branches, n_inst));
    if (s != SPH_OK) {
      fprintf(stderr, "sph_batch_create: %s\n", b->err.c_str());
      sph_batch_destroy(b);
      return s;
    }
  }
  *out = b;
  return SPH_OK;
}

sph_status sph_batch_tune(sph_batch* b, const int32_t* candidates, int32_t n_candidates, int32_t steps_each) {
  if (!b || !candidates || n_candidates <= 0 || steps_each <= 0) return SPH_ERR_INVALID_ARG;
  // Every trial starts from the same state (so each sees the same steps and
  // list rebuilds) and the state is put back afterwards.
  std::vector<std::unique_ptr<Temp>> saved, cols;
  std::vector<int64_t> steps0;
  for (sph_handle* h : b->inst) {
    saved.emplace_back(new Temp(h, sizeof(double) * (size_t)h->n * (size_t)h->dim));
    cols.emplace_back(new Temp(h, (size_t)h->n));
    steps0.push_back(h->steps);
    if (h->n > 0) {
      if (!saved.back()->p || !cols.back()->p) return batch_fail(b, SPH_ERR_OOM, "tuning snapshot allocation failed");
      sph_status s = positions_to(h, (double*)saved.back()->p);
      if (s != SPH_OK) return s;
      if (launch_get_colors(h->S, (uint8_t*)cols.back()->p, h->stream) != cudaSuccess)
        return batch_fail(b, SPH_ERR_CUDA, "tuning snapshot");
    }
  }
  auto restore = [&]() -> sph_status {
    for (size_t k = 0; k < b->inst.size(); ++k) {
      sph_handle* h = b->inst[k];
      if (h->n == 0) continue;
      sph_status s = set_state_at(h, (const double*)saved[k]->p, (const uint8_t*)cols[k]->p, steps0[k]);
      if (s != SPH_OK) return s;
    }
    return SPH_OK;
  };
  // the same launch configuration on every instance
  auto configure = [&](const sph_batch_trial& c) -> sph_status {
    for (sph_handle* h : b->inst) {
      sph_status s = sph_set_tuning(h, c.pass_threads, c.cell_factor, h->S.fp64 ? -1 : c.stage_views);
      if (s != SPH_OK) return s;
    }
    return SPH_OK;
  };
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  b->tuned_b.clear();
  b->tuned_ms.clear();
  b->trials.clear();
  // one trial: configure, capture, restore, a warm-up step (it rebuilds
  // every list), then steps_each timed graph launches
  auto trial = [&](sph_batch_trial c, float* ms_out) -> sph_status {
    sph_status st = configure(c);
    if (st == SPH_OK) st = batch_capture(b, c.branches);
    if (st == SPH_OK) st = restore();
    if (st != SPH_OK) return st;
    cudaGraphLaunch(b->gexec, b->stream);
    cudaEventRecord(e0, b->stream);
    for (int s = 0; s < steps_each; ++s) cudaGraphLaunch(b->gexec, b->stream);
    cudaEventRecord(e1, b->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) return batch_fail(b, SPH_ERR_CUDA, "tuning run failed");
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= (float)steps_each;
    c.ms_per_step = ms;
    b->trials.push_back(c);
    b->tuned_b.push_back(c.branches);
    b->tuned_ms.push_back(ms);
    *ms_out = ms;
    return SPH_OK;
  };
  sph_handle* h0 = b->inst[0];
  sph_batch_trial best{};
  best.branches = 0;
  best.pass_threads = h0->S.pass_threads;
  best.cell_factor = h0->par.cell_factor > 0 ? h0->par.cell_factor : 1.0;
  best.stage_views = h0->S.stage;
  float best_ms = 0.0f;
  sph_status st = SPH_OK;
  // 1. branch count
  for (int c = 0; c < n_candidates && st == SPH_OK; ++c) {
    sph_batch_trial t = best;
    t.branches = std::max(1, std::min<int>(candidates[c], (int)b->inst.size()));
    float ms = 0.0f;
    st = trial(t, &ms);
    if (st == SPH_OK && (best.branches == 0 || ms < best_ms)) {
      best = t;
      best_ms = ms;
    }
  }
  // 2. then, one knob at a time from the best so far: threads per block of
  // the pair passes, cell factor
  const int threads_alt[] = {128, 256};
  const double cf_alt[] = {0.75, 1.0, 1.5};
  const int threads0 = best.pass_threads;
  const double cf0 = best.cell_factor;
  for (int v : threads_alt) {
    if (st != SPH_OK || v == threads0) continue;
    sph_batch_trial t = best;
    t.pass_threads = v;
    float ms = 0.0f;
    st = trial(t, &ms);
    if (st == SPH_OK && ms < best_ms) { best = t; best_ms = ms; }
  }
  for (double v : cf_alt) {
    if (st != SPH_OK || v == cf0) continue;
    sph_batch_trial t = best;
    t.cell_factor = v;
    float ms = 0.0f;
    st = trial(t, &ms);
    if (st == SPH_OK && ms < best_ms) { best = t; best_ms = ms; }
  }
  // 3. the staged pass A on or off (FP32 instances)
  const int stage0 = best.stage_views;
  if (st == SPH_OK) {
    sph_batch_trial t = best;
    t.stage_views = stage0 ? 0 : 1;
    float ms = 0.0f;
    st = trial(t, &ms);
    if (st == SPH_OK && ms < best_ms) { best = t; best_ms = ms; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st == SPH_OK) st = configure(best);
  if (st == SPH_OK) st = restore();
  saved.clear();
  cols.clear();
  if (st != SPH_OK) return st;
  best.ms_per_step = best_ms;
  b->chosen = best;
  st = batch_capture(b, best.branches);
  if (st != SPH_OK) return st;
  return cudaStreamSynchronize(b->stream) == cudaSuccess ? SPH_OK : SPH_ERR_CUDA;
}

sph_status sph_batch_tuning(const sph_batch* b, sph_batch_trial* chosen, sph_batch_trial* trials, int32_t cap,
                            int32_t* n_trials) {
  if (!b) return SPH_ERR_INVALID_ARG;
  if (chosen) *chosen = b->chosen;
  const int nt = (int)b->trials.size();
  if (n_trials) *n_trials = nt;
  for (int q = 0; trials && q < nt && q < cap; ++q) trials[q] = b->trials[q];
  return SPH_OK;
}

sph_status sph_batch_step(sph_batch* b, int32_t n_steps) {
  if (!b || n_steps < 0) return SPH_ERR_INVALID_ARG;
  if (!b->gexec) {
    sph_status s = batch_capture(b, std::min<int>(16, (int)b->inst.size()));
    if (s != SPH_OK) return s;
  }
  for (int s = 0; s < n_steps; ++s)
    if (cudaGraphLaunch(b->gexec, b->stream) != cudaSuccess) return batch_fail(b, SPH_ERR_CUDA, "graph launch");
  for (sph_handle* h : b->inst) {
    h->steps += n_steps;
    h->recorded = h->par.record_fields != 0;
    h->rho_valid = h->rho_valid || n_steps > 0;
  }
  return SPH_OK;
}

sph_status sph_batch_step_each(sph_batch* b, int32_t n_steps) {
  if (!b || n_steps < 0) return SPH_ERR_INVALID_ARG;
  for (sph_handle* h : b->inst) {
    sph_status s = ensure_graph(h, h->par.record_fields ? 1 : 0);
    if (s != SPH_OK) return s;
  }
  for (int s = 0; s < n_steps; ++s)
    for (sph_handle* h : b->inst)
      if (h->n > 0 && cudaGraphLaunch(h->gexec, h->stream) != cudaSuccess)
        return batch_fail(b, SPH_ERR_CUDA, "graph launch");
  for (sph_handle* h : b->inst) {
    h->steps += n_steps;
    h->recorded = h->par.record_fields != 0;
    h->rho_valid = h->rho_valid || n_steps > 0;
  }
  return SPH_OK;
}

sph_status sph_batch_get(sph_batch* b, int32_t k, sph_handle** h) {
  if (!b || !h || k < 0 || k >= (int)b->inst.size()) return SPH_ERR_INVALID_ARG;
  *h = b->inst[k];
  return SPH_OK;
}

sph_status sph_batch_info(const sph_batch* b, int32_t* n_inst, int32_t* n_branches, int32_t* n_tuned,
                          int32_t* tuned_branches, float* tuned_ms) {
  if (!b) return SPH_ERR_INVALID_ARG;
  if (n_inst) *n_inst = (int32_t)b->inst.size();
  if (n_branches) *n_branches = b->n_branches;
  if (n_tuned) *n_tuned = (int32_t)b->tuned_b.size();
  for (size_t q = 0; q < b->tuned_b.size(); ++q) {
    if (tuned_branches) tuned_branches[q] = b->tuned_b[q];
    if (tuned_ms) tuned_ms[q] = b->tuned_ms[q];
  }
  return SPH_OK;
}

sph_status sph_batch_sync(sph_batch* b) {
  if (!b) return SPH_ERR_INVALID_ARG;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return batch_fail(b, SPH_ERR_CUDA, "sync");
  for (sph_handle* h : b->inst) {
    int flags = 0;
    sph_status s = read_flags(h, &flags);
    if (s != SPH_OK) return s;
    s = status_from_flags(h, flags);
    if (s != SPH_OK) return s;
  }
  return SPH_OK;
}

const char* sph_batch_last_error(const sph_batch* b) { return b ? b->err.c_str() : "null batch"; }

void sph_batch_destroy(sph_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  batch_drop_graph(b);
  for (sph_handle* h : b->inst) sph_destroy(h);
  for (cudaStream_t s : b->branch) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
}

const char* sph_last_error(const sph_handle* h) { return h ? h->err.c_str() : "null handle"; }

sph_status sph_get_info(const sph_handle* h, int64_t* n, int32_t* dim, double* rho_scale) {
  if (!h) return SPH_ERR_INVALID_ARG;
  if (n) *n = h->n;
  if (dim) *dim = h->dim;
  if (rho_scale) *rho_scale = h->rho_scale;
  return SPH_OK;
}

void sph_destroy(sph_handle* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  for (auto* v : {&h->adj.g_rerun, &h->adj.g_rev[0][0], &h->adj.g_rev[0][1], &h->adj.g_rev[1][0],
                  &h->adj.g_rev[1][1]})
    for (cudaGraphExec_t g : *v)
      if (g) cudaGraphExecDestroy(g);
  for (auto& b : h->blocks) h->alloc.free(b.first, b.second, h->alloc.ctx);
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->own_stream) cudaStreamDestroy(h->stream);
  delete h;
}

}  // extern "C"
