// Internal interface between the C-ABI host code and the kernel translation
// units. Not part of the public boundary (include/sphmesh.h).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "sph_device.cuh"

namespace sph {

// Raw device pointers of one relaxation instance. The particle state (integer
// positions, colours, ids) is double-buffered: ctl->buf names the buffer that
// holds it in the current (cell-sorted at the last list build) order; the list
// rebuild gathers it into the other buffer. Views are double-buffered by
// ctl->vp (pass B writes the next step's views while pass A/B read the current).
struct DevState {
  int n = 0, dim = 2, fp64 = 0, cap = 0;
  int pass_threads = 256;  // threads per block of the pair passes (128 or 256)
  void* X[2] = {nullptr, nullptr};       // int64 x, y, z (+ pad) per particle
  uint32_t* meta[2] = {nullptr, nullptr};  // colour
  uint32_t* pid[2] = {nullptr, nullptr};   // particle id
  void* view[2] = {nullptr, nullptr};    // int4 (FP32) or double4 (FP64)
  void* vbuild = nullptr;                // view at the list build, w = half skin
  void* view32 = nullptr;                // FP64 path: FP32 view (list build; pass A's screen)
  uint32_t* key = nullptr;               // cell key (old order, rebuild only)
  uint32_t* tmp = nullptr;               // scatter slots
  uint32_t* cnt = nullptr;               // per-cell counters (all zero between rebuilds)
  uint32_t* cstart = nullptr;            // exclusive prefix of cell counts, total+1 entries
  uint32_t* scan_part = nullptr;
  uint32_t total_cells = 0;
  uint32_t* list = nullptr;              // cap x n entries (j << 8 | colour_j), column per particle
  uint32_t* lcount = nullptr;            // entries per particle; bit 31: FP32 coarse test exact
  uint32_t* plist = nullptr;             // cap x n: the force pairs of the current step (pass A -> B)
  // staged pass A (FP32, 256-thread pair passes): per 256-target block its
  // distinct neighbours sj (kStageCap per block), their count scount (-1: not
  // staged) and the list again with ranks in that set (llist, cap x n)
  int stage = 0;
  uint32_t* llist = nullptr;
  int* scount = nullptr;
  int* sj = nullptr;
  uint32_t* pcount = nullptr;
  void* acc4 = nullptr;   // V4<T>: a_n and g = 0.05 rho_t r_c |a|
  void* rho = nullptr;    // T
  void* visc = nullptr;   // V4<T>: a~ (recorded steps only)
  void* pc = nullptr;     // T: p/rho^2 (general EOS only)
  Partial* partials = nullptr;
  Scalars* scal = nullptr;
  StepCtl* ctl = nullptr;
  unsigned* tickets = nullptr;
  int* err = nullptr;
  int* dbg_count = nullptr;        // 2n: density / force set sizes by particle id
  long long* dbg_sum = nullptr;    // 2n: sums of member ids
};

// per-step gate: flip the view buffer; start a list rebuild (flip the state
// buffer) when pass B asked for one or `force` is set
cudaError_t launch_gate(const DevState& S, int force, cudaStream_t st);
// the next step rebuilds the list (after set-up or a diagnostic evaluation)
cudaError_t launch_request_rebuild(const DevState& S, cudaStream_t st);
// overwrite the control block (a kernel: no host synchronisation)
cudaError_t launch_write_ctl(const DevState& S, const StepCtl& v, cudaStream_t st);
// cell list of the old order -> gather into the new order (predicated on ctl->rebuild)
cudaError_t build_cells(const DevState& S, cudaStream_t st);
// colours by particle id
cudaError_t launch_set_surface(const DevState& S, const uint8_t* flags, cudaStream_t st);
cudaError_t launch_get_colors(const DevState& S, uint8_t* out, cudaStream_t st);

// streaming multiprocessors of the current device (cached once per process)
inline int device_sms() {
  static const int sms = [] {
    int d = 0, v = 0;
    if (cudaGetDevice(&d) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d) != cudaSuccess)
      return 152;
    return v > 0 ? v : 152;
  }();
  return sms;
}
// Grid of a predicated list-rebuild kernel: grid-stride over n with at most
// per_sm blocks per SM. Most steps do not rebuild, and such a kernel then
// exits at once: with one block per 256 particles an 8M-particle grid took
// about 19 us to launch and retire its 32,768 blocks, a capped grid a few.
inline int rebuild_grid(int n, int tb, int per_sm) {
  const int g = (n + tb - 1) / tb, cap = device_sms() * per_sm;
  return g < 1 ? 1 : (g < cap ? g : cap);
}

struct PassFlags {
  int general_eos = 0;  // gamma != 2: density pass first, pressure p/rho^2
  int record = 0;       // keep rho and a~ for output
  int nbr_debug = 0;    // write neighbour-set sizes and id sums by particle id
  int advance = 1;      // count this pass as a step (sigma schedule, counter)
  int move = 1;         // pass B: integrate (0: only a~, for the reverse pass)
  const double* dt_fix = nullptr;  // pass A: prescribed {dt1, dt2} (device)
  double* dt_rec = nullptr;        // pass A: record {dt1, dt2} (device)
  const void* geo = nullptr;       // pass A: the Geom<T> of the handle (feature-surface normals)
  int surface = 0;                 // pass A: feature-surface particles may be flagged
  const Frame<float>* f32 = nullptr;  // FP64 path: frame of its FP32 views (view32), kept current
                                      // by pass B and screened on by pass A
};

template <int D, class T>
cudaError_t launch_rebuild(const DevState& S, const Grid<T>& G, const Frame<T>& F, const Geom<T>& g, T kappa,
                           cudaStream_t st, const Grid<float>* G32 = nullptr, const Frame<float>* F32 = nullptr);
template <int D, class T>
cudaError_t launch_pass_a(const DevState& S, const Frame<T>& F, const Phys<T>& P, PassFlags f, cudaStream_t st);
// the staged pass A wants the largest shared-memory carveout (5 blocks of
// 256 threads with 40 KB of staged views each); once per process
template <int D>
cudaError_t prepare_staged_pass();
// whether pass A runs staged for these flags (the variant exists for FP32,
// gamma = 2, no feature-surface particles, no neighbour diagnostics, 256 threads)
inline bool staged_pass(const DevState& S, const PassFlags& f) {
  return S.stage && !S.fp64 && S.pass_threads == 256 && !f.general_eos && !f.nbr_debug && !f.surface;
}
template <int D, class T>
cudaError_t launch_pass_b(const DevState& S, const Frame<T>& F, const Phys<T>& P, const Geom<T>& g, PassFlags f,
                          cudaStream_t st);
template <int D, class T>
cudaError_t launch_set_state(const DevState& S, const Frame<T>& F, const double* xyz, const uint8_t* col,
                             cudaStream_t st);
template <int D, class T>
cudaError_t launch_get_positions(const DevState& S, const Frame<T>& F, double* out, cudaStream_t st);
template <int D, class T>
cudaError_t launch_get_fields(const DevState& S, int which, double* out, cudaStream_t st);

// accumulated results (double slots of AdjBufs::acc)
enum AdjSlot : int {
  kAdjL = 0,       // objective value
  kAdjSigma0 = 1,  // dL/dsigma0
  kAdjGamma = 2,
  kAdjP0 = 3,
  kAdjPoly = 4,    // 8 slots: dL/dpoly[m]
  kAdjDt1b = 12,   // per step: adjoint of dt1 (reset by k_bwd_out)
  kAdjDt2b = 13,   // per step: adjoint of dt2
  kAdjMbar = 14,   // per step: adjoint of m = min r_c/|a|
  kAdjSlots = 16
};
constexpr int kAdjPartials = 12;  // doubles per block partial

template <class T>
struct AdjBufs {
  const double* gin = nullptr;  // n x D by id: adjoint of the state the step produced (or the seed)
  double* gout = nullptr;       // n x D by id: adjoint of the state it started from
  V4<double>* xb = nullptr;     // current order: adjoint of x (accumulating)
  V4<T>* atb = nullptr;         // adjoint of a~
  V4<T>* ab = nullptr;          // adjoint of a
  T* hb = nullptr;              // adjoint of h
  T* Tb = nullptr;              // adjoint of T = 1/rho_t^2
  T* rtb = nullptr;             // adjoint of rho_t
  T* rhob = nullptr;            // adjoint of rho
  double* part = nullptr;       // kAdjPartials per block
  double* acc = nullptr;        // kAdjSlots
  unsigned* ticket = nullptr;
};

// reverse pass of one step whose state, lists and forward quantities (a tape
// slot) are in S; B.gin -> B.gout
template <int D, class T>
cudaError_t launch_bwd_step(const DevState& S, const Frame<T>& F, const Phys<T>& P, const Geom<T>& geo,
                            const AdjBufs<T>& B, int recomputed_dt, int general_eos, cudaStream_t st);
// objective at the current state (list in place) and its gradient -> B.gout;
// B.gin (may be null) is an extra seed added to dL/dx
template <int D, class T>
cudaError_t launch_objective(const DevState& S, const Frame<T>& F, const Phys<T>& P, const Geom<T>& geo,
                             const AdjBufs<T>& B, double wd, double lambda, cudaStream_t st);

// copy the state pass A used (current order: X, meta, pid, view), ctl and
// scal into tape.X[0], meta[0], pid[0], view[0], ctl, scal
template <int D, class T>
cudaError_t launch_tape_snapshot(const DevState& S, const DevState& tape, cudaStream_t st);

// per-colour volume sum m/rho and particle count over the current order (rho
// of the last pass A); vpart/cpart hold color_volume_blocks(n) x 256 partials,
// vol/cnt 256 results (device)
int color_volume_blocks(int n);
template <class T>
cudaError_t launch_color_volumes(const DevState& S, double* vpart, unsigned long long* cpart, double* vol,
                                 long long* cnt, cudaStream_t st);

// initial sampling (create)
struct FieldBounds {
  double sum_w, min_seff, max_seff, max_w;
};
template <int D>
cudaError_t field_bounds(const Geom<double>& g, int res, FieldBounds* host_out, double* scratch,
                         cudaStream_t st);
int field_bounds_scratch_doubles();
template <int D>
cudaError_t sample_positions(const Geom<double>& g, int n, int n_colors, uint64_t seed, double wmax,
                             double* xyz, uint8_t* col, double* gens, int* err, cudaStream_t st);

}  // namespace sph
