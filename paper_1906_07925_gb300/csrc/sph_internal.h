// Internal interface between the C-ABI host code and the kernel translation
// units. Not part of the public boundary (include/sphmesh.h).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "sph_device.cuh"

namespace sph {

// Raw device pointers of one relaxation instance. "_u" arrays hold the state
// in the order the previous step left it (the next sort's input); "_s" arrays
// hold the same records sorted by cell key (the neighbour loops' input).
struct DevState {
  int n = 0, dim = 2, fp64 = 0, block = 256;
  void* pos4_u = nullptr;  // V4<T>: offsets in the particle's cell + h
  void* pos4_s = nullptr;
  uint32_t* meta_u = nullptr;  // (x cell coordinate << 8) | colour
  uint32_t* meta_s = nullptr;
  uint32_t* key_u = nullptr;   // cell key (level base + linear cell id)
  uint32_t* key_s = nullptr;
  uint32_t* pid_u = nullptr;   // original particle id
  uint32_t* pid_s = nullptr;
  uint32_t* cnt = nullptr;     // per-cell counters (all zero between steps)
  uint32_t* cstart = nullptr;  // exclusive prefix of cell counts, total+1 entries
  uint32_t* tmp = nullptr;     // scatter slots
  uint32_t* scan_part = nullptr;
  uint32_t total_cells = 0;
  void* acc4 = nullptr;        // V4<T>: a_n and g = 0.05 rho_t r_c |a| (sorted order)
  void* rho = nullptr;         // T: density (sorted order)
  void* visc = nullptr;        // V4<T>: a~ (sorted order; recorded steps only)
  void* pc = nullptr;          // T: p/rho^2 (general EOS only)
  Partial* partials = nullptr;
  Scalars* scal = nullptr;
  StepCtl* ctl = nullptr;
  unsigned* tickets = nullptr;  // [0] pass A
  int* err = nullptr;
  int* dbg_count = nullptr;         // 2n: density / force set sizes by particle id
  long long* dbg_sum = nullptr;     // 2n: sums of member ids
};

// cell list: count -> scan -> scatter -> stable gather into the _s arrays
cudaError_t build_cells(const DevState& S, cudaStream_t st);

struct PassFlags {
  int general_eos = 0;  // gamma != 2: density pass first, pressure p/rho^2
  int record = 0;       // keep rho and a~ for output
  int nbr_debug = 0;    // write neighbour-set sizes and id sums by particle id
  int advance = 1;      // count this pass as a step (sigma schedule, counter)
};

template <int D, class T>
cudaError_t launch_pass_a(const DevState& S, const Grid<T>& G, const Phys<T>& P, PassFlags f,
                          cudaStream_t st);
template <int D, class T>
cudaError_t launch_pass_b(const DevState& S, const Grid<T>& G, const Phys<T>& P, const Geom<T>& g,
                          PassFlags f, cudaStream_t st);
template <int D, class T>
cudaError_t launch_set_state(const DevState& S, const Grid<T>& G, const Grid<double>& Gd,
                             const Geom<T>& g, const double* xyz, const uint8_t* col,
                             cudaStream_t st);
template <int D, class T>
cudaError_t launch_get_positions(const DevState& S, const Grid<double>& Gd, double* out,
                                 cudaStream_t st);
template <int D, class T>
cudaError_t launch_get_fields(const DevState& S, int which, double* out, cudaStream_t st);

// initial sampling (create)
struct FieldBounds {
  double sum_w, min_seff, max_seff, max_w;
};
template <int D>
cudaError_t field_bounds(const Geom<double>& g, int res, FieldBounds* host_out, double* scratch,
                         cudaStream_t st);
int field_bounds_scratch_doubles();
// colours by particle id from the "_u" arrays
cudaError_t launch_get_colors(const DevState& S, uint8_t* out, cudaStream_t st);
template <int D>
cudaError_t sample_positions(const Geom<double>& g, int n, int n_colors, uint64_t seed, double wmax,
                             double* xyz, uint8_t* col, double* gens, int* err, cudaStream_t st);

}  // namespace sph
