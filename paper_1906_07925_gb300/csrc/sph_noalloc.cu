// Allocation-free evaluation of the first pass of a relaxation step
// (sph_eval_forces_noalloc in include/sphmesh.h).
//
// For callers that cannot allocate device memory: every scratch buffer the
// cell sort, the neighbour list and pass A need lives in one file-scope device
// array of fixed size, carved into segments below. The kernels are the same
// ones the handle path launches; only the origin of their pointers differs.
#include <cstdio>
#include <mutex>

#include "sph_host.h"
#include "sph_internal.h"

using namespace sph;

namespace {

constexpr size_t kN = SPH_NOALLOC_MAX_PARTICLES;
constexpr size_t kC = SPH_NOALLOC_MAX_CELLS;
constexpr size_t kCap = 96;  // list entries per particle (exact neighbour sets, no skin)

constexpr size_t al(size_t x) { return (x + 255) & ~size_t(255); }

// segment offsets (bytes) inside the scratch array
constexpr size_t kX0 = 0;
constexpr size_t kX1 = kX0 + al(32 * kN);
constexpr size_t kM0 = kX1 + al(32 * kN);
constexpr size_t kM1 = kM0 + al(4 * kN);
constexpr size_t kP0 = kM1 + al(4 * kN);
constexpr size_t kP1 = kP0 + al(4 * kN);
constexpr size_t kV0 = kP1 + al(4 * kN);
constexpr size_t kV1 = kV0 + al(16 * kN);
constexpr size_t kVb = kV1 + al(16 * kN);
constexpr size_t kKey = kVb + al(16 * kN);
constexpr size_t kTmp = kKey + al(4 * kN);
constexpr size_t kList = kTmp + al(4 * kN);
constexpr size_t kLcount = kList + al(4 * kCap * kN);
constexpr size_t kPlist = kLcount + al(4 * kN);
constexpr size_t kPcount = kPlist + al(4 * kCap * kN);
constexpr size_t kAcc4 = kPcount + al(4 * kN);
constexpr size_t kRho = kAcc4 + al(16 * kN);
constexpr size_t kPc = kRho + al(4 * kN);
constexpr size_t kCnt = kPc + al(4 * kN);
constexpr size_t kCstart = kCnt + al(4 * kC);
constexpr size_t kScanPart = kCstart + al(4 * (kC + 1));
constexpr size_t kPartials = kScanPart + al(4 * (kC / 4096 + 2));
constexpr size_t kScal = kPartials + al(sizeof(Partial) * (kN / 128 + 2));
constexpr size_t kCtl = kScal + al(2 * sizeof(Scalars));
constexpr size_t kTickets = kCtl + al(sizeof(StepCtl));
constexpr size_t kErr = kTickets + al(16);
constexpr size_t kBytes = kErr + al(16);

// The scratch array. Host code must not use its name as an address: the
// address comes from cudaGetSymbolAddress, per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kBytes];

std::mutex g_mu;
void* g_addr[256] = {nullptr};

// device address of the scratch array on the current device (looked up once)
cudaError_t scratch_base(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = (unsigned char*)g_addr[dev];
  return cudaSuccess;
}

// largest distance from a point of the box to the surface of shape s
double max_surface_distance(const sph_domain& d, int s) {
  double far = 0.0;
  for (int corner = 0; corner < (1 << d.dim); ++corner) {
    double r2 = 0.0;
    for (int k = 0; k < d.dim; ++k) {
      const double x = (corner >> k) & 1 ? d.hi[k] : d.lo[k];
      r2 += (x - d.shapes[s].center[k]) * (x - d.shapes[s].center[k]);
    }
    far = std::max(far, std::sqrt(r2));
  }
  double sz = 0.0;
  for (int k = 0; k < 3; ++k) sz = std::max(sz, std::fabs(d.shapes[s].size[k]));
  return far + sz;
}

}  // namespace

extern "C" sph_status sph_eval_forces_noalloc(const sph_domain* dom, const sph_field* field,
                                              const sph_params* params, int64_t n, const double* xyz_dev,
                                              const uint8_t* col_dev, double* rho_dev, double* acc_dev,
                                              double* dt_dev, void* stream) {
  std::string why;
  sph_status vs = validate(dom, field, n, 1, params, why);
  if (vs != SPH_OK) {
    fprintf(stderr, "sph_eval_forces_noalloc: %s\n", why.c_str());
    return vs;
  }
  if (n > (int64_t)kN) {
    fprintf(stderr, "sph_eval_forces_noalloc: %lld particles exceed the limit of %d\n", (long long)n,
            SPH_NOALLOC_MAX_PARTICLES);
    return SPH_ERR_INVALID_ARG;
  }
  if (params->precision != SPH_PREC_FP32_SPLIT || !(field->rho_scale > 0)) {
    fprintf(stderr, "sph_eval_forces_noalloc: needs FP32 split precision and an explicit rho_scale > 0\n");
    return SPH_ERR_INVALID_ARG;
  }
  if (n > 0 && (!xyz_dev || !col_dev || !rho_dev || !acc_dev)) return SPH_ERR_INVALID_ARG;
  if (!dt_dev) return SPH_ERR_INVALID_ARG;
  const int d = dom->dim;
  cudaStream_t st = (cudaStream_t)stream;

  // grid from analytic bounds of h over the box (no sampling pass)
  double S = 0.0;
  for (int k = 0; k < field->n_poly; ++k) S += std::fabs(field->poly[k]);
  const double hfac = params->tau * std::pow(field->rho_scale, -1.0 / d);
  double smin = field->s0, smax = field->s0;
  if (field->kind == SPH_FIELD_LINEAR_DISTANCE) {
    smin = field->a;
    smax = field->a + std::fabs(field->b) * max_surface_distance(*dom, field->dist_shape);
  } else if (field->kind == SPH_FIELD_TANH_DISTANCE) {
    smin = field->a;
    smax = field->a + std::fabs(field->b) * std::tanh(field->s0 * max_surface_distance(*dom, field->dist_shape));
  }
  const double hmin = hfac * smin * std::pow(1.0 + S, -1.0 / d);
  const double hmax = hfac * smax * std::pow(1.0 - S, -1.0 / d);
  const double lip = lipschitz_h(*dom, *field, hfac, smax, field_slope(*field));
  HostGrid hg;
  why = grid_setup(*dom, params->kappa, params->cell_factor, hmin, hmax, lip, hg);
  if (!why.empty()) {
    fprintf(stderr, "sph_eval_forces_noalloc: %s\n", why.c_str());
    return SPH_ERR_INVALID_ARG;
  }
  const uint32_t cells = hg.base[hg.n_levels];
  if (cells > kC) {
    fprintf(stderr, "sph_eval_forces_noalloc: the grid needs %u cells, above the limit of %d (raise cell_factor)\n",
            cells, SPH_NOALLOC_MAX_CELLS);
    return SPH_ERR_INVALID_ARG;
  }
  Frames fr;
  make_frames(*dom, params->kappa, 0.0, hg, fr);  // one evaluation: no skin
  Geom<float> geof;
  fill_geom<float>(*dom, *field, hfac, field->rho_scale, geof);
  Phys<float> Pf;
  fill_phys(d, *params, Pf);

  unsigned char* base = nullptr;
  cudaError_t e = scratch_base(&base);
  if (e != cudaSuccess) {
    fprintf(stderr, "sph_eval_forces_noalloc: cudaGetSymbolAddress: %s\n", cudaGetErrorString(e));
    return SPH_ERR_CUDA;
  }
  DevState Sd;
  Sd.n = (int)n;
  Sd.dim = d;
  Sd.fp64 = 0;
  Sd.cap = (int)kCap;
  Sd.X[0] = base + kX0;
  Sd.X[1] = base + kX1;
  Sd.meta[0] = (uint32_t*)(base + kM0);
  Sd.meta[1] = (uint32_t*)(base + kM1);
  Sd.pid[0] = (uint32_t*)(base + kP0);
  Sd.pid[1] = (uint32_t*)(base + kP1);
  Sd.view[0] = base + kV0;
  Sd.view[1] = base + kV1;
  Sd.vbuild = base + kVb;
  Sd.key = (uint32_t*)(base + kKey);
  Sd.tmp = (uint32_t*)(base + kTmp);
  Sd.list = (uint32_t*)(base + kList);
  Sd.lcount = (uint32_t*)(base + kLcount);
  Sd.plist = (uint32_t*)(base + kPlist);
  Sd.pcount = (uint32_t*)(base + kPcount);
  Sd.acc4 = base + kAcc4;
  Sd.rho = base + kRho;
  Sd.pc = base + kPc;
  Sd.cnt = (uint32_t*)(base + kCnt);
  Sd.cstart = (uint32_t*)(base + kCstart);
  Sd.scan_part = (uint32_t*)(base + kScanPart);
  Sd.total_cells = cells;
  Sd.partials = (Partial*)(base + kPartials);
  Sd.scal = (Scalars*)(base + kScal);
  Sd.ctl = (StepCtl*)(base + kCtl);
  Sd.tickets = (unsigned*)(base + kTickets);
  Sd.err = (int*)(base + kErr);

  // state that must start at zero: cell counters, the last-block ticket, the
  // error word, the statistics; the control block (step 0, no ramp; the gate
  // below moves the state set here from buffer 0 into buffer 1)
  StepCtl ctl{};
  ctl.step = 0;
  ctl.t0 = ctl.t1 = -1.0;
  ctl.sigma0 = params->sigma0;
  ctl.need_rebuild = 1;
#define NA_CUDA(expr)                                                                      \
  do {                                                                                     \
    cudaError_t e_ = (expr);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      fprintf(stderr, "sph_eval_forces_noalloc: %s: %s\n", #expr, cudaGetErrorString(e_)); \
      return SPH_ERR_CUDA;                                                                 \
    }                                                                                      \
  } while (0)
  NA_CUDA(cudaMemsetAsync(Sd.cnt, 0, sizeof(uint32_t) * cells, st));
  NA_CUDA(cudaMemsetAsync(Sd.tickets, 0, 16, st));
  NA_CUDA(cudaMemsetAsync(Sd.err, 0, sizeof(int), st));
  NA_CUDA(cudaMemsetAsync(Sd.scal, 0, sizeof(Scalars), st));
  NA_CUDA(cudaMemcpyAsync(Sd.ctl, &ctl, sizeof ctl, cudaMemcpyHostToDevice, st));
  if (n > 0) {
    PassFlags f;
    f.general_eos = params->gamma != 2.0;
    f.advance = 0;
    const float kappa = (float)params->kappa;
    if (d == 2) {
      NA_CUDA((launch_set_state<2, float>(Sd, fr.f, xyz_dev, col_dev, st)));
      NA_CUDA(launch_gate(Sd, 1, st));
      NA_CUDA((launch_rebuild<2, float>(Sd, fr.gf, fr.f, geof, kappa, st)));
      NA_CUDA((launch_pass_a<2, float>(Sd, fr.f, Pf, f, st)));
      NA_CUDA((launch_get_fields<2, float>(Sd, 0, rho_dev, st)));
      NA_CUDA((launch_get_fields<2, float>(Sd, 1, acc_dev, st)));
    } else {
      NA_CUDA((launch_set_state<3, float>(Sd, fr.f, xyz_dev, col_dev, st)));
      NA_CUDA(launch_gate(Sd, 1, st));
      NA_CUDA((launch_rebuild<3, float>(Sd, fr.gf, fr.f, geof, kappa, st)));
      NA_CUDA((launch_pass_a<3, float>(Sd, fr.f, Pf, f, st)));
      NA_CUDA((launch_get_fields<3, float>(Sd, 0, rho_dev, st)));
      NA_CUDA((launch_get_fields<3, float>(Sd, 1, acc_dev, st)));
    }
  }
  // dt1 and dt2 are the first two fields of the step scalars
  NA_CUDA(cudaMemcpyAsync(dt_dev, Sd.scal, 2 * sizeof(double), cudaMemcpyDeviceToDevice, st));
  int flags = 0;
  NA_CUDA(cudaMemcpyAsync(&flags, Sd.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  NA_CUDA(cudaStreamSynchronize(st));
#undef NA_CUDA
  if (flags & kErrNonfinite) return SPH_ERR_NONFINITE;
  if (flags & kErrOutOfDomain) return SPH_ERR_OUT_OF_DOMAIN;
  if (flags & kErrListOverflow) return SPH_ERR_CELL_OVERFLOW;
  if (flags & kErrTimeout) return SPH_ERR_TIMEOUT;
  if (flags) return SPH_ERR_CUDA;  // a device error bit this call does not name
  return SPH_OK;
}
