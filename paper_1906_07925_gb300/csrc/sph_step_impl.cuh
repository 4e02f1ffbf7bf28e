// Relaxation-step kernels (the step of Algorithm 1), templated on the
// dimension D and the working precision T. Instantiated per dimension in
// sph_step_2d.cu / sph_step_3d.cu.
//
// State. Each particle is an int64 coordinate per axis (Frame). Pair vectors
// come from a per-step view: FP32 keeps the low 32 bits of X >> sv and forms
// differences modulo 2^32 (exact for nearby particles) converted without the
// conversion unit; FP64 keeps physical coordinates. Either way the rounding of
// a pair vector is relative to the pair distance, not to the domain size.
//
// Neighbour list (the neighbour search of Algorithm 1). The list of particle i holds every j
// (itself included) that can come within kappa max(h_i, h_j) before some
// particle has moved half its skin; it is rebuilt, on the device, only then.
// The criterion is symmetric, so i also finds every j whose own support
// reaches i (the reverse pass gathers over such pairs).
// Passes A and B re-test the exact criteria of the current step for every
// listed pair, so the list only saves the search, never changes a result.
#pragma once

#include <algorithm>
#include <cfloat>
#include <climits>
#include <type_traits>

#include "sph_internal.h"

// resident 256-thread blocks per SM asked of the pair passes and of the list
// build (caps registers)
#ifndef SPH_PASS_MIN_BLOCKS
#define SPH_PASS_MIN_BLOCKS 5
#endif
// store of a force-pair list word (streaming: read once, by pass B)
#ifndef SPH_PLIST_STREAM
#define SPH_PLIST_STREAM 1
#endif
#if SPH_PLIST_STREAM
#define SPH_PLIST_STORE(p, v) __stcs((p), (v))
#else
#define SPH_PLIST_STORE(p, v) (*(p) = (v))
#endif
// the pair passes are compiled for 128 and 256 threads per block
// (DevState::pass_threads picks one at launch); resident blocks per SM asked
// of them scale so that the register budget per thread is the same
#ifndef SPH_PASSB_MIN_BLOCKS
#define SPH_PASSB_MIN_BLOCKS SPH_PASS_MIN_BLOCKS
#endif
#ifndef SPH_LIST_MIN_BLOCKS
#define SPH_LIST_MIN_BLOCKS 4
#endif
// the FP64 variants keep twice the registers live: at 5 blocks (48 registers)
// they spilled 600-1,000 bytes per thread; at 2 blocks (128 registers) none,
// and the 8M 3D FP64 step took 86 ms instead of 99.5 (3 blocks: 99.1)
#ifndef SPH_PASS_MIN_BLOCKS_FP64
#define SPH_PASS_MIN_BLOCKS_FP64 2
#endif
#ifndef SPH_PASSB_MIN_BLOCKS_FP64
#define SPH_PASSB_MIN_BLOCKS_FP64 2
#endif

namespace sph {

// ---------------------------------------------------------------- views ----
template <class T> struct ViewOf;
template <> struct ViewOf<float> { using type = int4; };
template <> struct ViewOf<double> { using type = V4<double>; };

// Difference of two view coordinates, in view units (finest cell edges).
// Precise (FAST = false): the exact integer difference, rounded once to float.
// Coarse (FAST = true, the inside/outside test of a listed pair): the view
// integers are dropped to 2^-kCoarseBits c0 and their difference d (|d| < 2^22,
// certified per particle by the list build) is added to the bits of
// 1.5 * 2^(23 - kCoarseBits), whose low mantissa bit weighs 2^-kCoarseBits: the
// float is then bias + d 2^-kCoarseBits exactly, converted by one integer add
// and one float subtract instead of the conversion unit.
template <bool FAST>
__device__ __forceinline__ float vd(const Frame<float>& F, int a, int b) {
  if (FAST) {
    // the modular difference is exact; shift it, not the (wrapped) operands
    constexpr int s = kViewBits - kCoarseBits;
    return __int_as_float(F.mbits + ((a - b) >> s)) - F.mbias;
  }
  return (float)(a - b) * F.vscale;
}
template <bool FAST>
__device__ __forceinline__ double vd(const Frame<double>&, double a, double b) {
  return a - b;
}
// radius H widened for a screening test on coarse vectors: each coarse component
// is the exact one floored to 2^-kCoarseBits c0, so |r_coarse - r| < sqrt(3) 2^-kCoarseBits;
// the relative term covers FP32 rounding of r^2. A pair that passes is tested
// again on the exact vectors, so the slack only admits a few extra candidates.
template <class T>
__device__ __forceinline__ T screen_radius(T H) {
  return H * T(1.0 + 1.0 / (1 << 20)) + T(1.0 / (1 << (kCoarseBits - 2)));
}
__device__ __forceinline__ float view_h(const int4& v) { return __int_as_float(v.w); }
__device__ __forceinline__ double view_h(const V4<double>& v) { return v.w; }

// The neighbour list of particle i is column i of a cap x n array, split at
// its build: the entries then inside their support (r < max(kappa h_i,
// kappa h_ij)) fill rows 0, 1, ... in candidate order, the others rows cap-1,
// cap-2, ... in candidate order. A pass walks the inside part first, so the
// entries that pass its exact tests cluster at the start of every list and a
// warp skips the pair body on the later rows, where no lane's entry passes.
// lcount packs both counts (bits 0-14 and 15-29); bit 31 certifies that
// every listed pair stays within the exact range of the FP32 fast conversion
// until the next rebuild.
constexpr uint32_t kFastBit = 0x80000000u;
constexpr uint32_t kCountMask = 0x7FFFu;
constexpr int kOutShift = 15;
__device__ __forceinline__ int list_in(uint32_t lc) { return (int)(lc & kCountMask); }
__device__ __forceinline__ int list_cnt(uint32_t lc) {
  return (int)(lc & kCountMask) + (int)((lc >> kOutShift) & kCountMask);
}

struct alignas(32) LL4 {
  long long x, y, z, w;
};

// physical position (relative to lo) of an integer coordinate
template <class T>
__device__ __forceinline__ T coord_phys(const Frame<T>& F, long long X) {
  return (T)X * F.q64t;
}

// view of a particle at integer position X with smoothing length h (physical):
// FP32 integers of 2^-kViewBits c0 (rounded; the low 32 bits suffice because
// only differences of nearby particles are used), FP64 c0 units; w = h / c0
template <int D>
__device__ __forceinline__ int4 make_view(const Frame<float>& F, const LL4& X, float h) {
  const long long half = 1LL << (F.sv - 1);
  return make_int4((int)((X.x + half) >> F.sv), (int)((X.y + half) >> F.sv), D == 3 ? (int)((X.z + half) >> F.sv) : 0,
                   __float_as_int(h * F.inv_qv));
}
template <int D>
__device__ __forceinline__ V4<double> make_view(const Frame<double>& F, const LL4& X, double h) {
  return V4<double>{(double)X.x * F.s2v, (double)X.y * F.s2v, D == 3 ? (double)X.z * F.s2v : 0.0, h * F.inv_qv};
}
__device__ __forceinline__ int4 with_w(int4 v, float w) { return make_int4(v.x, v.y, v.z, __float_as_int(w)); }
__device__ __forceinline__ V4<double> with_w(V4<double> v, double w) { return V4<double>{v.x, v.y, v.z, w}; }

// Visit the cnt listed entries of particle i (column i of the list) in
// batches of SPH_LIST_BATCH: the list words, then the neighbour views, are
// loaded before any is used, so each warp keeps several independent gathers in
// flight. List words are streamed (read once per pass).
#ifndef SPH_LIST_BATCH
#define SPH_LIST_BATCH 4
#endif
// Entry k of a list whose first n_in entries sit in rows 0.. and the rest in
// rows cap-1, cap-2, ... (a compact list: n_in = cnt).
__device__ __forceinline__ size_t list_row(int k, int n_in, int cap) {
  return (size_t)(k < n_in ? k : cap - 1 - (k - n_in));
}
template <class VT, class Fn>
__device__ __forceinline__ void for_list(const uint32_t* __restrict__ list, const VT* __restrict__ view, int n, int i,
                                         int cnt, int n_in, int cap, Fn&& pair) {
  constexpr int B = SPH_LIST_BATCH;
  int k = 0;
  for (; k + B <= cnt; k += B) {
    uint32_t e[B];
    VT v[B];
#pragma unroll
    for (int q = 0; q < B; ++q) e[q] = __ldcs(list + list_row(k + q, n_in, cap) * n + i);
#pragma unroll
    for (int q = 0; q < B; ++q) v[q] = view[e[q] >> 8];
#pragma unroll
    for (int q = 0; q < B; ++q) pair(e[q], v[q]);
  }
  for (; k < cnt; ++k) {
    const uint32_t e = __ldcs(list + list_row(k, n_in, cap) * n + i);
    pair(e, view[e >> 8]);
  }
}
// a compact list (rows 0 .. cnt-1)
template <class VT, class Fn>
__device__ __forceinline__ void for_list(const uint32_t* __restrict__ list, const VT* __restrict__ view, int n, int i,
                                         int cnt, Fn&& pair) {
  for_list(list, view, n, i, cnt, cnt, 0, pair);
}
// A compact list (rows 0 .. cnt-1) whose pair body also needs a record of
// the neighbour (its acceleration, an adjoint): that record, fetch(j), is
// loaded for the whole batch together with the views, so each thread keeps
// 2 x SPH_LIST_BATCH_X independent gathers in flight instead of meeting the
// record's latency inside every pair body.
#ifndef SPH_LIST_BATCH_X
#define SPH_LIST_BATCH_X 2  // 4 spilled at the 48 / 64-register budgets of the passes using it
#endif
template <class VT, class Fetch, class Fn>
__device__ __forceinline__ void for_list_x(const uint32_t* __restrict__ list, const VT* __restrict__ view, int n,
                                           int i, int cnt, Fetch&& fetch, Fn&& pair) {
  using XT = decltype(fetch(0));
  constexpr int B = SPH_LIST_BATCH_X;
  int k = 0;
  for (; k + B <= cnt; k += B) {
    uint32_t e[B];
    VT v[B];
    XT x[B];
#pragma unroll
    for (int q = 0; q < B; ++q) e[q] = __ldcs(list + (size_t)(k + q) * n + i);
#pragma unroll
    for (int q = 0; q < B; ++q) {
      v[q] = view[e[q] >> 8];
      x[q] = fetch((int)(e[q] >> 8));
    }
#pragma unroll
    for (int q = 0; q < B; ++q) pair(e[q], v[q], x[q]);
  }
  for (; k < cnt; ++k) {
    const uint32_t e = __ldcs(list + (size_t)k * n + i);
    pair(e, view[e >> 8], fetch((int)(e >> 8)));
  }
}
// the skin list of particle i (split at its build, see kFastBit)
template <class VT, class Fn>
__device__ __forceinline__ void for_skin_list(const uint32_t* __restrict__ list, const VT* __restrict__ view, int n,
                                              int i, uint32_t lc, int cap, Fn&& pair) {
  for_list(list, view, n, i, list_cnt(lc), list_in(lc), cap, pair);
}

// The FP64 path's skin list screened on its FP32 views (v32, kept current
// every step): each entry is first tested on coarse FP32 differences
// (screen), and only the entries that pass gather their FP64 view for the
// exact FP64 tests (pair). The screen is conservative, so the pairs the
// exact tests accept are the same as with an FP64 screen; the entries it
// rejects cost no FP64 arithmetic (the FP64 pipe bounds that pass).
template <class VT, class Screen, class Fn>
__device__ __forceinline__ void for_skin_list_s32(const uint32_t* __restrict__ list, const int4* __restrict__ v32,
                                                  const VT* __restrict__ view, int n, int i, uint32_t lc, int cap,
                                                  Screen&& screen, Fn&& pair) {
  constexpr int B = SPH_LIST_BATCH;
  const int cnt = list_cnt(lc), n_in = list_in(lc);
  int k = 0;
  for (; k + B <= cnt; k += B) {
    uint32_t e[B];
    int4 w[B];
    bool ok[B];
    VT v[B];
#pragma unroll
    for (int q = 0; q < B; ++q) e[q] = __ldcs(list + list_row(k + q, n_in, cap) * n + i);
#pragma unroll
    for (int q = 0; q < B; ++q) w[q] = v32[e[q] >> 8];
#pragma unroll
    for (int q = 0; q < B; ++q) {
      ok[q] = screen(w[q]);
      if (ok[q]) v[q] = view[e[q] >> 8];
    }
#pragma unroll
    for (int q = 0; q < B; ++q)
      if (ok[q]) pair(e[q], v[q]);
  }
  for (; k < cnt; ++k) {
    const uint32_t e = __ldcs(list + list_row(k, n_in, cap) * n + i);
    if (screen(v32[e >> 8])) pair(e, view[e >> 8]);
  }
}

// Staged lists (pass A, FP32): in a block whose distinct neighbours fit in
// shared memory, entry k of particle i's list is also stored, at the same
// position of llist, as (rank << 8 | colour_j) with bit kStageSelf set for
// j = i; rank numbers j within the block's staged set (sj). The views of the
// set are gathered into shared memory once per step, so the list walk reads
// them there instead of gathering each from global memory.
constexpr uint32_t kStageSelf = 1u << 20;
__device__ __forceinline__ int stage_rank(uint32_t e) {
  const int r = (int)((e >> 8) & 0xFFFu);
  return r < kStageCap ? r : kStageCap - 1;  // in range by construction; the clamp keeps any stale word in bounds
}
template <class VT, class Fn>
__device__ __forceinline__ void for_staged_list(const uint32_t* __restrict__ llist, const VT* sview, int n, int i,
                                                uint32_t lc, int cap, Fn&& pair) {
  constexpr int B = SPH_LIST_BATCH;
  const int cnt = list_cnt(lc), n_in = list_in(lc);
  int k = 0;
  for (; k + B <= cnt; k += B) {
    uint32_t e[B];
    VT v[B];
#pragma unroll
    for (int q = 0; q < B; ++q) e[q] = __ldcs(llist + list_row(k + q, n_in, cap) * n + i);
#pragma unroll
    for (int q = 0; q < B; ++q) v[q] = sview[stage_rank(e[q])];
#pragma unroll
    for (int q = 0; q < B; ++q) pair(e[q], v[q]);
  }
  for (; k < cnt; ++k) {
    const uint32_t e = __ldcs(llist + list_row(k, n_in, cap) * n + i);
    pair(e, sview[stage_rank(e)]);
  }
}
// 16-byte asynchronous copy global -> shared (cp.async, L2 only), and the wait
// for every copy this thread issued
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// a length in state units rounded to the nearest integer (ties to even): the
// FP32 value converts directly (the same integer as rounding its exact FP64
// widening, without the FP64 conversion)
__device__ __forceinline__ long long state_units(float x) { return __float2ll_rn(x); }
__device__ __forceinline__ long long state_units(double x) { return llrint(x); }

template <class T> __device__ __forceinline__ T pair_r(T r2);
template <> __device__ __forceinline__ float pair_r<float>(float r2) { return r2 * rsqrtf(r2); }
template <> __device__ __forceinline__ double pair_r<double>(double r2) { return sqrt(r2); }

template <int D, class T>
__device__ __forceinline__ void abs_pos(const Frame<T>& F, const LL4& X, T* x) {
  x[0] = F.lo[0] + coord_phys(F, X.x);
  x[1] = F.lo[1] + coord_phys(F, X.y);
  x[2] = D == 3 ? F.lo[2] + coord_phys(F, X.z) : T(0);
}

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
// minimum and where it sits; ties go to the smaller index (order-independent)
__device__ __forceinline__ void argmin_merge(double& v, long long& k, double ov, long long ok) {
  if (ov < v || (ov == v && ok < k)) {
    v = ov;
    k = ok;
  }
}
__device__ __forceinline__ void warp_argmin(double& v, long long& k) {
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, v, o);
    const long long ok = __shfl_xor_sync(0xffffffffu, k, o);
    argmin_merge(v, k, ov, ok);
  }
}

// fixed-order block reduction of a Partial (deterministic); valid in warp 0
__device__ __forceinline__ Partial block_reduce(Partial p, Partial* sm) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  warp_argmin(p.min_rc_a, p.amin);
  p.max_a = warp_max(p.max_a);
  p.sum_rho = warp_sum(p.sum_rho);
  p.err_l2 = warp_sum(p.err_l2);
  p.err_max = warp_max(p.err_max);
  p.ipairs = warp_sum(p.ipairs);
  p.fpairs = warp_sum(p.fpairs);
  p.lentries = warp_sum(p.lentries);
  if (lane == 0) sm[w] = p;
  __syncthreads();
  if (w == 0) {
    Partial q;
    if (lane < nw) q = sm[lane];
    else q = Partial{DBL_MAX, 0.0, 0.0, 0.0, 0.0, 0, 0, 0, -1};
    warp_argmin(q.min_rc_a, q.amin);
    q.max_a = warp_max(q.max_a);
    q.sum_rho = warp_sum(q.sum_rho);
    q.err_l2 = warp_sum(q.err_l2);
    q.err_max = warp_max(q.err_max);
    q.ipairs = warp_sum(q.ipairs);
    q.fpairs = warp_sum(q.fpairs);
    q.lentries = warp_sum(q.lentries);
    p = q;
  }
  __syncthreads();
  return p;
}

// ------------------------------------------------------------------------
// List rebuild (runs only when ctl->rebuild). Old order: buffer 1 - buf.
// ------------------------------------------------------------------------

// cell key of each particle in the old order: level from h at its position,
// cell coordinates X >> (cshift + level)
template <int D, class T>
__global__ void __launch_bounds__(256) k_rekey(int n, const StepCtl* __restrict__ ctl, const LL4* __restrict__ X0,
                                               const LL4* __restrict__ X1, Frame<T> F, Grid<T> G, Geom<T> geo,
                                               uint32_t* __restrict__ key) {
  if (!ctl->rebuild) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const LL4 X = (ctl->buf ? X0 : X1)[i];
    T x[3];
    abs_pos<D, T>(F, X, x);
    const int l = level_of_h(G, h_of<D, T>(geo, x));
    const int sh = G.cshift + l;
    const int c[3] = {(int)min((long long)G.nx[l] - 1, X.x >> sh), (int)min((long long)G.ny[l] - 1, X.y >> sh),
                      D == 3 ? (int)min((long long)G.nz[l] - 1, X.z >> sh) : 0};
    key[i] = G.base[l] + (uint32_t)c[0] + (uint32_t)G.nx[l] * ((uint32_t)c[1] + (uint32_t)G.ny[l] * (uint32_t)c[2]);
  }
}

// views of the (new) current order and the reference view for the skin test
template <int D, class T>
__global__ void __launch_bounds__(256) k_make_view(int n, const StepCtl* __restrict__ ctl, int force,
                                                   const LL4* __restrict__ X0, const LL4* __restrict__ X1,
                                                   Frame<T> F, Geom<T> geo, typename ViewOf<T>::type* __restrict__ v0,
                                                   typename ViewOf<T>::type* __restrict__ v1,
                                                   typename ViewOf<T>::type* __restrict__ vbuild) {
  if (!force && !ctl->rebuild) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const LL4 X = (ctl->buf ? X1 : X0)[i];
    T x[3];
    abs_pos<D, T>(F, X, x);
    const T h = h_of<D, T>(geo, x);
    const auto v = make_view<D>(F, X, h);
    (ctl->vp ? v1 : v0)[i] = v;
    vbuild[i] = with_w(v, T(0.5) * F.skin * view_h(v));  // half the skin, view units (kappa folded in by the host)
  }
}

// FP32 view of the FP64 path's particles, made at a list rebuild for its list
// build (and kept current every step by pass B for pass A's FP32 screen): the
// list only has to hold every pair the exact FP64 tests can accept before the
// next rebuild, and an FP32 candidate test errs by ~1e-7 of the distance, far
// inside the list's margins (the skin and the 1e-5 factor), while FP64
// arithmetic runs at a small fraction of the FP32 rate on this GPU.
template <int D>
__global__ void __launch_bounds__(256) k_view32(int n, const StepCtl* __restrict__ ctl,
                                                const LL4* __restrict__ X0, const LL4* __restrict__ X1,
                                                Frame<float> F, const V4<double>* __restrict__ vd0,
                                                const V4<double>* __restrict__ vd1, int4* __restrict__ out) {
  if (!ctl->rebuild) return;
  const long long half = 1LL << (F.sv - 1);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const LL4 X = (ctl->buf ? X1 : X0)[i];
    const double hv = (ctl->vp ? vd1 : vd0)[i].w;  // h in view units (c0, both precisions)
    out[i] = make_int4((int)((X.x + half) >> F.sv), (int)((X.y + half) >> F.sv),
                       D == 3 ? (int)((X.z + half) >> F.sv) : 0, __float_as_int((float)hv));
  }
}

// Neighbour list of each particle: every j (itself included) with
//   r < kappa max(h_i, h_j) (1 + 1e-5) + kappa lip_h s_max / 2 + s_max,
// s = skin (kappa folded) of i and j: after both moved at most half their skin
// (and h changed by at most lip_h times that), any pair inside the exact
// criteria is still listed. Candidates come from rows of cells of every level
// that can hold such a j, in the order (level, z row, y row, x).
template <int D, class T>
__global__ void __launch_bounds__(256, SPH_LIST_MIN_BLOCKS) k_list_build(int n, StepCtl* __restrict__ ctl,
                                                    const LL4* __restrict__ X0, const LL4* __restrict__ X1,
                                                    const uint32_t* __restrict__ m0, const uint32_t* __restrict__ m1,
                                                    const typename ViewOf<T>::type* __restrict__ v0,
                                                    const typename ViewOf<T>::type* __restrict__ v1,
                                                    const uint32_t* __restrict__ cstart, Frame<T> F, Grid<T> G,
                                                    T kappa, int cap, uint32_t* __restrict__ list,
                                                    uint32_t* __restrict__ lcount, int* __restrict__ err) {
  using VT = typename ViewOf<T>::type;
  if (!ctl->rebuild) return;
  const int buf = ctl->buf;
  const VT* __restrict__ view = ctl->vp ? v1 : v0;
  const uint32_t* __restrict__ meta = buf ? m1 : m0;
  int cmax = 0;  // longest list of this thread's targets
  bool over_any = false;
  // grid-stride over the targets (one per thread at the grid it is launched with)
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
  const LL4 X = (buf ? X1 : X0)[i];
  const VT vi = view[i];
  const T hv = view_h(vi);                 // view units
  const T sk = F.skin * hv;                // skin of i, view units (kappa folded in by the host)
  const T sk_hv = F.skin;                  // skin per unit h
  const T lip = G.lip_h;
  // search radius: bound h_j by Lipschitz continuity, iterate twice
  T hhi = hv, Rs = kappa * hv * G.rfac + sk * (T(1) + T(0.5) * kappa * lip);
  for (int it = 0; it < 2; ++it) {
    hhi = hv * T(1.00001) + lip * Rs;
    const T shi = sk * hhi / hv;
    Rs = kappa * hhi * G.rfac + shi * (T(1) + T(0.5) * kappa * lip);
    Rs = Rs > kappa * hv * G.rfac ? Rs : kappa * hv * G.rfac;
  }
  const T hlo = hv * T(0.99999) - lip * Rs;
  const T qv = F.qv;
  const int l0 = level_of_h(G, hlo * qv), l1 = level_of_h(G, hhi * qv);
  const T R2 = Rs * Rs;
  int cnt = 0, n_in = 0, n_out = 0;  // accepted; written inside / outside entries
  bool over = false;
  T reach = 0;
  const T Hd = kappa * hv;

  // one candidate: every test is evaluated without a branch (most candidates
  // fail, and a branch over the acceptance tests ran for a few lanes of the
  // warp in nearly every iteration); only the list store is conditional
  const T cl = T(1) + T(0.5) * kappa * lip;
  auto cand = [&](int jc, const VT& vj) {
    const T dx = vd<false>(F, vi.x, vj.x), dy2 = vd<false>(F, vi.y, vj.y);
    const T dz2 = D == 3 ? vd<false>(F, vi.z, vj.z) : T(0);
    const T r2 = dx * dx + dy2 * dy2 + dz2 * dz2;
    const T hj = view_h(vj);
    const T skj = sk_hv * hj;
    const T smax = sk > skj ? sk : skj;
    const T hm = hv > hj ? hv : hj;  // symmetric: j lists i whenever i lists j
    // h_j is known here: only rounding and the h change over the skin need a margin
    const T Rl = kappa * hm * T(1.00001) + smax * cl;
    const bool acc = r2 < R2 && r2 < Rl * Rl;
    // inside its support now (density or force): the front of the list
    const T Hf = T(0.5) * kappa * (hv + hj);
    const T Hp = Hf > Hd ? Hf : Hd;
    const bool inside = r2 < Hp * Hp;
    // largest axis separation this pair can reach before the next rebuild
    const T ax = fabs(dx) > fabs(dy2) ? fabs(dx) : fabs(dy2);
    const T am = (ax > fabs(dz2) ? ax : fabs(dz2)) + smax;
    reach = acc && am > reach ? am : reach;
    if (acc) {
      if (cnt < cap) {
        const int row = inside ? n_in++ : cap - 1 - n_out++;
        list[(size_t)row * n + i] = ((uint32_t)jc << 8) | (meta[jc] & 0xFFu);
      } else {
        over = true;
      }
      ++cnt;
    }
  };

  for (int l = l0; l <= l1; ++l) {
    const int sh = G.cshift + l;
    const int nx = G.nx[l], ny = G.ny[l], nz = G.nz[l];
    const int cxl = (int)min((long long)nx - 1, X.x >> sh);
    const int cyl = (int)min((long long)ny - 1, X.y >> sh);
    const int czl = D == 3 ? (int)min((long long)nz - 1, X.z >> sh) : 0;
    const T c = G.cellv[l], ic = T(1) / c;
    // target position inside its level-l cell, view units
    const T fx = (T)((double)(X.x - ((long long)cxl << sh)) * F.s2v);
    const T fy = (T)((double)(X.y - ((long long)cyl << sh)) * F.s2v);
    const T fz = D == 3 ? (T)((double)(X.z - ((long long)czl << sh)) * F.s2v) : T(0);
    const uint32_t base = G.base[l];
    int zlo = 0, zhi = 0;
    if (D == 3) {
      zlo = (int)dfloor((fz - Rs) * ic);
      zhi = (int)dfloor((fz + Rs) * ic);
    }
    const int ylo = (int)dfloor((fy - Rs) * ic), yhi = (int)dfloor((fy + Rs) * ic);
    for (int dz = zlo; dz <= zhi; ++dz) {
      const int czz = czl + dz;
      if (D == 3 && (czz < 0 || czz >= nz)) continue;
      T dzp = 0;
      if (D == 3) {
        const T zrel = fz - (T)dz * c;
        dzp = zrel < T(0) ? -zrel : (zrel > c ? zrel - c : T(0));
      }
      for (int dy = ylo; dy <= yhi; ++dy) {
        const int cyy = cyl + dy;
        if (cyy < 0 || cyy >= ny) continue;
        const T yrel = fy - (T)dy * c;
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
        const int jb = (int)cstart[krow + (uint32_t)x0], je = (int)cstart[krow + (uint32_t)x1 + 1];
        // candidates in ascending order, two views loaded before either is
        // tested (two loads in flight per thread: a rebuild of the 8M 3D
        // workload 3.5 % faster than one at a time)
        int j = jb;
        for (; j + 2 <= je; j += 2) {
          const VT va = view[j], vb = view[j + 1];
          cand(j, va);
          cand(j + 1, vb);
        }
        for (; j < je; ++j) cand(j, view[j]);
      }
    }
  }
  // the coarse FP32 conversion is exact below 2^22 coarse integers = 2^(22 - kCoarseBits) c0
  const bool fast = reach < T(0.999) * T(1 << (22 - kCoarseBits));
  lcount[i] = (uint32_t)n_in | ((uint32_t)n_out << kOutShift) | (fast ? kFastBit : 0u);
  over_any |= over;
  cmax = cnt > cmax ? cnt : cmax;
  }  // targets
  if (over_any) atomicOr(err, kErrListOverflow);
  // longest list of this build (one atomic per warp; every lane gets here)
  const int wmax = __reduce_max_sync(0xffffffffu, cmax);
  if ((threadIdx.x & 31) == 0 && wmax > 0) atomicMax(&ctl->lmax, wmax);
}

// Staged pass A, set up at a list rebuild: one block per kStageBlock targets
// (the blocks of pass A). The distinct neighbours j of the block's lists go
// into a hash set in shared memory (linear probing); the occupied slots in slot
// order number them (rank), sj[block][rank] = j and scount[block] = their
// count; every list entry is written again into llist as (rank << 8 | colour),
// with kStageSelf for j = i. A block with more than kStageCap neighbours, or a
// set too crowded to probe, gets scount = -1: pass A gathers its views from
// global memory. The ranks depend on the order of the hash inserts, but pass
// A's sums follow the list order, so its results do not.
constexpr int kStageHashBits = 12;
static_assert((1 << kStageHashBits) == kStageHash, "hash set size");
constexpr int kStageProbe = 64;
__device__ __forceinline__ uint32_t stage_hash(int j) { return ((uint32_t)j * 2654435761u) >> (32 - kStageHashBits); }

template <int D>
__global__ void __launch_bounds__(kStageBlock) k_stage(int n, const StepCtl* __restrict__ ctl,
                                                      const uint32_t* __restrict__ list,
                                                      const uint32_t* __restrict__ lcount, int cap,
                                                      uint32_t* __restrict__ llist, int* __restrict__ scount,
                                                      int* __restrict__ sj) {
  if (!ctl->rebuild) return;
  __shared__ int tab[kStageHash];
  __shared__ int rnk[kStageHash];
  __shared__ int wsum[kStageBlock / 32];
  __shared__ int bad;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  for (int q = t; q < kStageHash; q += kStageBlock) tab[q] = -1;
  if (t == 0) bad = 0;
  __syncthreads();
  const int i = blockIdx.x * kStageBlock + t;
  const uint32_t lc = i < n ? lcount[i] : 0u;
  const int cnt = list_cnt(lc), n_in = list_in(lc);
  for (int k = 0; k < cnt; ++k) {
    const int j = (int)(list[list_row(k, n_in, cap) * n + i] >> 8);
    uint32_t q = stage_hash(j);
    int p = 0;
    for (; p < kStageProbe; ++p) {
      const int old = atomicCAS(&tab[q], -1, j);
      if (old == -1 || old == j) break;
      q = (q + 1) & (kStageHash - 1);
    }
    if (p == kStageProbe) bad = 1;
  }
  __syncthreads();
  const bool crowded = bad != 0;
  // ranks: thread t owns slots [per t, per (t + 1)); exclusive scan of the counts
  constexpr int per = kStageHash / kStageBlock;
  int c = 0;
  for (int q = 0; q < per; ++q) c += tab[t * per + q] >= 0;
  int x = c;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  int r = x - c, m = 0;
  for (int q = 0; q < kStageBlock / 32; ++q) {
    r += q < w ? wsum[q] : 0;
    m += wsum[q];
  }
  if (crowded || m > kStageCap) {
    if (t == 0) scount[blockIdx.x] = -1;
    return;
  }
  int* __restrict__ sjb = sj + (size_t)blockIdx.x * kStageCap;
  for (int q = 0; q < per; ++q) {
    const int slot = t * per + q;
    const int j = tab[slot];
    if (j >= 0) {
      rnk[slot] = r;
      sjb[r] = j;
      ++r;
    }
  }
  __syncthreads();
  for (int k = 0; k < cnt; ++k) {
    const size_t pos = list_row(k, n_in, cap) * n + i;
    const uint32_t e = list[pos];
    const int j = (int)(e >> 8);
    uint32_t q = stage_hash(j);
    for (int p = 0; p < kStageProbe && tab[q] != j; ++p) q = (q + 1) & (kStageHash - 1);
    llist[pos] = ((uint32_t)rnk[q] << 8) | (e & 0xFFu) | (j == i ? kStageSelf : 0u);
  }
  if (t == 0) scount[blockIdx.x] = m;
}

// --------------------------------------------------------------------------
// Density pass (general gamma): rho_i (Eq. density_sum) and p_i / rho_i^2 with
// p = P0 (rho/rho_t)^gamma (Eq. EOS_current), needed by the neighbours' forces.
// --------------------------------------------------------------------------
template <int D, class T>
__global__ void __launch_bounds__(256) k_density(int n, const StepCtl* __restrict__ ctl,
                                                 const typename ViewOf<T>::type* __restrict__ v0,
                                                 const typename ViewOf<T>::type* __restrict__ v1,
                                                 const uint32_t* __restrict__ list,
                                                 const uint32_t* __restrict__ lcount, int cap, Frame<T> F,
                                                 Phys<T> P, T* __restrict__ rho_out, T* __restrict__ pc_out) {
  using VT = typename ViewOf<T>::type;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const VT* __restrict__ view = ctl->vp ? v1 : v0;
  const VT vi = view[i];
  const T hv = view_h(vi);
  const T Hd = P.kappa * hv, Hd2 = Hd * Hd, invHd = T(1) / Hd;
  const uint32_t lc = lcount[i];
  const int cnt = list_cnt(lc), n_in = list_in(lc);
  const T Hs = (lc & kFastBit) ? screen_radius<T>(Hd) : Hd, Hs2 = Hs * Hs;
  T acc = 0;
  auto loop = [&](auto fastc) {
    constexpr bool FAST = decltype(fastc)::value;
    for (int k = 0; k < cnt; ++k) {
      const uint32_t e = list[list_row(k, n_in, cap) * n + i];
      const VT vj = view[e >> 8];
      T dx = vd<FAST>(F, vi.x, vj.x), dy = vd<FAST>(F, vi.y, vj.y);
      T dz = D == 3 ? vd<FAST>(F, vi.z, vj.z) : T(0);
      T r2 = dx * dx + dy * dy + dz * dz;
      if (r2 < Hs2) {
        if (FAST) {
          dx = vd<false>(F, vi.x, vj.x);
          dy = vd<false>(F, vi.y, vj.y);
          dz = D == 3 ? vd<false>(F, vi.z, vj.z) : T(0);
          r2 = dx * dx + dy * dy + dz * dz;
          if (!(r2 < Hd2)) continue;
        }
        const T q = r2 > T(0) ? pair_r<T>(r2) * invHd : T(0);
        const T u = T(1) - q, u2 = u * u;
        acc += u2 * u2 * (T(1) + T(4) * q);
      }
    }
  };
  if (lc & kFastBit) loop(std::true_type{});
  else loop(std::false_type{});
  const T Hphys = Hd * F.qv;
  const T rho = acc * P.alpha / (D == 2 ? Hphys * Hphys : Hphys * Hphys * Hphys);
  const T irt2 = inv_rho_t2<D, T>(hv * F.qv, P.inv_tau);
  const T rt = T(1) / dsqrt(irt2);
  rho_out[i] = rho;
  pc_out[i] = P.P0 * (T)pow((double)(rho / rt), (double)P.gamma) / (rho * rho);
}

// --------------------------------------------------------------------------
// Pass A (Algorithm 1: velocity reset, forces, first time step): per target i,
// over its listed j
//   rho_i = sum_j W(r_ij, h_i)                                 (Eq. density_sum)
//   a_i   = -sum_j [(P_i + P_j) + beta_ij P0 (1/rho_t,i^2 + 1/rho_t,j^2)]
//                  dW(r_ij, h_ij)/dr e_ij                      (Eqs. sph_pressure_force_2,
//                                                                   sph_st_force, sph_st_beta)
// with P = P0/rho_t^2 at gamma = 2 (Eq. EOS_2) or p/rho^2 otherwise;
// e_ij = (r_i - r_j)/r_ij, h_ij = (h_i + h_j)/2, and for the Wendland C2 kernel
// of support H: dW/dr e_ij = -20 alpha (1 - q)^3 (r_i - r_j) / H^(D+2).
// Writes a_i and g_i = 0.05 rho_t,i r_c,i |a_i| (eta_i = dt1 g_i, Eq.
// viscosity_coefficient with v~ = a dt1 / 2); FP64 block partials of
// min r_c/|a|, max |a|, sum rho, sum (rho/rho_t - 1)^2, max |rho/rho_t - 1|,
// pair counts; the last block reduces them in fixed order and sets dt1, dt2
// (Eq. time_step_size, see below).
// --------------------------------------------------------------------------
template <int D, class T, bool GENERAL, bool DBG, bool SURF, int NT, bool STG = false>
__global__ void __launch_bounds__(NT, (sizeof(T) == 8 ? SPH_PASS_MIN_BLOCKS_FP64 : SPH_PASS_MIN_BLOCKS) * 256 / NT) k_pass_a(int n, StepCtl* ctl,
                                                const typename ViewOf<T>::type* __restrict__ v0,
                                                const typename ViewOf<T>::type* __restrict__ v1,
                                                const uint32_t* __restrict__ m0, const uint32_t* __restrict__ m1,
                                                const uint32_t* __restrict__ p0, const uint32_t* __restrict__ p1,
                                                const uint32_t* __restrict__ list,
                                                const uint32_t* __restrict__ lcount, int cap, Frame<T> F,
                                                Phys<T> P, const T* __restrict__ pc, V4<T>* __restrict__ acc_out,
                                                T* __restrict__ rho_out, Partial* __restrict__ partials,
                                                Scalars* __restrict__ scal, unsigned* __restrict__ ticket,
                                                int* __restrict__ err, int advance, int* __restrict__ dbg_count,
                                                long long* __restrict__ dbg_sum, uint32_t* __restrict__ plist,
                                                uint32_t* __restrict__ pcount, const double* __restrict__ dt_fix,
                                                double* __restrict__ dt_rec, const LL4* __restrict__ X0,
                                                const LL4* __restrict__ X1, Geom<T> geo,
                                                const uint32_t* __restrict__ llist, const int* __restrict__ scount,
                                                const int* __restrict__ sj, const int4* __restrict__ v32,
                                                Frame<float> F32) {
  using VT = typename ViewOf<T>::type;
  static_assert(!STG || (std::is_same<T, float>::value && !GENERAL && !DBG && !SURF && NT == kStageBlock),
                "staged pass A: FP32, gamma = 2, 256-target blocks");
  __shared__ Partial sm[8];
  __shared__ bool last;
  extern __shared__ __align__(16) unsigned char stage_smem[];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const StepCtl cc = *ctl;
  const long long step = cc.step;
  const int buf = cc.buf;
  const VT* __restrict__ view = cc.vp ? v1 : v0;
  const T sigma = (T)sigma_of(cc, step);
  Partial part{DBL_MAX, 0.0, 0.0, 0.0, 0.0, 0, 0, 0, -1};
  // staged block: this step's views of its neighbour set into shared memory
  bool staged = false;
  const int* __restrict__ sjb = nullptr;
  VT* sview = reinterpret_cast<VT*>(stage_smem);
  if constexpr (STG) {
    const int m = min(scount[blockIdx.x], kStageCap);
    staged = m >= 0;
    if (staged) {
      sjb = sj + (size_t)blockIdx.x * kStageCap;
      for (int k = threadIdx.x; k < m; k += NT) cp_async16(sview + k, view + min(__ldg(sjb + k), n - 1));
      cp_async_wait_all();
    }
    __syncthreads();
  }
  if (i < n) {
    const uint32_t* __restrict__ pid = buf ? p1 : p0;
    const VT vi = view[i];
    const uint32_t* __restrict__ meta = buf ? m1 : m0;
    const uint32_t mi = meta[i];
    const uint32_t ci = mi & 0xFFu;
    // a feature-surface particle (Sec. 3.5) takes forces from surface particles
    // only (SURF: the variant launched when the handle has any)
    const bool surf = SURF && (mi & kSurfaceBit) != 0;
    const T hv = view_h(vi);
    const T qv = F.qv;
    const T Hd = P.kappa * hv, Hd2 = Hd * Hd, invHd = T(1) / Hd;
    const T inv_tau_v = P.inv_tau * qv;           // h in view units -> (h/tau)
    const T qi = inv_rho_t2<D, T>(hv, inv_tau_v);  // 1/rho_t,i^2
    const T Pi = GENERAL ? pc[i] : P.P0 * qi;
    const T sP0 = sigma * P.P0;
    const T half_kappa = T(0.5) * P.kappa;
    T dsum = 0, ax = 0, ay = 0, az = 0;
    int nf = 0, ni = 0, nd = 0;
    long long sd = 0, sf = 0;
    const uint32_t lc = lcount[i];
    const int cnt = list_cnt(lc);
    // Every skin-list entry: a screening test on the coarse vectors (when the
    // list build certified them), then the exact vectors and criteria for the
    // pairs that pass. This step's force pairs go to column i of plist.
    // FP64 path with current FP32 views: the screen in FP32 (for_skin_list_s32)
    constexpr bool S32_OK = std::is_same<T, double>::value && !GENERAL && !DBG && !SURF;
    auto loop = [&](auto fastc, auto stagedc, auto s32c) {
      constexpr bool FAST = decltype(fastc)::value;
      constexpr bool ST = decltype(stagedc)::value;  // e = (rank << 8 | colour), view from shared memory
      constexpr bool S32 = decltype(s32c)::value;    // entries arrive screened on the FP32 views
      auto pair = [&](uint32_t e, const VT& vj) {
        const int j = ST ? -1 : (int)(e >> 8);  // global index (unstaged entries)
        const bool self = ST ? (e & kStageSelf) != 0 : j == i;
        T dx = vd<FAST>(F, vi.x, vj.x), dy = vd<FAST>(F, vi.y, vj.y);
        T dz = D == 3 ? vd<FAST>(F, vi.z, vj.z) : T(0);
        T r2 = dx * dx + dy * dy + dz * dz;
        const T hj = view_h(vj);
        const T Hf = half_kappa * (hv + hj);
        if (FAST) {
          const T Hm = screen_radius<T>(GENERAL || Hf > Hd ? Hf : Hd);
          if (!(r2 < Hm * Hm)) return;
          dx = vd<false>(F, vi.x, vj.x);
          dy = vd<false>(F, vi.y, vj.y);
          dz = D == 3 ? vd<false>(F, vi.z, vj.z) : T(0);
          r2 = dx * dx + dy * dy + dz * dz;
        }
        const bool inD = !GENERAL && r2 < Hd2;
        const bool inF = r2 < Hf * Hf && !self && (!surf || (meta[j] & kSurfaceBit));
        if (!(inD || inF)) return;
        const T r = r2 > T(0) ? pair_r<T>(r2) : T(0);
        if (inD) {
          const T q = r * invHd;
          const T u = T(1) - q, u2 = u * u;
          dsum += u2 * u2 * (T(1) + T(4) * q);
          if (DBG) {
            ++nd;
            sd += pid[j];
          }
        }
        if (inF) {
          const T invH = drcp<T>(Hf);
          const T q = r * invH;
          const T u = T(1) - q;
          const T invH2 = invH * invH;
          const T w = u * u * u * (D == 2 ? invH2 * invH2 : invH2 * invH2 * invH);
          const T qj = inv_rho_t2<D, T>(hj, inv_tau_v);
          const T Pj = GENERAL ? pc[j] : P.P0 * qj;
          const bool other = (e & 0xFFu) != ci;
          const T coef = (Pi + Pj) + (other ? sP0 * (qi + qj) : T(0));
          const T s = coef * w;
          ax += s * dx;
          ay += s * dy;
          az += s * dz;
          // this step's force pairs (global index | colour), for pass B
          const uint32_t eg = ST ? ((uint32_t)__ldg(sjb + stage_rank(e)) << 8) | (e & 0xFFu) : e;
          SPH_PLIST_STORE(plist + (size_t)nf * n + i, eg);
          ++nf;
          ni += other;
          if (DBG) sf += pid[j];
        }
      };
      if constexpr (ST) {
        for_staged_list(llist, (const VT*)sview, n, i, lc, cap, pair);
      } else if constexpr (S32) {
        const int4 wi = v32[i];
        const float hv32 = __int_as_float(wi.w), hk32 = 0.5f * (float)P.kappa, Hd32 = (float)P.kappa * hv32;
        auto screen = [&](const int4& w) {
          const float cx = vd<true>(F32, wi.x, w.x), cy = vd<true>(F32, wi.y, w.y);
          const float cz = D == 3 ? vd<true>(F32, wi.z, w.z) : 0.0f;
          const float Hf32 = hk32 * (hv32 + __int_as_float(w.w));
          const float Hm = screen_radius<float>(Hf32 > Hd32 ? Hf32 : Hd32);
          return cx * cx + cy * cy + cz * cz < Hm * Hm;
        };
        for_skin_list_s32(list, v32, view, n, i, lc, cap, screen, pair);
      } else {
        for_skin_list(list, view, n, i, lc, cap, pair);
      }
    };
    if (STG && staged) {
      if (lc & kFastBit) loop(std::true_type{}, std::integral_constant<bool, STG>{}, std::false_type{});
      else loop(std::false_type{}, std::integral_constant<bool, STG>{}, std::false_type{});
    } else if (S32_OK && v32 && (lc & kFastBit)) {
      loop(std::false_type{}, std::false_type{}, std::integral_constant<bool, S32_OK>{});
    } else {
      if (lc & kFastBit) loop(std::true_type{}, std::false_type{}, std::false_type{});
      else loop(std::false_type{}, std::false_type{}, std::false_type{});
    }
    pcount[i] = (uint32_t)nf;
    // back to physical units: rho ~ 1/H^D, a ~ (view length)^-(D+1)
    const T Hphys = Hd * qv;
    const T rho = GENERAL ? rho_out[i] : dsum * P.alpha / (D == 2 ? Hphys * Hphys : Hphys * Hphys * Hphys);
    const T iq = F.inv_qv;
    const T k20 = T(20) * P.alpha * (D == 2 ? iq * iq * iq : iq * iq * iq * iq);
    ax *= k20;
    ay *= k20;
    az *= k20;
    if (surf) {  // Eq. force_surface: the normal component is dropped
      T xa[3], N[3];
      abs_pos<D, T>(F, (buf ? X1 : X0)[i], xa);
      surface_normal(geo, xa, D, N);
      const T dn = ax * N[0] + ay * N[1] + az * N[2];
      ax -= dn * N[0];
      ay -= dn * N[1];
      az -= dn * N[2];
    }
    const T an = dsqrt(ax * ax + ay * ay + az * az);
    const T rt = T(1) / dsqrt(qi);
    const T rc = Hphys;
    const T g = T(0.05) * rt * rc * an;
    acc_out[i] = V4<T>{ax, ay, az, g};
    if (!GENERAL && rho_out) rho_out[i] = rho;
    const double e = (double)rho / (double)rt - 1.0;
    part.min_rc_a = an > T(0) ? (double)rc / (double)an : DBL_MAX;
    part.amin = an > T(0) ? (long long)i : -1;
    part.max_a = (double)an;
    part.sum_rho = (double)rho;
    part.err_l2 = e * e;
    part.err_max = fabs(e);
    part.ipairs = ni;
    part.fpairs = nf;
    part.lentries = cnt;
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
  // last block: fixed-order reduction of every block partial (L2 reads)
  __threadfence();
  Partial acc{DBL_MAX, 0.0, 0.0, 0.0, 0.0, 0, 0, 0, -1};
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
    const double* qd = (const double*)&partials[b];
    const long long* ql = (const long long*)&partials[b];
    argmin_merge(acc.min_rc_a, acc.amin, __ldcg(qd + 0), __ldcg(ql + 8));
    acc.max_a = fmax(acc.max_a, __ldcg(qd + 1));
    acc.sum_rho += __ldcg(qd + 2);
    acc.err_l2 += __ldcg(qd + 3);
    acc.err_max = fmax(acc.err_max, __ldcg(qd + 4));
    acc.ipairs += __ldcg(ql + 5);
    acc.fpairs += __ldcg(ql + 6);
    acc.lentries += __ldcg(ql + 7);
  }
  acc = block_reduce(acc, sm);
  if (threadIdx.x == 0) {
    // Eq. time_step_size with v_n = 0 (the velocity reset of Algorithm 1): the
    // first time step keeps only the body-force term, dt1 = min_i 0.25
    // sqrt(r_c,i/|a_i|). With v~_i = a_i dt1/2 and nu_i = 0.1 r_c,i |v~_i|, the
    // second time step's terms are
    // r_c/(40|v~|) = m/(20 dt1) and 0.125 r_c^2/nu = 2.5 m/dt1, m = min r_c/|a|
    // (all three are monotone in r_c,i/|a_i|, so their minima share the argmin).
    const double m = acc.min_rc_a;
    double dt1 = 0.0, dt2 = 0.0;
    if (m < DBL_MAX) {
      dt1 = 0.25 * sqrt(m);
      dt2 = fmin(dt1, fmin(m / (20.0 * dt1), 2.5 * m / dt1));
    }
    if (dt_fix) {  // prescribed step sizes
      dt1 = dt_fix[0];
      dt2 = dt_fix[1];
    }
    if (dt_rec) {
      dt_rec[0] = dt1;
      dt_rec[1] = dt2;
    }
    // the step-size history of a reverse-pass run: replay or record
    const long long hk = step - cc.dt_base;
    if (cc.dt_mode && cc.dt_hist && hk >= 0 && hk < cc.dt_len) {
      if (cc.dt_mode == 2) {
        dt1 = cc.dt_hist[2 * hk];
        dt2 = cc.dt_hist[2 * hk + 1];
      } else {
        cc.dt_hist[2 * hk] = dt1;
        cc.dt_hist[2 * hk + 1] = dt2;
      }
    }
    scal->dt1 = dt1;
    scal->dt2 = dt2;
    scal->min_rc_a = m;
    scal->argmin = acc.amin;
    scal->max_a = acc.max_a;
    scal->sum_rho = acc.sum_rho;
    scal->err_l2 = acc.err_l2;
    scal->err_max = acc.err_max;
    scal->sigma = (double)sigma;
    scal->ipairs = acc.ipairs / 2;
    scal->fpairs = acc.fpairs / 2;
    scal->lentries = acc.lentries;
    scal->wall_moved = 0;
    scal->step_of_stats = step;
    if (advance && cc.auto_on && !cc.auto_done) {
      // convergence of the partition (Sec. 3.3): the interface-pair count stays
      // within auto_tol of the count that opened the run for auto_window steps;
      // then the ramp of Eq. sph_st_sigma starts: t0 = this step, t1 = (1 + theta) t0
      const long long ip = acc.ipairs / 2;
      long long ref = cc.auto_ref;
      int stable = cc.auto_stable;
      if (ref >= 0 && fabs((double)(ip - ref)) <= cc.auto_tol * (double)ref) {
        ++stable;
      } else {
        ref = ip;
        stable = 0;
      }
      ctl->auto_ref = ref;
      ctl->auto_stable = stable;
      if (stable >= cc.auto_window) {
        ctl->t0 = (double)step;
        ctl->t1 = (1.0 + cc.auto_theta) * (double)step;
        ctl->auto_done = 1;
      }
    }
    if (advance) ctl->step = step + 1;
    *ticket = 0u;
  }
}

// --------------------------------------------------------------------------
// Pass B (Algorithm 1: viscous force, kicks, drift, projection): viscous force (Eq. sph_viscous_force with
// rho := rho_t, Eq. sph_viscous_force_2), the kicks and the drift
// (Eqs. time_int_01..03) and the level-set projection (Eq. displacement_surface).
// With v~ = a dt1/2 and eta = dt1 g:
//   a~_i = (dt1^2 / 2) B_i,
//   B_i  = sum_j HM(g_i, g_j) (1/rho_t,i^2 + 1/rho_t,j^2) (dW/dr / r)(a_i - a_j),
//   v_i  = dt1 a_i / 2 + dt2 a~_i / 2,   r_i += v_i dt2.
// The new view goes to the other view buffer; a particle that moved half its
// skin since the list was built raises need_rebuild.
// --------------------------------------------------------------------------
template <int D, class T, int NT>
__global__ void __launch_bounds__(NT, (sizeof(T) == 8 ? SPH_PASSB_MIN_BLOCKS_FP64 : SPH_PASSB_MIN_BLOCKS) * 256 / NT) k_pass_b(int n, StepCtl* __restrict__ ctl,
                                                const typename ViewOf<T>::type* __restrict__ v0,
                                                const typename ViewOf<T>::type* __restrict__ v1,
                                                typename ViewOf<T>::type* __restrict__ w0,
                                                typename ViewOf<T>::type* __restrict__ w1,
                                                const typename ViewOf<T>::type* __restrict__ vbuild,
                                                LL4* __restrict__ X0, LL4* __restrict__ X1,
                                                const uint32_t* __restrict__ plist,
                                                const uint32_t* __restrict__ pcount,
                                                const V4<T>* __restrict__ acc, Frame<T> F, Phys<T> P, Geom<T> geo,
                                                const Scalars* __restrict__ scal, V4<T>* __restrict__ visc_out,
                                                int* __restrict__ err, unsigned long long* __restrict__ wall_moved,
                                                int move, const uint32_t* __restrict__ m0,
                                                const uint32_t* __restrict__ m1, int4* __restrict__ v32out,
                                                int sv32) {
  using VT = typename ViewOf<T>::type;
  __shared__ int moved_sm[8];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int vp = ctl->vp, buf = ctl->buf;
  int moved = 0, far = 0;
  if (i < n) {
    const VT* __restrict__ view = vp ? v1 : v0;
    const VT vi = view[i];
    const T hv = view_h(vi);
    const T qv = F.qv;
    const T inv_tau_v = P.inv_tau * qv;
    const T qi = inv_rho_t2<D, T>(hv, inv_tau_v);
    const V4<T> ai = acc[i];
    const T half_kappa = T(0.5) * P.kappa;
    T bx = 0, by = 0, bz = 0;
    // this step's pairs as pass A compacted them (same positions); the force
    // support is tested again on the exact vectors
    const int cnt = (int)pcount[i];
    for_list_x(plist, view, n, i, cnt, [&](int j) { return acc[j]; }, [&](uint32_t e, const VT& vj, const V4<T>& aj) {
      const int j = (int)(e >> 8);
      const T dx = vd<false>(F, vi.x, vj.x), dy = vd<false>(F, vi.y, vj.y);
      const T dz = D == 3 ? vd<false>(F, vi.z, vj.z) : T(0);
      const T r2 = dx * dx + dy * dy + dz * dz;
      const T hj = view_h(vj);
      const T Hf = half_kappa * (hv + hj);
      if (!(r2 < Hf * Hf) || j == i) return;
      const T gs = ai.w + aj.w;
      const T hm = gs > T(0) ? T(2) * ai.w * aj.w * drcp<T>(gs) : T(0);
      const T invH = drcp<T>(Hf);
      const T q = r2 > T(0) ? pair_r<T>(r2) * invH : T(0);
      const T u = T(1) - q;
      const T invH2 = invH * invH;
      const T w = u * u * u * (D == 2 ? invH2 * invH2 : invH2 * invH2 * invH);
      const T s = hm * (qi + inv_rho_t2<D, T>(hj, inv_tau_v)) * w;
      bx += s * (ai.x - aj.x);
      by += s * (ai.y - aj.y);
      bz += s * (ai.z - aj.z);
    });
    // dW/dr / r = -20 alpha (1-q)^3 / H^(D+2); view lengths -> physical
    const T iq = F.inv_qv;
    const T km = T(-20) * P.alpha * (D == 2 ? iq * iq * iq * iq : iq * iq * iq * iq * iq);
    bx *= km;
    by *= km;
    bz *= km;
    const bool surf = ((buf ? m1 : m0)[i] & kSurfaceBit) != 0;
    if (surf) {  // Eq. force_surface for the viscous force too
      T xs[3], N[3];
      abs_pos<D, T>(F, (buf ? X1 : X0)[i], xs);
      surface_normal(geo, xs, D, N);
      const T dn = bx * N[0] + by * N[1] + bz * N[2];
      bx -= dn * N[0];
      by -= dn * N[1];
      bz -= dn * N[2];
    }
    const T dt1 = (T)scal->dt1, dt2 = (T)scal->dt2;
    const T kv = T(0.5) * dt1 * dt1;  // a~ = kv B
    // a~ for the caller when asked (a run-time test: one compiled kernel, so
    // recording cannot change the arithmetic of the step)
    if (visc_out) visc_out[i] = V4<T>{kv * bx, kv * by, kv * bz, T(0)};
    if (move) {
    T d[3];
    d[0] = (T(0.5) * dt1 * ai.x + T(0.5) * dt2 * kv * bx) * dt2;
    d[1] = (T(0.5) * dt1 * ai.y + T(0.5) * dt2 * kv * by) * dt2;
    d[2] = D == 3 ? (T(0.5) * dt1 * ai.z + T(0.5) * dt2 * kv * bz) * dt2 : T(0);
    LL4* __restrict__ Xs = buf ? X1 : X0;
    LL4 X = Xs[i];
    const bool finite = isfinite((double)d[0]) && isfinite((double)d[1]) && isfinite((double)d[2]);
    if (!finite) atomicOr(err, kErrNonfinite);
    if (finite) {
      long long* Xc[3] = {&X.x, &X.y, &X.z};
      for (int k = 0; k < D; ++k) {
        long long v = *Xc[k] + state_units(d[k] * F.inv_q64t);
        // bounding box (first constraint): clamp, the closest point
        if (v < 0) { v = 0; moved |= !surf; }
        if (v > F.xmax[k]) { v = F.xmax[k]; moved |= !surf; }
        *Xc[k] = v;
      }
      // shape constraints, in order, at the absolute position; a feature-surface
      // particle goes onto the surface it belongs to instead (Eq. displacement_surface)
      T xa[3];
      abs_pos<D, T>(F, X, xa);
      int mv = 0;
      if (surf) {
        project_to_surface(geo, xa, D);
        mv = 1;
      } else {
        for (int s = 0; s < geo.n_shapes; ++s) mv |= project_shape(geo, s, xa, D);
        moved |= mv;
      }
      if (mv) {
        for (int k = 0; k < D; ++k) {
          long long v = state_units((xa[k] - F.lo[k]) * F.inv_q64t);
          v = v < 0 ? 0 : (v > F.xmax[k] ? F.xmax[k] : v);
          *Xc[k] = v;
        }
        abs_pos<D, T>(F, X, xa);
      }
      Xs[i] = X;
      // smoothing length at the new position (the target field of the next step)
      const T hn = h_of<D, T>(geo, xa);
      const VT vn = make_view<D>(F, X, hn);
      (vp ? w0 : w1)[i] = vn;
      if (v32out) {  // FP64 path: its FP32 view of the next step (as k_view32 makes it)
        const long long half = 1LL << (sv32 - 1);
        v32out[i] = make_int4((int)((X.x + half) >> sv32), (int)((X.y + half) >> sv32),
                              D == 3 ? (int)((X.z + half) >> sv32) : 0, __float_as_int((float)view_h(vn)));
      }
      // skin test against the view at list build
      const VT vb = vbuild[i];
      const T ex = vd<false>(F, vn.x, vb.x), ey = vd<false>(F, vn.y, vb.y);
      const T ez = D == 3 ? vd<false>(F, vn.z, vb.z) : T(0);
      const T lim = view_h(vb);
      far = (ex * ex + ey * ey + ez * ez) >= lim * lim;
    } else {
      (vp ? w0 : w1)[i] = vi;
    }
    }  // move
  }
  if (__syncthreads_or(far) && threadIdx.x == 0) ctl->need_rebuild = 1;
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
                                                   const uint8_t* __restrict__ col, Frame<T> F,
                                                   LL4* __restrict__ X0, uint32_t* __restrict__ meta0,
                                                   uint32_t* __restrict__ pid0, int* __restrict__ err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  long long v[3] = {0, 0, 0};
  for (int k = 0; k < D; ++k) {
    const double x = xyz[(size_t)i * D + k];
    if (!isfinite(x)) {
      atomicOr(err, kErrNonfinite);
      continue;
    }
    const double u = (x - F.lod[k]) * F.inv_q64;
    if (u < 0.0 || u > (double)F.xmax[k] + 0.5) atomicOr(err, kErrOutOfDomain);
    long long w = (long long)llrint(u < 0.0 ? 0.0 : (u > (double)F.xmax[k] ? (double)F.xmax[k] : u));
    v[k] = w;
  }
  X0[i] = LL4{v[0], v[1], v[2], 0};
  meta0[i] = (uint32_t)col[i];
  pid0[i] = (uint32_t)i;
}

template <int D, class T>
__global__ void __launch_bounds__(256) k_get_positions(int n, const StepCtl* __restrict__ ctl,
                                                       const LL4* __restrict__ X0, const LL4* __restrict__ X1,
                                                       const uint32_t* __restrict__ p0,
                                                       const uint32_t* __restrict__ p1, Frame<T> F,
                                                       double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int buf = ctl->buf;
  const LL4 X = (buf ? X1 : X0)[i];
  const uint32_t id = (buf ? p1 : p0)[i];
  out[(size_t)id * D + 0] = F.lod[0] + (double)X.x * F.q64;
  out[(size_t)id * D + 1] = F.lod[1] + (double)X.y * F.q64;
  if (D == 3) out[(size_t)id * D + 2] = F.lod[2] + (double)X.z * F.q64;
}

// which: 0 rho (n), 1 acc (n x D), 2 visc (n x D); source arrays in the current order
template <int D, class T>
__global__ void __launch_bounds__(256) k_get_fields(int n, int which, const StepCtl* __restrict__ ctl,
                                                    const uint32_t* __restrict__ p0,
                                                    const uint32_t* __restrict__ p1, const T* __restrict__ rho,
                                                    const V4<T>* __restrict__ acc, const V4<T>* __restrict__ visc,
                                                    double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t id = (ctl->buf ? p1 : p0)[i];
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
cudaError_t launch_rebuild(const DevState& S, const Grid<T>& G, const Frame<T>& F, const Geom<T>& g, T kappa,
                           cudaStream_t st, const Grid<float>* G32, const Frame<float>* F32) {
  using VT = typename ViewOf<T>::type;
  // the cheap per-particle kernels on a capped grid (an idle launch costs a
  // few us); the list build on one block per 256 targets: a grid capped at
  // 16 or 32 blocks per SM made its rebuilds of the 8M 3D workload slower
  // (cells 2.01 / 1.93 vs 1.86 ms per step), its blocks no longer finishing
  // and refilling the SMs independently
  const int tb = 256, gb = rebuild_grid(S.n, tb, 8), gl = grid_for(S.n, tb);
  const LL4* X0 = (const LL4*)S.X[0];
  const LL4* X1 = (const LL4*)S.X[1];
  k_rekey<D, T><<<gb, tb, 0, st>>>(S.n, S.ctl, X0, X1, F, G, g, S.key);
#define SPH_LIST_BUILD(TT) k_list_build<D, TT><<<gl, tb, 0, st>>>
  cudaError_t e = build_cells(S, st);
  if (e != cudaSuccess) return e;
  k_make_view<D, T><<<gb, tb, 0, st>>>(S.n, S.ctl, 0, X0, X1, F, g, (VT*)S.view[0], (VT*)S.view[1],
                                       (VT*)S.vbuild);
  if constexpr (std::is_same<T, double>::value) {
    // the FP64 path lists its pairs through an FP32 view (same frame origin,
    // same cells, same list format)
    if (!S.view32 || !F32 || !G32) return cudaErrorInvalidValue;
    k_view32<D><<<gb, tb, 0, st>>>(S.n, S.ctl, X0, X1, *F32, (const V4<double>*)S.view[0],
                                   (const V4<double>*)S.view[1], (int4*)S.view32);
    SPH_LIST_BUILD(float)(S.n, S.ctl, X0, X1, S.meta[0], S.meta[1], (const int4*)S.view32,
                          (const int4*)S.view32, S.cstart, *F32, *G32, (float)kappa, S.cap, S.list, S.lcount,
                          S.err);
  } else {
    SPH_LIST_BUILD(T)(S.n, S.ctl, X0, X1, S.meta[0], S.meta[1], (const VT*)S.view[0], (const VT*)S.view[1],
                      S.cstart, F, G, kappa, S.cap, S.list, S.lcount, S.err);
    if (S.stage && S.llist)
      k_stage<D><<<grid_for(S.n, kStageBlock), kStageBlock, 0, st>>>(S.n, S.ctl, S.list, S.lcount, S.cap, S.llist,
                                                                  S.scount, S.sj);
  }
#undef SPH_LIST_BUILD
  return cudaGetLastError();
}

template <int D, class T>
cudaError_t launch_pass_a(const DevState& S, const Frame<T>& F, const Phys<T>& P, PassFlags f, cudaStream_t st) {
  using VT = typename ViewOf<T>::type;
  Geom<T> geo{};
  if (f.geo) geo = *(const Geom<T>*)f.geo;
  const int tb = S.pass_threads == 128 ? 128 : 256, gb = grid_for(S.n, tb);
  T* rho = (T*)S.rho;
  T* pc = (T*)S.pc;
  // the FP64 path screens on its FP32 views when the caller passes their frame
  const bool s32 = std::is_same<T, double>::value && S.view32 && f.f32;
  const int4* v32 = s32 ? (const int4*)S.view32 : nullptr;
  const Frame<float> f32 = s32 ? *f.f32 : Frame<float>{};
  if (f.general_eos)
    k_density<D, T><<<grid_for(S.n, 256), 256, 0, st>>>(S.n, S.ctl, (const VT*)S.view[0], (const VT*)S.view[1],
                                                        S.list, S.lcount, S.cap, F, P, rho, pc);
#define SPH_PASS_A_NT(GEN, DBG, NT)                                                                             \
  (f.surface ? k_pass_a<D, T, GEN, DBG, true, NT> : k_pass_a<D, T, GEN, DBG, false, NT>)<<<gb, tb, 0, st>>>(    \
                                              S.n, S.ctl, (const VT*)S.view[0], (const VT*)S.view[1],           \
                                              S.meta[0], S.meta[1], S.pid[0], S.pid[1], S.list, S.lcount, S.cap, \
                                              F, P,                                                             \
                                              pc, (V4<T>*)S.acc4, rho, S.partials, S.scal, S.tickets, S.err,   \
                                              f.advance, S.dbg_count, S.dbg_sum, S.plist, S.pcount, f.dt_fix,     \
                                              f.dt_rec, (const LL4*)S.X[0], (const LL4*)S.X[1], geo, S.llist,     \
                                              S.scount, S.sj, v32, f32)
#define SPH_PASS_A(GEN, DBG)           \
  do {                                 \
    if (tb == 128)                     \
      SPH_PASS_A_NT(GEN, DBG, 128);    \
    else                               \
      SPH_PASS_A_NT(GEN, DBG, 256);    \
  } while (0)
  if constexpr (std::is_same<T, float>::value) {
    if (staged_pass(S, f)) {
      k_pass_a<D, float, false, false, false, kStageBlock, true>
          <<<grid_for(S.n, kStageBlock), kStageBlock, kStageCap * sizeof(int4), st>>>(
              S.n, S.ctl, (const int4*)S.view[0], (const int4*)S.view[1], S.meta[0], S.meta[1], S.pid[0], S.pid[1],
              S.list, S.lcount, S.cap, F, P, pc, (V4<float>*)S.acc4, rho, S.partials, S.scal, S.tickets, S.err,
              f.advance, S.dbg_count, S.dbg_sum, S.plist, S.pcount, f.dt_fix, f.dt_rec, (const LL4*)S.X[0],
              (const LL4*)S.X[1], geo, S.llist, S.scount, S.sj, nullptr, Frame<float>{});
      return cudaGetLastError();
    }
  }
  if (f.general_eos) {
    if (f.nbr_debug) SPH_PASS_A(true, true);
    else SPH_PASS_A(true, false);
  } else {
    if (f.nbr_debug) SPH_PASS_A(false, true);
    else SPH_PASS_A(false, false);
  }
#undef SPH_PASS_A
#undef SPH_PASS_A_NT
  return cudaGetLastError();
}

template <int D>
cudaError_t prepare_staged_pass() {
  static cudaError_t e = cudaFuncSetAttribute(k_pass_a<D, float, false, false, false, kStageBlock, true>,
                                              cudaFuncAttributePreferredSharedMemoryCarveout,
                                              (int)cudaSharedmemCarveoutMaxShared);
  return e;
}

template <int D, class T>
cudaError_t launch_pass_b(const DevState& S, const Frame<T>& F, const Phys<T>& P, const Geom<T>& g, PassFlags f,
                          cudaStream_t st) {
  using VT = typename ViewOf<T>::type;
  const int tb = S.pass_threads == 128 ? 128 : 256, gb = grid_for(S.n, tb);
  unsigned long long* wm = (unsigned long long*)&S.scal->wall_moved;
  (tb == 128 ? k_pass_b<D, T, 128> : k_pass_b<D, T, 256>)<<<gb, tb, 0, st>>>(
      S.n, S.ctl, (const VT*)S.view[0], (const VT*)S.view[1], (VT*)S.view[0], (VT*)S.view[1], (const VT*)S.vbuild,
      (LL4*)S.X[0], (LL4*)S.X[1], S.plist, S.pcount, (const V4<T>*)S.acc4, F, P, g, S.scal,
      f.record ? (V4<T>*)S.visc : nullptr, S.err, wm, f.move, S.meta[0], S.meta[1],
      (std::is_same<T, double>::value && S.view32 && f.f32) ? (int4*)S.view32 : nullptr, f.f32 ? f.f32->sv : 0);
  return cudaGetLastError();
}

template <int D, class T>
cudaError_t launch_set_state(const DevState& S, const Frame<T>& F, const double* xyz, const uint8_t* col,
                             cudaStream_t st) {
  const int tb = 256, gb = grid_for(S.n, tb);
  if (S.n > 0)
    k_set_state<D, T><<<gb, tb, 0, st>>>(S.n, xyz, col, F, (LL4*)S.X[0], S.meta[0], S.pid[0], S.err);
  return cudaGetLastError();
}

template <int D, class T>
cudaError_t launch_get_positions(const DevState& S, const Frame<T>& F, double* out, cudaStream_t st) {
  const int tb = 256, gb = grid_for(S.n, tb);
  if (S.n > 0)
    k_get_positions<D, T><<<gb, tb, 0, st>>>(S.n, S.ctl, (const LL4*)S.X[0], (const LL4*)S.X[1], S.pid[0],
                                             S.pid[1], F, out);
  return cudaGetLastError();
}

template <int D, class T>
cudaError_t launch_get_fields(const DevState& S, int which, double* out, cudaStream_t st) {
  const int tb = 256, gb = grid_for(S.n, tb);
  if (S.n > 0)
    k_get_fields<D, T><<<gb, tb, 0, st>>>(S.n, which, S.ctl, S.pid[0], S.pid[1], (const T*)S.rho,
                                          (const V4<T>*)S.acc4, (const V4<T>*)S.visc, out);
  return cudaGetLastError();
}

#define SPH_INSTANTIATE_STEP(D, T)                                                                             \
  template cudaError_t launch_rebuild<D, T>(const DevState&, const Grid<T>&, const Frame<T>&, const Geom<T>&, \
                                            T, cudaStream_t, const Grid<float>*, const Frame<float>*);        \
  template cudaError_t launch_pass_a<D, T>(const DevState&, const Frame<T>&, const Phys<T>&, PassFlags,       \
                                           cudaStream_t);                                                     \
  template cudaError_t launch_pass_b<D, T>(const DevState&, const Frame<T>&, const Phys<T>&, const Geom<T>&,  \
                                           PassFlags, cudaStream_t);                                          \
  template cudaError_t launch_set_state<D, T>(const DevState&, const Frame<T>&, const double*, const uint8_t*, \
                                              cudaStream_t);                                                  \
  template cudaError_t launch_get_positions<D, T>(const DevState&, const Frame<T>&, double*, cudaStream_t);   \
  template cudaError_t launch_get_fields<D, T>(const DevState&, int, double*, cudaStream_t);

}  // namespace sph
