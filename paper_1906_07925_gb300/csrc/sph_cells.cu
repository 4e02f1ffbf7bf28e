// Cell-linked list of the multi-resolution grid (the neighbour search of Algorithm 1).
//
// At a neighbour-list rebuild, particles are ordered by cell key with a
// counting sort over the dense key range: warp-aggregated atomic counts per
// cell, an exclusive scan of the counts (which is also the cell-start table the
// list build reads), an atomic scatter that counts each cell back down to zero,
// and a gather that orders each cell by particle id (so the order is a function
// of the keys alone: by key, then id) while it moves the particle state into
// the other buffer. Every
// kernel here returns at once on steps without a rebuild (ctl->rebuild == 0),
// so one captured graph serves every step.
#include "sph_internal.h"

namespace sph {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

__global__ void k_gate(StepCtl* __restrict__ ctl, int force) {
  StepCtl c = *ctl;
  c.vp ^= 1;
  if (c.need_rebuild || force) {
    c.rebuild = 1;
    c.buf ^= 1;
    c.need_rebuild = 0;
    c.rebuilds += 1;
    c.lmax = 0;
  } else {
    c.rebuild = 0;
  }
  *ctl = c;
}

__global__ void k_request_rebuild(StepCtl* __restrict__ ctl) { ctl->need_rebuild = 1; }
__global__ void k_write_ctl(StepCtl* __restrict__ ctl, StepCtl v) { *ctl = v; }

__global__ void __launch_bounds__(256) k_count(int n, const StepCtl* __restrict__ ctl, const uint32_t* __restrict__ key,
                                               uint32_t* __restrict__ cnt) {
  if (!ctl->rebuild) return;
  for (int b0 = blockIdx.x * blockDim.x; b0 < n; b0 += gridDim.x * blockDim.x) {
    const int i = b0 + threadIdx.x;
    const bool active = i < n;
    const unsigned mask = __ballot_sync(0xffffffffu, active);
    if (!active) continue;
    const uint32_t k = key[i];
    const unsigned peers = __match_any_sync(mask, k);
    const int leader = __ffs(peers) - 1;
    if ((int)(threadIdx.x & 31) == leader) atomicAdd(&cnt[k], (uint32_t)__popc(peers));
  }
}

__global__ void __launch_bounds__(256) k_scatter(int n, const StepCtl* __restrict__ ctl,
                                                 const uint32_t* __restrict__ key,
                                                 const uint32_t* __restrict__ cstart,
                                                 uint32_t* __restrict__ cnt,
                                                 uint32_t* __restrict__ slots) {
  if (!ctl->rebuild) return;
  for (int b0 = blockIdx.x * blockDim.x; b0 < n; b0 += gridDim.x * blockDim.x) {
    const int i = b0 + threadIdx.x;
    const bool active = i < n;
    const unsigned mask = __ballot_sync(0xffffffffu, active);
    if (!active) continue;
    const uint32_t k = key[i];
    const unsigned peers = __match_any_sync(mask, k);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(peers) - 1;
    uint32_t top = 0;
    if (lane == leader) top = atomicSub(&cnt[k], (uint32_t)__popc(peers));
    top = __shfl_sync(peers, top, leader);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    slots[cstart[k] + top - 1 - rank] = (uint32_t)i;
  }
}

// per block: sum of a tile of kScanTile counts
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const StepCtl* __restrict__ ctl,
                                                              const uint32_t* __restrict__ in,
                                                              uint32_t n, uint32_t* __restrict__ part) {
  if (!ctl->rebuild) return;
  __shared__ uint32_t red[kScanThreads / 32];
  size_t base = (size_t)blockIdx.x * kScanTile;
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    size_t idx = base + (size_t)k * kScanThreads + threadIdx.x;
    if (idx < n) s += in[idx];
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < kScanThreads / 32 ? red[threadIdx.x] : 0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
  }
}

// exclusive scan of the block sums, in place (one block of 1024 threads)
__global__ void __launch_bounds__(1024) k_scan_top(const StepCtl* __restrict__ ctl, uint32_t* __restrict__ part,
                                                   int nb) {
  if (!ctl->rebuild) return;
  __shared__ uint32_t wsum[32];
  int per = (nb + blockDim.x - 1) / blockDim.x;
  int b0 = threadIdx.x * per;
  uint32_t local = 0;
  for (int k = 0; k < per; ++k)
    if (b0 + k < nb) local += part[b0 + k];
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t incl = local;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) wsum[w] = incl;
  __syncthreads();
  if (w == 0) {
    uint32_t v = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
    uint32_t vi = v;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t u = __shfl_up_sync(0xffffffffu, vi, o);
      if (lane >= o) vi += u;
    }
    wsum[lane] = vi - v;
  }
  __syncthreads();
  uint32_t run = wsum[w] + incl - local;
  for (int k = 0; k < per; ++k)
    if (b0 + k < nb) {
      uint32_t v = part[b0 + k];
      part[b0 + k] = run;
      run += v;
    }
}

// exclusive scan of each tile plus its block offset; out has n + 1 entries
__global__ void __launch_bounds__(kScanThreads) k_scan_down(const StepCtl* __restrict__ ctl,
                                                            const uint32_t* __restrict__ in, uint32_t n,
                                                            const uint32_t* __restrict__ part,
                                                            uint32_t* __restrict__ out) {
  if (!ctl->rebuild) return;
  __shared__ uint32_t wtot[kScanThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  // each warp owns kScanItems * 32 consecutive entries of the tile
  size_t wbase = (size_t)blockIdx.x * kScanTile + (size_t)w * kScanItems * 32;
  uint32_t v[kScanItems];
  uint32_t run = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    size_t idx = wbase + (size_t)k * 32 + lane;
    uint32_t x = idx < n ? in[idx] : 0u;
    uint32_t incl = x;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    v[k] = run + incl - x;
    run += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (lane == 0) wtot[w] = run;
  __syncthreads();
  uint32_t off = part[blockIdx.x];
  for (int q = 0; q < w; ++q) off += wtot[q];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    size_t idx = wbase + (size_t)k * 32 + lane;
    if (idx < n) out[idx] = off + v[k];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == kScanThreads - 1) {
    uint32_t tot = part[blockIdx.x];
    for (int q = 0; q < kScanThreads / 32; ++q) tot += wtot[q];
    out[n] = tot;
  }
}

struct alignas(32) State64 {
  long long x, y, z, w;
};

// slot s of the scatter holds old index i; its rank among the cell's members by
// particle id gives its destination (cells ordered by key, each cell by
// particle id), where the state is copied
__global__ void __launch_bounds__(256) k_stable_gather(
    int n, const StepCtl* __restrict__ ctl, const uint32_t* __restrict__ slots, const uint32_t* __restrict__ key,
    const uint32_t* __restrict__ cstart, State64* __restrict__ X0, State64* __restrict__ X1,
    uint32_t* __restrict__ m0, uint32_t* __restrict__ m1, uint32_t* __restrict__ p0, uint32_t* __restrict__ p1) {
  if (!ctl->rebuild) return;
  const int nb = ctl->buf;  // new buffer; the old order lives in the other one
  const uint32_t* __restrict__ pold = nb ? p0 : p1;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
    const uint32_t i = slots[s];
    const uint32_t k = key[i];
    const uint32_t id = pold[i];
    const uint32_t b = cstart[k], e = cstart[k + 1];
    uint32_t rank = 0;
    for (uint32_t t = b; t < e; ++t) rank += pold[slots[t]] < id;
    const uint32_t d = b + rank;
    (nb ? X1 : X0)[d] = (nb ? X0 : X1)[i];
    (nb ? m1 : m0)[d] = (nb ? m0 : m1)[i];
    (nb ? p1 : p0)[d] = (nb ? p0 : p1)[i];
  }
}

// feature-surface flags by particle id into the current meta words (colours kept)
__global__ void __launch_bounds__(256) k_set_surface(int n, const StepCtl* __restrict__ ctl,
                                                     const uint32_t* __restrict__ p0, const uint32_t* __restrict__ p1,
                                                     uint32_t* __restrict__ m0, uint32_t* __restrict__ m1,
                                                     const uint8_t* __restrict__ flags) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int buf = ctl->buf;
  uint32_t* __restrict__ m = buf ? m1 : m0;
  const uint32_t id = (buf ? p1 : p0)[i];
  const uint32_t v = m[i] & ~kSurfaceBit;
  m[i] = (flags && flags[id]) ? (v | kSurfaceBit) : v;
}

__global__ void __launch_bounds__(256) k_get_colors(int n, const StepCtl* __restrict__ ctl,
                                                    const uint32_t* __restrict__ m0, const uint32_t* __restrict__ m1,
                                                    const uint32_t* __restrict__ p0, const uint32_t* __restrict__ p1,
                                                    uint8_t* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int buf = ctl->buf;
  if (i < n) out[(buf ? p1 : p0)[i]] = (uint8_t)((buf ? m1 : m0)[i] & 0xFFu);
}

}  // namespace

cudaError_t launch_gate(const DevState& S, int force, cudaStream_t st) {
  k_gate<<<1, 1, 0, st>>>(S.ctl, force);
  return cudaGetLastError();
}

cudaError_t launch_write_ctl(const DevState& S, const StepCtl& v, cudaStream_t st) {
  k_write_ctl<<<1, 1, 0, st>>>(S.ctl, v);
  return cudaGetLastError();
}

cudaError_t launch_request_rebuild(const DevState& S, cudaStream_t st) {
  k_request_rebuild<<<1, 1, 0, st>>>(S.ctl);
  return cudaGetLastError();
}

cudaError_t launch_set_surface(const DevState& S, const uint8_t* flags, cudaStream_t st) {
  if (S.n > 0)
    k_set_surface<<<(S.n + 255) / 256, 256, 0, st>>>(S.n, S.ctl, S.pid[0], S.pid[1], S.meta[0], S.meta[1], flags);
  return cudaGetLastError();
}

cudaError_t launch_get_colors(const DevState& S, uint8_t* out, cudaStream_t st) {
  if (S.n > 0)
    k_get_colors<<<(S.n + 255) / 256, 256, 0, st>>>(S.n, S.ctl, S.meta[0], S.meta[1], S.pid[0], S.pid[1], out);
  return cudaGetLastError();
}

cudaError_t build_cells(const DevState& S, cudaStream_t st) {
  const int n = S.n;
  if (n <= 0) return cudaSuccess;
  const int tb = 256;
  const int gb = rebuild_grid(n, tb, 8);
  k_count<<<gb, tb, 0, st>>>(n, S.ctl, S.key, S.cnt);
  const uint32_t m = S.total_cells;
  const int nb = (int)((m + kScanTile - 1) / kScanTile);
  k_scan_reduce<<<nb, kScanThreads, 0, st>>>(S.ctl, S.cnt, m, S.scan_part);
  k_scan_top<<<1, 1024, 0, st>>>(S.ctl, S.scan_part, nb);
  k_scan_down<<<nb, kScanThreads, 0, st>>>(S.ctl, S.cnt, m, S.scan_part, S.cstart);
  k_scatter<<<gb, tb, 0, st>>>(n, S.ctl, S.key, S.cstart, S.cnt, S.tmp);
  k_stable_gather<<<gb, tb, 0, st>>>(n, S.ctl, S.tmp, S.key, S.cstart, (State64*)S.X[0], (State64*)S.X[1],
                                     S.meta[0], S.meta[1], S.pid[0], S.pid[1]);
  return cudaGetLastError();
}

}  // namespace sph
