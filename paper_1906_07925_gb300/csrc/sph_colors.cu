// Per-colour volume of the partition (Sec. 2.1: the sub-domains are to be of
// equal size; Sec. 2.3, Eq. mass_for_partition: each receives its share of the
// total mass): V_c = sum over particles of colour c of m_i / rho_i, with the
// summation density rho_i of the last step and unit mass, and the particle
// count per colour. FP64 reduction in a fixed order, so repeated calls give
// identical bits:
//   k_color_partials  each block walks a contiguous chunk of particles 32 at a
//                     time; the lanes of a warp that share a colour are summed
//                     by the lowest of them in ascending lane order into the
//                     warp's own per-colour accumulator; the block adds its
//                     warps in warp order and writes one partial per colour;
//   k_color_final     one thread per colour adds the block partials in block
//                     order.
#include "sph_internal.h"

namespace sph {

namespace {

constexpr int kColorThreads = 256;
constexpr int kColorWarps = kColorThreads / 32;

template <class T>
__global__ void __launch_bounds__(kColorThreads) k_color_partials(int n, int chunk, const StepCtl* __restrict__ ctl,
                                                                  const uint32_t* __restrict__ m0,
                                                                  const uint32_t* __restrict__ m1,
                                                                  const T* __restrict__ rho,
                                                                  double* __restrict__ vpart,
                                                                  unsigned long long* __restrict__ cpart) {
  __shared__ double wvol[kColorWarps][256];
  __shared__ unsigned wcnt[kColorWarps][256];
  __shared__ double lanev[kColorWarps][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int c = lane; c < 256; c += 32) {
    wvol[w][c] = 0.0;
    wcnt[w][c] = 0u;
  }
  __syncwarp();
  const uint32_t* __restrict__ meta = ctl->buf ? m1 : m0;
  const int b0 = blockIdx.x * chunk;
  const int b1 = min(n, b0 + chunk);
  // the warp's share of the block's chunk, contiguous
  const int per = (chunk + kColorWarps - 1) / kColorWarps;
  const int w0 = b0 + w * per, w1 = min(b1, w0 + per);
  for (int base = w0; base < w1; base += 32) {
    const int i = base + lane;
    const bool on = i < w1;
    const uint32_t c = on ? (meta[i] & 0xFFu) : 256u;
    const double v = on ? 1.0 / (double)rho[i] : 0.0;
    lanev[w][lane] = v;
    __syncwarp();
    const unsigned peers = __match_any_sync(0xffffffffu, c);
    if (on && lane == __ffs(peers) - 1) {
      double s = 0.0;
      for (unsigned m = peers; m; m &= m - 1) s += lanev[w][__ffs(m) - 1];
      wvol[w][c] += s;
      wcnt[w][c] += (unsigned)__popc(peers);
    }
    __syncwarp();
  }
  __syncthreads();
  const int c = threadIdx.x;  // one thread per colour
  double s = 0.0;
  unsigned long long k = 0;
  for (int q = 0; q < kColorWarps; ++q) {
    s += wvol[q][c];
    k += wcnt[q][c];
  }
  vpart[(size_t)blockIdx.x * 256 + c] = s;
  cpart[(size_t)blockIdx.x * 256 + c] = k;
}

__global__ void __launch_bounds__(256) k_color_final(int nblocks, const double* __restrict__ vpart,
                                                     const unsigned long long* __restrict__ cpart,
                                                     double* __restrict__ vol, long long* __restrict__ cnt) {
  const int c = threadIdx.x;
  double s = 0.0;
  unsigned long long k = 0;
  for (int b = 0; b < nblocks; ++b) {
    s += vpart[(size_t)b * 256 + c];
    k += cpart[(size_t)b * 256 + c];
  }
  vol[c] = s;
  cnt[c] = (long long)k;
}

}  // namespace

int color_volume_blocks(int n) {
  // chunks of at least 8192 particles, at most 1024 blocks
  int nb = (n + 8191) / 8192;
  return nb < 1 ? 1 : (nb > 1024 ? 1024 : nb);
}

template <class T>
cudaError_t launch_color_volumes(const DevState& S, double* vpart, unsigned long long* cpart, double* vol,
                                 long long* cnt, cudaStream_t st) {
  const int nb = color_volume_blocks(S.n);
  const int chunk = (S.n + nb - 1) / nb;
  k_color_partials<T><<<nb, kColorThreads, 0, st>>>(S.n, chunk, S.ctl, S.meta[0], S.meta[1], (const T*)S.rho,
                                                     vpart, cpart);
  k_color_final<<<1, 256, 0, st>>>(nb, vpart, cpart, vol, cnt);
  return cudaGetLastError();
}

template cudaError_t launch_color_volumes<float>(const DevState&, double*, unsigned long long*, double*, long long*,
                                                 cudaStream_t);
template cudaError_t launch_color_volumes<double>(const DevState&, double*, unsigned long long*, double*, long long*,
                                                  cudaStream_t);

}  // namespace sph
