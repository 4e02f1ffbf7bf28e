// Set-up kernels of sph_create: bounds and total mass of the target field
// (Sec. 3.2, Eq. total_mass_2) and the initial particle state (density-
// proportional sampling in the region, colours from the nearest of n_colors
// generators drawn uniformly in the region: the Voronoi initialisation of
// Sec. 4.2). Random numbers come from Philox4x32-10 keyed by the seed.
#include <cfloat>

#include "sph_internal.h"

namespace sph {

namespace {

constexpr int kBoundsBlocks = 1024;
constexpr int kMaxAttempts = 1 << 20;

template <int D>
__device__ __forceinline__ void weight_and_seff(const Geom<double>& g, const double* x, double& w, double& seff) {
  const double s = spacing_of(g, x);
  const double f = poly_factor(g, x);
  w = (D == 2 ? 1.0 / (s * s) : 1.0 / (s * s * s)) * f;  // s^-d (1 + P)
  seff = s * (D == 2 ? rsqrt(f) : rcbrt(f));            // h / hfac
}

template <int D>
__global__ void __launch_bounds__(256) k_field_bounds(Geom<double> g, int res, double* __restrict__ part) {
  __shared__ double sm[4][8];
  const long long total = D == 2 ? (long long)res * res : (long long)res * res * res;
  double sw = 0.0, smin = DBL_MAX, smax = 0.0, wmax = 0.0;
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < total;
       c += (long long)gridDim.x * blockDim.x) {
    double x[3] = {0, 0, 0};
    long long r = c;
    for (int k = 0; k < D; ++k) {
      x[k] = g.lo[k] + ((double)(r % res) + 0.5) * (g.ext[k] / res);
      r /= res;
    }
    if (!in_region(g, x)) continue;
    double w, seff;
    weight_and_seff<D>(g, x, w, seff);
    sw += w;
    smin = fmin(smin, seff);
    smax = fmax(smax, seff);
    wmax = fmax(wmax, w);
  }
  for (int o = 16; o > 0; o >>= 1) {
    sw += __shfl_xor_sync(0xffffffffu, sw, o);
    smin = fmin(smin, __shfl_xor_sync(0xffffffffu, smin, o));
    smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
    wmax = fmax(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    sm[0][w] = sw;
    sm[1][w] = smin;
    sm[2][w] = smax;
    sm[3][w] = wmax;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = DBL_MAX, c = 0.0, d = 0.0;
    for (int q = 0; q < 8; ++q) {
      a += sm[0][q];
      b = fmin(b, sm[1][q]);
      c = fmax(c, sm[2][q]);
      d = fmax(d, sm[3][q]);
    }
    part[4 * blockIdx.x + 0] = a;
    part[4 * blockIdx.x + 1] = b;
    part[4 * blockIdx.x + 2] = c;
    part[4 * blockIdx.x + 3] = d;
  }
}

template <int D>
__device__ __forceinline__ void box_point(const Geom<double>& g, uint4 r, double* x) {
  const uint32_t u[3] = {r.x, r.y, r.z};
  for (int k = 0; k < D; ++k) x[k] = g.lo[k] + g.ext[k] * u01(u[k]);
}

template <int D>
__global__ void __launch_bounds__(256) k_generators(Geom<double> g, int ng, uint2 key, double* __restrict__ gens,
                                                    int* __restrict__ err) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= ng) return;
  double x[3] = {0, 0, 0};
  for (int a = 0; a < kMaxAttempts; ++a) {
    const uint4 r = philox4x32_10(make_uint4((uint32_t)q, (uint32_t)a, 0x9E11u, 1u), key);
    box_point<D>(g, r, x);
    if (in_region(g, x)) {
      for (int k = 0; k < 3; ++k) gens[3 * q + k] = x[k];
      return;
    }
  }
  atomicOr(err, kErrTimeout);
  for (int k = 0; k < 3; ++k) gens[3 * q + k] = k < D ? g.lo[k] + 0.5 * g.ext[k] : 0.0;
}

template <int D>
__global__ void __launch_bounds__(256) k_sample(Geom<double> g, int n, int ng, uint2 key, double wmax,
                                                const double* __restrict__ gens, double* __restrict__ xyz,
                                                uint8_t* __restrict__ col, int* __restrict__ err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double x[3] = {0, 0, 0};
  bool ok = false;
  for (int a = 0; a < kMaxAttempts && !ok; ++a) {
    const uint4 r = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)a, 0u, 0u), key);
    box_point<D>(g, r, x);
    if (!in_region(g, x)) continue;
    double w, seff;
    weight_and_seff<D>(g, x, w, seff);
    ok = u01(r.w) * wmax < w;
  }
  if (!ok) atomicOr(err, kErrTimeout);
  for (int k = 0; k < D; ++k) xyz[(size_t)i * D + k] = x[k];
  // nearest generator (ties: lowest index)
  int best = 0;
  double bd = DBL_MAX;
  for (int q = 0; q < ng; ++q) {
    double d2 = 0.0;
    for (int k = 0; k < D; ++k) {
      const double d = x[k] - gens[3 * q + k];
      d2 += d * d;
    }
    if (d2 < bd) {
      bd = d2;
      best = q;
    }
  }
  col[i] = (uint8_t)best;
}

}  // namespace

template <int D>
cudaError_t field_bounds(const Geom<double>& g, int res, FieldBounds* out, double* scratch, cudaStream_t st) {
  k_field_bounds<D><<<kBoundsBlocks, 256, 0, st>>>(g, res, scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  static thread_local double host[4 * kBoundsBlocks];
  e = cudaMemcpyAsync(host, scratch, sizeof(double) * 4 * kBoundsBlocks, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  FieldBounds b{0.0, DBL_MAX, 0.0, 0.0};
  for (int q = 0; q < kBoundsBlocks; ++q) {
    b.sum_w += host[4 * q];
    b.min_seff = fmin(b.min_seff, host[4 * q + 1]);
    b.max_seff = fmax(b.max_seff, host[4 * q + 2]);
    b.max_w = fmax(b.max_w, host[4 * q + 3]);
  }
  *out = b;
  return cudaSuccess;
}

int field_bounds_scratch_doubles() { return 4 * kBoundsBlocks; }

template <int D>
cudaError_t sample_positions(const Geom<double>& g, int n, int n_colors, uint64_t seed, double wmax, double* xyz,
                             uint8_t* col, double* gens, int* err, cudaStream_t st) {
  const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
  k_generators<D><<<(n_colors + 255) / 256, 256, 0, st>>>(g, n_colors, key, gens, err);
  if (n > 0) k_sample<D><<<(n + 255) / 256, 256, 0, st>>>(g, n, n_colors, key, wmax, gens, xyz, col, err);
  return cudaGetLastError();
}

template cudaError_t field_bounds<2>(const Geom<double>&, int, FieldBounds*, double*, cudaStream_t);
template cudaError_t field_bounds<3>(const Geom<double>&, int, FieldBounds*, double*, cudaStream_t);
template cudaError_t sample_positions<2>(const Geom<double>&, int, int, uint64_t, double, double*, uint8_t*,
                                         double*, int*, cudaStream_t);
template cudaError_t sample_positions<3>(const Geom<double>&, int, int, uint64_t, double, double*, uint8_t*,
                                         double*, int*, cudaStream_t);

}  // namespace sph
