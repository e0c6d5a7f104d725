// Shared device helpers of libsfx: grid levels, metric (cell volumes and
// face areas of Sec. 3.2, App. A and App. B), indexing and reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sfx.h"

namespace sfx {

constexpr double kPi = 3.14159265358979323846;

// One uniform grid level, passed to kernels by value.
struct Level {
  int geom;
  int nx, ny, nz;
  double h;
  __host__ __device__ int ndim() const { return geom == SFX_CART3D ? 3 : 2; }
  __host__ __device__ size_t ncell() const { return (size_t)nx * ny * nz; }
  __host__ __device__ int extent(int d) const { return d == 0 ? nx : (d == 1 ? ny : nz); }
  __host__ __device__ size_t nface(int d) const {
    return (size_t)(nx + (d == 0)) * (ny + (d == 1)) * (nz + (d == 2));
  }
};

__host__ __device__ inline size_t cidx(const Level& L, int i, int j, int k) {
  return ((size_t)k * L.ny + j) * L.nx + i;
}
// face (i,j,k) in direction d: the face on the minus side of cell (i,j,k)
__host__ __device__ inline size_t fidx(const Level& L, int d, int i, int j, int k) {
  int fx = L.nx + (d == 0), fy = L.ny + (d == 1);
  return ((size_t)k * fy + j) * fx + i;
}

// Cell volume: h^2 (planar, unit depth), h^3 (3D), pi (2i+1) h^3 (ring).
__host__ __device__ inline double cell_volume(const Level& L, int i) {
  double h = L.h;
  if (L.geom == SFX_PLANAR2D) return h * h;
  if (L.geom == SFX_CART3D) return h * h * h;
  return kPi * (double)(2 * i + 1) * h * h * h;
}
// Area of the minus-side face of cell column i in direction d: planar h,
// 3D h^2, axisymmetric radial 2 pi (i h) h, axial pi (2i+1) h^2.
__host__ __device__ inline double face_area(const Level& L, int d, int i) {
  double h = L.h;
  if (L.geom == SFX_PLANAR2D) return h;
  if (L.geom == SFX_CART3D) return h * h;
  if (d == 0) return 2.0 * kPi * (double)i * h * h;
  return kPi * (double)(2 * i + 1) * h * h;
}

// ---------------------------------------------------------------- reductions
// Max of non-negative doubles via their bit patterns (order-independent,
// hence deterministic).  NaN sets the flag instead.
__device__ inline void atomic_max_nonneg(unsigned long long* slot, double v) {
  atomicMax(slot, (unsigned long long)__double_as_longlong(v));
}

template <typename T>
__device__ inline T warp_max(T v) {
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Error-free sum (Knuth two-sum).
__device__ inline void two_sum(double a, double b, double& s, double& e) {
  s = a + b;
  double bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Compensated pair reduction across a warp: (s, c) with value s + c.
__device__ inline void warp_sum_comp(double& s, double& c) {
  for (int o = 16; o > 0; o >>= 1) {
    double so = __shfl_down_sync(0xffffffffu, s, o);
    double co = __shfl_down_sync(0xffffffffu, c, o);
    double t, e;
    two_sum(s, so, t, e);
    s = t;
    c = c + co + e;
  }
}

// n is undefined where phi is flat: beyond the redistancing band phi is
// flat up to variations far below its own profile slope phi (1 - phi)/eps,
// whose direction is set by the last bits of phi.  With q = |grad phi| /
// (phi (1 - phi)/eps), n fades out continuously: it is scaled by
// w = clamp(q/kNormalKappa - 1, 0, 1) (0 at or below kNormalKappa, the
// unit vector at or above twice it), and n = 0 where |grad phi| < 1e-30.
// A hard cut-off would make the step jump when a round-off change of phi
// moves q of a band-edge cell across it.
constexpr double kNormalKappa = 1e-3;

__device__ __forceinline__ double normal_fade(double m, double slope) {
  return m < 1e-30 ? 0.0 : fmin(fmax(m / (kNormalKappa * slope) - 1.0, 0.0), 1.0);
}

// Unit normal component n_d = (grad phi)_d / |grad phi| at cell (i,j,k):
// centred differences, zero-gradient walls, faded out where phi is flat
// (above).
template <typename P>
__device__ __forceinline__ double normal_comp(const Level& L, const P* __restrict__ phi, int i,
                                              int j, int k, int d, double eps) {
  double g[3] = {0.0, 0.0, 0.0};
  const double inv2h = 0.5 / L.h;
  int ip = min(i + 1, L.nx - 1), im = max(i - 1, 0);
  int jp = min(j + 1, L.ny - 1), jm = max(j - 1, 0);
  g[0] = ((double)phi[cidx(L, ip, j, k)] - (double)phi[cidx(L, im, j, k)]) * inv2h;
  g[1] = ((double)phi[cidx(L, i, jp, k)] - (double)phi[cidx(L, i, jm, k)]) * inv2h;
  if (L.geom == SFX_CART3D) {
    int kp = min(k + 1, L.nz - 1), km = max(k - 1, 0);
    g[2] = ((double)phi[cidx(L, i, j, kp)] - (double)phi[cidx(L, i, j, km)]) * inv2h;
  }
  double m = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
  const double pc = (double)phi[cidx(L, i, j, k)];
  const double slope = pc * (1.0 - pc) / eps;
  const double w = normal_fade(m, slope);
  return w > 0.0 ? w * (g[d] / m) : 0.0;
}

}  // namespace sfx
