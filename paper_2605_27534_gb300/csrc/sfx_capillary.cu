// Capillary force F_cap = sigma kappa delta_s n (Sec. 2.4) with the mean
// curvature kappa = -div n (Sec. 2.2) and delta_s = |grad C|.
//
// n = grad phi/|grad phi| at cell centres (centred differences, zero where
// phi is flat); div n in flux form over the cell's faces, each face taking
// the mean of its two cells' normal components:
//   kappa = -(1/h) sum_d (w+ nbar+ - w- nbar-),
// w = 1 except on the radial faces of the axisymmetric grid, where
// w+- = A+-/(V/h) = 2(i+1)/(2i+1), 2i/(2i+1) (the hoop term).  Wall faces
// carry no normal component; the axis face has zero area.  grad C is
// centred with zero-gradient ghosts.
//
// One pass: a block owns a 32 x 8 column of cells and walks its planes in
// z, keeping the unit normals of planes k-1, k, k+1 (with a one-cell halo
// in x and y) in a ring of shared-memory buffers, so that every normal is
// evaluated once per block instead of once per face that uses it.
#include <algorithm>

#include "sfx_f32_dev.cuh"
#include "sfx_internal.h"

namespace sfx {
namespace {

constexpr int kCapX = 32, kCapY = 8, kCapZChunk = 32;
constexpr int kCapHX = kCapX + 2, kCapHY = kCapY + 2;

// all components of n at (i,j,k) in FP64 (the arithmetic of normal_comp)
__device__ __forceinline__ void normal3_f64(const Level& L, const double* __restrict__ phi, int i,
                                            int j, int k, double eps, double* n) {
  const double inv2h = 0.5 / L.h;
  const int ip = min(i + 1, L.nx - 1), im = max(i - 1, 0);
  const int jp = min(j + 1, L.ny - 1), jm = max(j - 1, 0);
  double g0 = (phi[cidx(L, ip, j, k)] - phi[cidx(L, im, j, k)]) * inv2h;
  double g1 = (phi[cidx(L, i, jp, k)] - phi[cidx(L, i, jm, k)]) * inv2h;
  double g2 = 0.0;
  if (L.geom == SFX_CART3D) {
    const int kp = min(k + 1, L.nz - 1), km = max(k - 1, 0);
    g2 = (phi[cidx(L, i, j, kp)] - phi[cidx(L, i, j, km)]) * inv2h;
  }
  const double m = sqrt(g0 * g0 + g1 * g1 + g2 * g2);
  const double pc = phi[cidx(L, i, j, k)];
  const double w = normal_fade(m, pc * (1.0 - pc) / eps);
  if (!(w > 0.0)) {
    n[0] = n[1] = n[2] = 0.0;
    return;
  }
  n[0] = w * (g0 / m);
  n[1] = w * (g1 / m);
  n[2] = w * (g2 / m);
}

template <typename T>
struct CapNormal;
template <>
struct CapNormal<double> {
  static __device__ __forceinline__ void eval(const Level& L, const double* phi, int i, int j,
                                              int k, double eps, double* n) {
    normal3_f64(L, phi, i, j, k, eps, n);
  }
};
template <>
struct CapNormal<float> {
  static __device__ __forceinline__ void eval(const Level& L, const double* phi, int i, int j,
                                              int k, double eps, float* n) {
    normal3_f32(L, phi, i, j, k, (float)(1.0 / eps), n);
  }
};

// T: arithmetic type (double in SFX_F64 contexts, float in SFX_F32);
// P: storage type of C, sigma, kappa and the force.
template <typename T, typename P>
__global__ void __launch_bounds__(kCapX* kCapY)
    k_capillary(Level L, const double* __restrict__ phi, const P* __restrict__ C,
                const P* __restrict__ sigma, double eps, P* __restrict__ kappa,
                P* __restrict__ force) {
  // ring of three planes of normals, each with a one-cell halo in x and y
  __shared__ T sn[3][3][kCapHY][kCapHX];
  const int tx = threadIdx.x % kCapX, ty = threadIdx.x / kCapX;
  const int i0 = blockIdx.x * kCapX, j0 = blockIdx.y * kCapY;
  const int i = i0 + tx, j = j0 + ty;
  const bool is3d = L.geom == SFX_CART3D;
  const int k0 = is3d ? blockIdx.z * kCapZChunk : 0;
  const int k1 = is3d ? min(k0 + kCapZChunk, L.nz) : 1;
  const size_t N = L.ncell();
  const T inv_h = (T)(1.0 / L.h);

  // normals of plane k (tile and halo) into ring slot (k + 3) % 3
  auto fill = [&](int k) {
    T(*s)[kCapHY][kCapHX] = sn[(k + 3) % 3];
    for (int q = threadIdx.x; q < kCapHX * kCapHY; q += kCapX * kCapY) {
      const int hx = q % kCapHX, hy = q / kCapHX;
      const int a = i0 + hx - 1, b = j0 + hy - 1;
      T n[3] = {(T)0, (T)0, (T)0};
      if (a >= 0 && a < L.nx && b >= 0 && b < L.ny) CapNormal<T>::eval(L, phi, a, b, k, eps, n);
      s[0][hy][hx] = n[0];
      s[1][hy][hx] = n[1];
      s[2][hy][hx] = n[2];
    }
  };

  if (is3d && k0 > 0) fill(k0 - 1);
  fill(k0);
  for (int k = k0; k < k1; ++k) {
    if (is3d && k + 1 < L.nz) fill(k + 1);
    __syncthreads();
    if (i < L.nx && j < L.ny) {
      T(*s)[kCapHY][kCapHX] = sn[(k + 3) % 3];
      const int hx = tx + 1, hy = ty + 1;
      T wm = (T)1, wp = (T)1;
      if (L.geom == SFX_AXISYM) {
        const T den = (T)(2 * i + 1);
        wm = (T)(2 * i) / den;
        wp = (T)(2 * i + 2) / den;
      }
      const T nx0 = s[0][hy][hx], ny0 = s[1][hy][hx];
      T div = (T)0;
      if (i > 0) div -= wm * ((T)0.5 * (nx0 + s[0][hy][hx - 1]));
      if (i < L.nx - 1) div += wp * ((T)0.5 * (nx0 + s[0][hy][hx + 1]));
      if (j > 0) div -= (T)0.5 * (ny0 + s[1][hy - 1][hx]);
      if (j < L.ny - 1) div += (T)0.5 * (ny0 + s[1][hy + 1][hx]);
      T nz0 = (T)0;
      if (is3d) {
        nz0 = s[2][hy][hx];
        if (k > 0) div -= (T)0.5 * (nz0 + sn[(k + 2) % 3][2][hy][hx]);
        if (k < L.nz - 1) div += (T)0.5 * (nz0 + sn[(k + 1) % 3][2][hy][hx]);
      }
      const T kap = -div * inv_h;
      // delta_s = |grad C|, centred, zero-gradient ghosts
      const T inv2h = (T)0.5 * inv_h;
      const int ip = min(i + 1, L.nx - 1), im = max(i - 1, 0);
      const int jp = min(j + 1, L.ny - 1), jm = max(j - 1, 0);
      const T gx = ((T)C[cidx(L, ip, j, k)] - (T)C[cidx(L, im, j, k)]) * inv2h;
      const T gy = ((T)C[cidx(L, i, jp, k)] - (T)C[cidx(L, i, jm, k)]) * inv2h;
      T q = gx * gx + gy * gy;
      if (is3d) {
        const int kp = min(k + 1, L.nz - 1), km = max(k - 1, 0);
        const T gz = ((T)C[cidx(L, i, j, kp)] - (T)C[cidx(L, i, j, km)]) * inv2h;
        q += gz * gz;
      }
      const size_t c = cidx(L, i, j, k);
      const T a = (T)sigma[c] * kap * sqrt(q);
      force[c] = (P)(a * nx0);
      force[N + c] = (P)(a * ny0);
      if (is3d) force[2 * N + c] = (P)(a * nz0);
      if (kappa) kappa[c] = (P)kap;
    }
    __syncthreads();   // slot (k + 2) % 3 is refilled by the next plane
  }
}

template <typename T, typename P>
sfx_status capillary_impl(sfx_ctx* c, const double* phi, const P* C, const P* sigma, double eps,
                          P* kappa, P* force, cudaStream_t s) {
  const Level& L = c->lev[0].lv;
  const unsigned gz = L.geom == SFX_CART3D ? (unsigned)((L.nz + kCapZChunk - 1) / kCapZChunk) : 1u;
  const dim3 grid((unsigned)((L.nx + kCapX - 1) / kCapX), (unsigned)((L.ny + kCapY - 1) / kCapY),
                  gz);
  SFX_KERNEL(c, K_FORCES, (k_capillary<T, P>), grid, kCapX * kCapY, s, L, phi, C, sigma, eps,
             kappa, force);
  SFX_LAUNCH_CHECK();
  return SFX_OK;
}

}  // namespace

sfx_status capillary(sfx_ctx* c, const sfx_params* p, const double* phi, const void* C,
                     const void* sigma, void* kappa, void* force, cudaStream_t s) {
  if (((size_t)c->lev[0].lv.ny + kCapY - 1) / kCapY > 65535u) return SFX_ERR_ARG;
  if (c->prec == SFX_F32)
    return capillary_impl<float, float>(c, phi, (const float*)C, (const float*)sigma, p->eps,
                                        (float*)kappa, (float*)force, s);
  return capillary_impl<double, double>(c, phi, (const double*)C, (const double*)sigma, p->eps,
                                        (double*)kappa, (double*)force, s);
}

}  // namespace sfx
