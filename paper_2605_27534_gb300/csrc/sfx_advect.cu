// Explicit advection step of Sec. 3.1: xi* = xi - dt div(u xi) with the
// unsplit Bell-Colella-Glaz predictor for the face values.
//
// Face value at a face with normal velocity u and Courant number c = u dt/h:
// take the upwind cell U, extrapolate along the normal over half a step,
//   xi_U + (sign(u) - c)/2 * slope_U       (monotonised-central slope),
// and subtract half a step of transverse advection
//   - dt/2 * vbar_U * (upwinded transverse difference)/h
// with vbar_U the cell-centred transverse velocity.  Inflow walls carry
// bc_in; walls reuse the wall cell (zero gradient) for slopes.
#include <cmath>
#include <cstring>

#include "sfx_internal.h"

namespace sfx {
namespace {

__device__ __forceinline__ double mc_limited(double xm, double x0, double xp) {
  double dl = x0 - xm, dr = xp - x0;
  if (dl * dr <= 0.0) return 0.0;
  double dc = 0.5 * (xp - xm);
  double m = fmin(fabs(dc), 2.0 * fmin(fabs(dl), fabs(dr)));
  return dc > 0.0 ? m : -m;
}

template <typename U>
struct Vel {
  const U* u[3];
};

// value of xi at cell idx shifted by s along d (the cell itself outside)
__device__ __forceinline__ double nb(const Level& L, const double* __restrict__ xi,
                                     const int* idx, size_t c, int d, int s) {
  int p = idx[d] + s;
  if (p < 0 || p >= L.extent(d)) return xi[c];
  size_t stride = d == 0 ? 1 : (d == 1 ? (size_t)L.nx : (size_t)L.nx * L.ny);
  return s > 0 ? xi[c + stride] : xi[c - stride];
}

// BCG face value on the face of direction d whose plus-side cell is f
// (f[d] in 0..extent; f[d] = 0 or extent is a wall).
template <typename U>
__device__ double face_value(const Level& L, const Vel<U>& v, double dt,
                             const double* __restrict__ xi, double bc_in, int d, const int* f,
                             double u) {
  int n = L.extent(d);
  int uc[3] = {f[0], f[1], f[2]};
  if (u > 0.0) {
    if (f[d] == 0) return bc_in;
    uc[d] -= 1;
  } else if (f[d] == n) {
    return bc_in;
  }
  size_t U_ = cidx(L, uc[0], uc[1], uc[2]);
  double x0 = xi[U_];
  double sgn = u > 0.0 ? 1.0 : -1.0;
  double slope = mc_limited(nb(L, xi, uc, U_, d, -1), x0, nb(L, xi, uc, U_, d, +1));
  double val = x0 + 0.5 * (sgn - u * dt / L.h) * slope;
  for (int t = 0; t < L.ndim(); ++t) {
    if (t == d) continue;
    int ap[3] = {uc[0], uc[1], uc[2]};
    ap[t] += 1;
    double vbar = 0.5 * ((double)v.u[t][fidx(L, t, uc[0], uc[1], uc[2])] +
                         (double)v.u[t][fidx(L, t, ap[0], ap[1], ap[2])]);
    double dif = vbar > 0.0 ? x0 - nb(L, xi, uc, U_, t, -1) : nb(L, xi, uc, U_, t, +1) - x0;
    val -= 0.5 * dt * vbar * dif / L.h;
  }
  return val;
}

template <typename U>
__global__ void k_advect(Level L, Vel<U> v, double dt, const double* __restrict__ xi,
                         double bc_in, double* __restrict__ out) {
  const size_t n = L.ncell();
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x) {
    int idx[3] = {(int)(c % L.nx), (int)((c / L.nx) % L.ny), (int)(c / ((size_t)L.nx * L.ny))};
    double div = 0.0;
    for (int d = 0; d < L.ndim(); ++d) {
      const U* ud = v.u[d];
      double um = (double)ud[fidx(L, d, idx[0], idx[1], idx[2])];
      if (um != 0.0)
        div -= face_area(L, d, idx[0]) * um * face_value(L, v, dt, xi, bc_in, d, idx, um);
      int p[3] = {idx[0], idx[1], idx[2]};
      p[d] += 1;
      double up = (double)ud[fidx(L, d, p[0], p[1], p[2])];
      if (up != 0.0)
        div += face_area(L, d, p[0]) * up * face_value(L, v, dt, xi, bc_in, d, p, up);
    }
    out[c] = xi[c] - dt * div / cell_volume(L, idx[0]);
  }
}

template <typename U>
__global__ void k_umax(size_t n, const U* __restrict__ u, unsigned long long* slot) {
  double m = 0.0;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n;
       q += (size_t)gridDim.x * blockDim.x)
    m = fmax(m, fabs((double)u[q]));
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0) atomic_max_nonneg(slot, m);
}

}  // namespace

sfx_status advect(sfx_ctx* c, const void* ux, const void* uy, const void* uz, double dt,
                  const double* xi, double bc_in, double* out, cudaStream_t s) {
  const Level& L = c->lev[0].lv;
  const int nb = blocks_for(L.ncell(), 256);
  if (c->prec == SFX_F64) {
    Vel<double> v{{(const double*)ux, (const double*)uy, (const double*)uz}};
    SFX_KERNEL(c, K_ADVECT, k_advect<double>, nb, 256, s, L, v, dt, xi, bc_in, out);
  } else {
    Vel<float> v{{(const float*)ux, (const float*)uy, (const float*)uz}};
    SFX_KERNEL(c, K_ADVECT, k_advect<float>, nb, 256, s, L, v, dt, xi, bc_in, out);
  }
  SFX_LAUNCH_CHECK();
  return SFX_OK;
}

sfx_status cfl_umax(sfx_ctx* c, const void* ux, const void* uy, const void* uz, double* umax,
                    cudaStream_t s) {
  const Level& L = c->lev[0].lv;
  SFX_CUDA(cudaMemsetAsync(c->d_norms, 0, 8 * sizeof(unsigned long long), s));
  const void* u[3] = {ux, uy, uz};
  for (int d = 0; d < L.ndim(); ++d) {
    size_t n = L.nface(d);
    if (c->prec == SFX_F64)
      SFX_KERNEL(c, K_OTHER, k_umax<double>, blocks_for(n, 256), 256, s, n, (const double*)u[d], c->d_norms);
    else
      SFX_KERNEL(c, K_OTHER, k_umax<float>, blocks_for(n, 256), 256, s, n, (const float*)u[d], c->d_norms);
  }
  SFX_LAUNCH_CHECK();
  SFX_CUDA(cudaMemcpyAsync(c->h_norms, c->d_norms, sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, s));
  SFX_CUDA(cudaStreamSynchronize(s));
  unsigned long long b = c->h_norms[0];
  memcpy(umax, &b, sizeof(double));
  return SFX_OK;
}

}  // namespace sfx
