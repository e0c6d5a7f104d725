// Phase-field carrier from the VoF fraction (Sec. 2.5): signed distance by
// Hamilton-Jacobi redistancing, then the tanh profile and its regularised
// delta (Sec. 2.6).
//
// chi0 = 2h(C - 1/2) (positive inside fluid 1).  Each Jacobi step:
//   away from the interface  chi <- chi - dtau s (|grad chi|_G - 1)
//     with s = sign(chi0) and |grad chi|_G the first-order Godunov upwind
//     gradient;
//   in cells whose chi0 changes sign against a face neighbour (the
//   Russo-Smereka sub-cell fix)  chi <- chi - (dtau/h)(s |chi| - d)
//     with d = h chi0 / |Delta chi0| the distance estimated from chi0 alone.
#include <cmath>

#include "sfx_internal.h"

namespace sfx {
namespace {

__global__ void k_chi0(size_t n, double h, const double* __restrict__ C, double* __restrict__ chi0,
                       double* __restrict__ chi) {
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x) {
    double v = 2.0 * h * (C[c] - 0.5);
    chi0[c] = v;
    chi[c] = v;
  }
}

__global__ void k_redistance_step(Level L, double dtau, const double* __restrict__ chi0,
                                  const double* __restrict__ cin, double* __restrict__ cout) {
  const size_t n = L.ncell();
  const int nd = L.ndim();
  const double h = L.h;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x) {
    int idx[3] = {(int)(c % L.nx), (int)((c / L.nx) % L.ny), (int)(c / ((size_t)L.nx * L.ny))};
    const double s0 = chi0[c];
    const double sg = s0 > 0.0 ? 1.0 : (s0 < 0.0 ? -1.0 : 0.0);
    const double x0 = cin[c];
    // neighbour offsets along each direction (0 outside: mirrored wall)
    size_t stride[3] = {1, (size_t)L.nx, (size_t)L.nx * L.ny};
    bool cut = false;
    double gsum = 0.0, dsum = 0.0;
    for (int d = 0; d < nd; ++d) {
      bool hasm = idx[d] > 0, hasp = idx[d] + 1 < L.extent(d);
      size_t cm = hasm ? c - stride[d] : c, cp = hasp ? c + stride[d] : c;
      double z0m = chi0[cm], z0p = chi0[cp];
      if ((hasm && s0 * z0m < 0.0) || (hasp && s0 * z0p < 0.0)) cut = true;
      // sub-cell estimate of |grad chi0| h along d
      double q = fabs(z0p - z0m) * 0.5;
      q = fmax(q, fabs(z0p - s0));
      q = fmax(q, fabs(s0 - z0m));
      dsum += q * q;
      // Godunov upwind gradient of the current iterate
      double bwd = (x0 - cin[cm]) / h, fwd = (cin[cp] - x0) / h;
      double t;
      if (sg > 0.0) {
        double ap = fmax(bwd, 0.0), bm = fmin(fwd, 0.0);
        t = fmax(ap * ap, bm * bm);
      } else {
        double am = fmin(bwd, 0.0), bp = fmax(fwd, 0.0);
        t = fmax(am * am, bp * bp);
      }
      gsum += t;
    }
    double v;
    if (cut) {
      double dchi = fmax(sqrt(dsum), 1e-300);
      v = x0 - (dtau / h) * (sg * fabs(x0) - h * s0 / dchi);
    } else {
      v = x0 - dtau * sg * (sqrt(gsum) - 1.0);
    }
    cout[c] = v;
  }
}

__global__ void k_phi_delta64(size_t n, double eps, const double* __restrict__ chi,
                              double* __restrict__ phi, double* __restrict__ delta) {
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x) {
    double p = 0.5 * (1.0 - tanh(chi[c] / (2.0 * eps)));
    phi[c] = p;
    if (delta) delta[c] = p * (1.0 - p) / eps;
  }
}

}  // namespace

sfx_status phase_field_build(sfx_ctx* c, const double* C, double* chi, void* phi, void* delta,
                             int iters, double dtau, double eps, cudaStream_t s) {
  const Level& L = c->lev[0].lv;
  const size_t n = L.ncell();
  const int nb = blocks_for(n, 256);
  SFX_KERNEL(c, K_PHASE, k_chi0, nb, 256, s, n, L.h, C, c->chi0, chi);
  SFX_LAUNCH_CHECK();
  double* a = chi;
  double* b = c->chi_tmp;
  for (int it = 0; it < iters; ++it) {
    SFX_KERNEL(c, K_PHASE, k_redistance_step, nb, 256, s, L, dtau, c->chi0, a, b);
    double* t = a;
    a = b;
    b = t;
  }
  SFX_LAUNCH_CHECK();
  if (a != chi)
    SFX_CUDA(cudaMemcpyAsync(chi, a, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  SFX_KERNEL(c, K_PHASE, k_phi_delta64, nb, 256, s, n, eps, chi, (double*)phi, (double*)delta);
  SFX_LAUNCH_CHECK();
  return SFX_OK;
}

}  // namespace sfx
