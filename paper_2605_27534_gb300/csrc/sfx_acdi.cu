// ACDI transport of the phase field (Sec. 2.5):
//   d phi/dt + div(u phi) = div(zeta {eps grad phi
//                              - 1/4 (1 - tanh^2(psi/(2 eps))) grad psi/|grad psi|}),
//   psi = eps ln r,  r = (phi + veps)/(1 - phi + veps),  veps = 1e-6,
// FP64 in both context precisions (phi is double everywhere).  The
// advective part is the BCG step of the transported fields (inflow faces
// carry phi = 1); the regularisation is explicit, in flux form, with the
// central face fluxes
//   a_f = zeta [eps (phi*_R - phi*_L)/h - 1/4 w_f nbar_f],
// nbar_f the mean of the two cells' unit normals of psi along the face and
// w_f = 1 - tanh^2((psi_L + psi_R)/(4 eps)).  With s = sqrt(r_L r_R),
// tanh((psi_L + psi_R)/(4 eps)) = (s - 1)/(s + 1), so w_f = 4 s/(1 + s)^2:
// the face needs no transcendental beyond the square root.
//
// Three passes over the grid: r and psi per cell, the unit normals of psi
// per cell, then the face fluxes and the update (clipped to [0, 1] on
// request: the scheme overshoots by O(veps) where phi saturates, and the
// surfactant step divides by phi + eta).
#include <algorithm>

#include "sfx_internal.h"

namespace sfx {
namespace {

constexpr double kAcdiVeps = 1e-6;
// n is undefined where psi is flat: where phi saturates, the direction of
// grad psi is set by the last bits of phi while 1 - tanh^2 stays ~4 veps.
// n = 0 where |grad psi| is below kAcdiKappa times its equilibrium value 1
// (psi is a signed distance at equilibrium) or below 1e-30; |grad psi|
// falls below 0.1 only where veps dominates psi (phi or 1 - phi below
// ~0.1 veps).
constexpr double kAcdiKappa = 0.1;

__global__ void k_acdi_psi(size_t n, const double* __restrict__ ps, double eps,
                           double* __restrict__ r, double* __restrict__ psi) {
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x) {
    // phi* may overshoot [0, 1] by O(veps) where it saturates; past
    // 1 + veps psi would have no value, so it is formed from phi* in [0, 1]
    const double p = fmin(fmax(ps[c], 0.0), 1.0);
    const double rc = (p + kAcdiVeps) / (1.0 - p + kAcdiVeps);
    r[c] = rc;
    psi[c] = eps * log(rc);
  }
}

// n = grad psi/|grad psi| (centred differences, zero-gradient ghosts), 0
// where psi is flat (above)
__global__ void k_acdi_normal(Level L, const double* __restrict__ psi, double* __restrict__ nv) {
  const size_t n = L.ncell();
  const int nd = L.ndim();
  const double inv2h = 0.5 / L.h;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x) {
    const int ix[3] = {(int)(c % L.nx), (int)((c / L.nx) % L.ny),
                       (int)(c / ((size_t)L.nx * L.ny))};
    double g[3] = {0.0, 0.0, 0.0}, m2 = 0.0;
    for (int d = 0; d < nd; ++d) {
      int pp[3] = {ix[0], ix[1], ix[2]}, pm[3] = {ix[0], ix[1], ix[2]};
      pp[d] = min(pp[d] + 1, L.extent(d) - 1);
      pm[d] = max(pm[d] - 1, 0);
      g[d] = (psi[cidx(L, pp[0], pp[1], pp[2])] - psi[cidx(L, pm[0], pm[1], pm[2])]) * inv2h;
      m2 += g[d] * g[d];
    }
    const double m = sqrt(m2);
    const bool flat = m < 1e-30 || m < kAcdiKappa;
    for (int d = 0; d < nd; ++d) nv[(size_t)d * n + c] = flat ? 0.0 : g[d] / m;
  }
}

// phi = phi* + dt/V sum_f (+-) A_f a_f; wall faces carry nothing and the
// axis face has zero area
__global__ void k_acdi_update(Level L, const double* __restrict__ ps,
                              const double* __restrict__ r, const double* __restrict__ nv,
                              double zeta, double eps, double dt, int clip,
                              double* __restrict__ phi) {
  const size_t n = L.ncell();
  const int nd = L.ndim();
  const double invh = 1.0 / L.h;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x) {
    const int ix[3] = {(int)(c % L.nx), (int)((c / L.nx) % L.ny),
                       (int)(c / ((size_t)L.nx * L.ny))};
    const double pc = ps[c], rc = r[c];
    double div = 0.0;
    for (int d = 0; d < nd; ++d) {
      const double* nd_ = nv + (size_t)d * n;
      const double ncd = nd_[c];
      for (int s = -1; s <= 1; s += 2) {
        int q[3] = {ix[0], ix[1], ix[2]};
        q[d] += s;
        if (q[d] < 0 || q[d] >= L.extent(d)) continue;
        const size_t o = cidx(L, q[0], q[1], q[2]);
        // face area over V/h: 1, or the ring ratios on radial faces
        double w = 1.0;
        if (L.geom == SFX_AXISYM && d == 0) {
          const int iface = s < 0 ? ix[0] : ix[0] + 1;
          w = 2.0 * (double)iface / (double)(2 * ix[0] + 1);
        }
        const double sq = sqrt(rc * r[o]);
        const double wt = 4.0 * sq / ((1.0 + sq) * (1.0 + sq));
        const double nbar = 0.5 * (ncd + nd_[o]);
        // flux along +d through the face; phi_R - phi_L = s (phi_o - phi_c)
        const double af = zeta * (eps * (double)s * (ps[o] - pc) * invh - 0.25 * wt * nbar);
        div += (double)s * w * af;
      }
    }
    const double v = pc + dt * div * invh;
    phi[c] = clip ? fmin(fmax(v, 0.0), 1.0) : v;
  }
}

}  // namespace

sfx_status acdi_step(sfx_ctx* c, const void* ux, const void* uy, const void* uz, double dt,
                     double zeta, double eps, int clip, double* phi, cudaStream_t s) {
  const Level& L = c->lev[0].lv;
  const size_t n = L.ncell();
  if (!c->acdi) {
    SFX_CUDA(cudaMalloc((void**)&c->acdi, (size_t)(3 + L.ndim()) * n * sizeof(double)));
    c->allocations.push_back(c->acdi);
  }
  double* ps = c->acdi;
  double* r = ps + n;
  double* psi = r + n;
  double* nv = psi + n;
  if (ux) {
    sfx_status st = advect(c, ux, uy, uz, dt, phi, 1.0, ps, s);
    if (st != SFX_OK) return st;
  } else {
    SFX_CUDA(cudaMemcpyAsync(ps, phi, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  const int nb = blocks_for(n, 256);
  SFX_KERNEL(c, K_PHASE, k_acdi_psi, nb, 256, s, n, ps, eps, r, psi);
  SFX_KERNEL(c, K_PHASE, k_acdi_normal, nb, 256, s, L, psi, nv);
  SFX_KERNEL(c, K_PHASE, k_acdi_update, nb, 256, s, L, ps, r, nv, zeta, eps, dt, clip, phi);
  SFX_LAUNCH_CHECK();
  return SFX_OK;
}

}  // namespace sfx
