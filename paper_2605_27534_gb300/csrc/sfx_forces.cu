// Conserved totals (compensated, deterministic), the surface-tension EOS of
// Sec. 2.3 and the Marangoni force of Sec. 2.4.
#include <cmath>
#include <cstring>

#include "sfx_internal.h"
#include "sfx_op64.cuh"
#include "sfx_plic.cuh"

namespace sfx {
namespace {

constexpr int kTotThreads = kTotalsThreads;

// Per-block compensated partial sums of V x for field `fi`.
__global__ void k_total_partials(Level L, const double* __restrict__ x, int fi,
                                 double* __restrict__ partials) {
  const size_t n = L.ncell();
  double s = 0.0, cc = 0.0;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x) {
    double v = cell_volume(L, (int)(c % L.nx)) * x[c];
    double t, e;
    two_sum(s, v, t, e);
    s = t;
    cc += e;
  }
  warp_sum_comp(s, cc);
  __shared__ double ss[kTotThreads / 32], sc[kTotThreads / 32];
  int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { ss[w] = s; sc[w] = cc; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = ss[0], b = sc[0];
    for (int q = 1; q < kTotThreads / 32; ++q) {
      double t, e;
      two_sum(a, ss[q], t, e);
      a = t;
      b += sc[q] + e;
    }
    size_t o = 2 * ((size_t)fi * gridDim.x + blockIdx.x);
    partials[o] = a;
    partials[o + 1] = b;
  }
}

// One block per field: fixed-order combination of the block partials.
__global__ void k_total_final(const double* __restrict__ partials, int nblk,
                              double* __restrict__ out) {
  const int fi = blockIdx.x;
  double s = 0.0, cc = 0.0;
  for (int q = threadIdx.x; q < nblk; q += blockDim.x) {
    size_t o = 2 * ((size_t)fi * nblk + q);
    double t, e;
    two_sum(s, partials[o], t, e);
    s = t;
    cc += partials[o + 1] + e;
  }
  warp_sum_comp(s, cc);
  __shared__ double ss[kTotThreads / 32], sc[kTotThreads / 32];
  int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { ss[w] = s; sc[w] = cc; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = ss[0], b = sc[0];
    for (int q = 1; q < kTotThreads / 32; ++q) {
      double t, e;
      two_sum(a, ss[q], t, e);
      a = t;
      b += sc[q] + e;
    }
    out[fi] = a + b;
  }
}

struct EosArgs {
  double ginf, eps, sigma0, E;
  int eos;
};

// Gamma = f/delta_phi where delta_phi >= 1e-3/eps, else 0; sigma in double.
template <typename P>
__global__ void k_eos(size_t n, EosArgs q, const double* __restrict__ f,
                      const P* __restrict__ phi, double* __restrict__ sigma) {
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x) {
    double p = (double)phi[c];
    double del = p * (1.0 - p) / q.eps;
    double G = del >= 1e-3 / q.eps ? f[c] / del : 0.0;
    double x = G / q.ginf;
    double s;
    if (q.eos == SFX_EOS_LANGMUIR) {
      x = fmin(x, 1.0 - 1e-12);          // stay below saturation
      s = q.sigma0 * (1.0 + q.E * log1p(-x));
    } else if (q.eos == SFX_EOS_LINEAR) {
      s = q.sigma0 * (1.0 - q.E * x);
    } else {
      s = q.sigma0 * (1.0 - tanh(q.E * x));
    }
    sigma[c] = s;
  }
}

// d sigma/d Gamma of the EOS above (0 where the Langmuir sigma is clamped)
__device__ __forceinline__ double eos_slope(const EosArgs& q, double G) {
  const double x = G / q.ginf;
  if (q.eos == SFX_EOS_LANGMUIR)
    return x < 1.0 - 1e-12 ? -q.sigma0 * q.E / (q.ginf * (1.0 - x)) : 0.0;
  if (q.eos == SFX_EOS_LINEAR) return -q.sigma0 * q.E / q.ginf;
  const double t = tanh(q.E * x);
  return -q.sigma0 * q.E / q.ginf * (1.0 - t * t);
}

template <typename P>
__global__ void k_force(Level L, const P* __restrict__ phi, const double* __restrict__ C,
                        const double* __restrict__ sigma, int dm_mode, double eps,
                        double* __restrict__ force, double* __restrict__ dm_out) {
  const size_t n = L.ncell();
  const int nd = L.ndim();
  const double inv2h = 0.5 / L.h;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x) {
    int idx[3] = {(int)(c % L.nx), (int)((c / L.nx) % L.ny), (int)(c / ((size_t)L.nx * L.ny))};
    double gs[3] = {0, 0, 0}, nn[3] = {0, 0, 0}, ndg = 0.0;
    for (int d = 0; d < nd; ++d) {
      int pp[3] = {idx[0], idx[1], idx[2]}, pm[3] = {idx[0], idx[1], idx[2]};
      pp[d] = min(pp[d] + 1, L.extent(d) - 1);
      pm[d] = max(pm[d] - 1, 0);
      gs[d] = (sigma[cidx(L, pp[0], pp[1], pp[2])] - sigma[cidx(L, pm[0], pm[1], pm[2])]) * inv2h;
      nn[d] = normal_comp(L, phi, idx[0], idx[1], idx[2], d, eps);
      ndg += nn[d] * gs[d];
    }
    double dm;
    if (dm_mode == 0) {
      double q = 0.0;
      for (int d = 0; d < nd; ++d) {
        int pp[3] = {idx[0], idx[1], idx[2]}, pm[3] = {idx[0], idx[1], idx[2]};
        pp[d] = min(pp[d] + 1, L.extent(d) - 1);
        pm[d] = max(pm[d] - 1, 0);
        double g = (C[cidx(L, pp[0], pp[1], pp[2])] - C[cidx(L, pm[0], pm[1], pm[2])]) * inv2h;
        q += g * g;
      }
      dm = sqrt(q);
    } else {
      double Cc = C[c];
      // interface cells: 1e-6 < C < 1 - 1e-6 (nearer fractions are the
      // round-off of empty or full cells)
      if (Cc > 1e-6 && Cc < 1.0 - 1e-6) {
        // Youngs normal: minus the (1,2,1)-weighted gradient of C
        double m[3] = {0, 0, 0};
        int kr = nd == 3 ? 1 : 0;
        for (int dk = -kr; dk <= kr; ++dk)
          for (int dj = -1; dj <= 1; ++dj)
            for (int di = -1; di <= 1; ++di) {
              int a = min(max(idx[0] + di, 0), L.nx - 1);
              int b = min(max(idx[1] + dj, 0), L.ny - 1);
              int e = min(max(idx[2] + dk, 0), L.nz - 1);
              double w = (di == 0 ? 2.0 : 1.0) * (dj == 0 ? 2.0 : 1.0) *
                         (nd == 3 ? (dk == 0 ? 2.0 : 1.0) : 1.0);
              double v = C[cidx(L, a, b, e)];
              m[0] -= w * di * v;
              m[1] -= w * dj * v;
              m[2] -= w * dk * v;
            }
        dm = plic_unit_area(nd, m, Cc) / L.h;
      } else {
        dm = 0.0;
      }
    }
    for (int d = 0; d < nd; ++d) force[(size_t)d * n + c] = dm * (gs[d] - nn[d] * ndg);
    if (dm_out) dm_out[c] = dm;
  }
}

// Loss L = sum_c V_c |F_Ma,c|^2: block partials of the sum and, when G is
// given, G_c = dL/d(grad sigma)_c = 2 V_c delta_m,c F_Ma,c (F_Ma is already
// tangential, so the projector (I - n n) maps it to itself).
__global__ void k_loss_partials(Level L, const double* __restrict__ force,
                                const double* __restrict__ dm, double* __restrict__ G,
                                double* __restrict__ part) {
  const size_t n = L.ncell();
  const int nd = L.ndim();
  double s = 0.0, e = 0.0;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x) {
    const double V = cell_volume(L, (int)(c % L.nx));
    double q = 0.0;
    for (int d = 0; d < nd; ++d) {
      const double Fd = force[(size_t)d * n + c];
      q += Fd * Fd;
      if (G) G[(size_t)d * n + c] = 2.0 * V * dm[c] * Fd;
    }
    double u, w;
    two_sum(s, V * q, u, w);
    s = u;
    e += w;
  }
  block_sum_comp<kTotThreads>(s, e);
  if (threadIdx.x == 0) {
    part[2 * (size_t)blockIdx.x] = s;
    part[2 * (size_t)blockIdx.x + 1] = e;
  }
}

// dL/df: the transpose of the centred gradient with its one-sided copies at
// walls (grad sigma_c = (sigma_{c+} - sigma_{c-})/2h, c+ = c at the upper
// wall, c- = c at the lower one) gives dL/dsigma; then through the EOS and
// Gamma = f/delta_phi.
__global__ void k_loss_grad(Level L, EosArgs q, const double* __restrict__ f,
                            const double* __restrict__ phi, const double* __restrict__ G,
                            double* __restrict__ out) {
  const size_t n = L.ncell();
  const int nd = L.ndim();
  const double inv2h = 0.5 / L.h;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x) {
    const int idx[3] = {(int)(c % L.nx), (int)((c / L.nx) % L.ny),
                        (int)(c / ((size_t)L.nx * L.ny))};
    double g = 0.0;
    for (int d = 0; d < nd; ++d) {
      const double* Gd = G + (size_t)d * n;
      const size_t st = d == 0 ? 1 : (d == 1 ? (size_t)L.nx : (size_t)L.nx * L.ny);
      const int p = idx[d], m = L.extent(d);
      if (p >= 1) g += Gd[c - st];
      if (p == m - 1) g += Gd[c];
      if (p <= m - 2) g -= Gd[c + st];
      if (p == 0) g -= Gd[c];
    }
    g *= inv2h;
    const double ph = phi[c];
    const double del = ph * (1.0 - ph) / q.eps;
    out[c] = del >= 1e-3 / q.eps ? g * eos_slope(q, f[c] / del) / del : 0.0;
  }
}

}  // namespace

sfx_status marangoni_loss(sfx_ctx* c, const sfx_params* p, const double* f, const double* phi,
                          const double* C, int dm_mode, double* loss, double* grad,
                          cudaStream_t s) {
  sfx_status st = adj_ensure_scratch(c);
  if (st != SFX_OK) return st;
  const Level& L = c->lev[0].lv;
  const size_t n = L.ncell();
  const int nb = blocks_for(n, 256);
  EosArgs q{p->gamma_inf, p->eps, p->sigma0, p->E, p->eos};
  SFX_KERNEL(c, K_FORCES, k_eos<double>, nb, 256, s, n, q, f, phi, c->adj.sig);
  SFX_KERNEL(c, K_FORCES, k_force<double>, nb, 256, s, L, phi, C, c->adj.sig, dm_mode, p->eps,
             c->adj.force, c->adj.dm);
  const int nbp = c->adj.nblk;
  SFX_KERNEL(c, K_FORCES, k_loss_partials, nbp, kTotThreads, s, L, c->adj.force, c->adj.dm,
             grad ? c->adj.G : nullptr, c->adj.part);
  SFX_KERNEL(c, K_FORCES, k_total_final, 1, kTotThreads, s, c->adj.part, nbp, c->adj.d_out);
  if (grad)
    SFX_KERNEL(c, K_FORCES, k_loss_grad, nb, 256, s, L, q, f, phi, c->adj.G, grad);
  SFX_LAUNCH_CHECK();
  SFX_CUDA(cudaMemcpyAsync(c->adj.h_out, c->adj.d_out, sizeof(double), cudaMemcpyDeviceToHost, s));
  SFX_CUDA(cudaStreamSynchronize(s));
  *loss = c->adj.h_out[0];
  return SFX_OK;
}

sfx_status totals(sfx_ctx* c, const double* const* fields, int nf, double* out, cudaStream_t s) {
  const Level& L = c->lev[0].lv;
  const int nblk = c->n_partial_blocks;
  for (int i = 0; i < nf; ++i)
    SFX_KERNEL(c, K_TOTALS, k_total_partials, nblk, kTotThreads, s, L, fields[i], i, c->partials);
  SFX_KERNEL(c, K_TOTALS, k_total_final, nf, kTotThreads, s, c->partials, nblk, c->d_sums);
  SFX_LAUNCH_CHECK();
  SFX_CUDA(cudaMemcpyAsync(c->h_sums, c->d_sums, nf * sizeof(double), cudaMemcpyDeviceToHost, s));
  SFX_CUDA(cudaStreamSynchronize(s));
  memcpy(out, c->h_sums, nf * sizeof(double));
  return SFX_OK;
}

sfx_status marangoni(sfx_ctx* c, const sfx_params* p, const double* f, const void* phi,
                     const double* C, int dm_mode, double* sigma, double* force,
                     cudaStream_t s) {
  const Level& L = c->lev[0].lv;
  const size_t n = L.ncell();
  EosArgs q{p->gamma_inf, p->eps, p->sigma0, p->E, p->eos};
  const int nb = blocks_for(n, 256);
  SFX_KERNEL(c, K_FORCES, k_eos<double>, nb, 256, s, n, q, f, (const double*)phi, sigma);
  SFX_KERNEL(c, K_FORCES, k_force<double>, nb, 256, s, L, (const double*)phi, C, sigma, dm_mode,
             p->eps, force, (double*)nullptr);
  SFX_LAUNCH_CHECK();
  return SFX_OK;
}

}  // namespace sfx
