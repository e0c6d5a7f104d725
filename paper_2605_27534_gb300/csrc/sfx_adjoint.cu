// Discrete adjoint of the no-flow coupled step (App. C), FP64.
//
// One step solves R(x1; x0, theta) = 0 for x1 = (f, F) with the residual of
// both App. C equations
//   R_f = (f* - f)/dt + N_f f + q,   R_F = (F* - F)/dt + N_F F - q,
//   q = k_a F (f_inf - f)/(phi + eta) - k_d f,
// N the finite-volume flux divergence of Sec. 3.1-3.2 (diffusivity D and
// drift B, both proportional to D) and f* = f^n, F* = F^n.  With
// -J = -dR/dx1 = [[a - N_f, -b], [-d, e - N_F]] per cell, where
//   a = 1/dt + k_d + c1 F,  b = c1 (f_inf - f),  d = c1 F + k_d,
//   e = 1/dt + b,  c1 = k_a/(phi + eta),
// a loss gradient lam1 = dL/dx1 pulls back by solving
//   (-J)^T nu = lam1,   lam0 = nu/dt,   dL/dtheta += (dR/dtheta)^T nu,
// with dR_f/dk_a = F (f_inf - f)/(phi + eta) = -dR_F/dk_a,
// dR_f/dk_d = -f = -dR_F/dk_d, dR_f/dD_f = N^_f f and dR_F/dD_F = N^_F F
// (N^ at unit diffusivity).  The transposed system is solved by defect
// correction: the FP64 residual r = lam - (-J)^T nu decides convergence and
// the correction e of (-J)^T e = r is relaxed by FP32 red-black Gauss-Seidel
// with a 2x2 solve per cell (the coupling is pointwise) on coefficients
// precomputed once per step from the FP64 operator.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "sfx_internal.h"
#include "sfx_op64.cuh"

namespace sfx {
namespace {

constexpr int kAdjThreads = 256;

struct AdjP {
  Level L;
  double Df, DF, inv_dt, ka, kd, ginf, eps, eta;
  int literal;
  const double* Bf[3];   // unit-diffusivity drift faces
  const double* BF[3];
};

__device__ __forceinline__ Op op_of(const AdjP& p, int field, double D) {
  Op o;
  o.D = D;
  for (int d = 0; d < 3; ++d) o.B[d] = field ? p.BF[d] : p.Bf[d];
  o.literal = p.literal;
  o.lam = nullptr;
  o.Bs = D;
  return o;
}

struct Kin {
  double a, b, d, e, c1, finf, pe;
};

__device__ __forceinline__ Kin kin_at(const AdjP& p, double ph, double f, double F) {
  Kin k;
  k.pe = ph + p.eta;
  k.c1 = p.ka / k.pe;
  k.finf = p.ginf * ph * (1.0 - ph) / p.eps;
  k.b = k.c1 * (k.finf - f);
  k.d = k.c1 * F + p.kd;
  k.a = p.inv_dt + p.kd + k.c1 * F;
  k.e = p.inv_dt + k.b;
  return k;
}

__device__ __forceinline__ void cell_ijk(const Level& L, size_t c, int& i, int& j, int& k) {
  i = (int)(c % L.nx);
  j = (int)((c / L.nx) % L.ny);
  k = (int)(c / ((size_t)L.nx * L.ny));
}

// out = (-J) v, or (-J)^T v with transpose != 0
__global__ void k_adj_apply(AdjP p, const double* __restrict__ phi, const double* __restrict__ f,
                            const double* __restrict__ F, const double* __restrict__ vf,
                            const double* __restrict__ vF, int transpose,
                            double* __restrict__ of, double* __restrict__ oF) {
  const Level& L = p.L;
  const size_t n = L.ncell();
  const Op opf = op_of(p, 0, p.Df), opF = op_of(p, 1, p.DF);
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x) {
    int i, j, k;
    cell_ijk(L, c, i, j, k);
    const Kin q = kin_at(p, phi[c], f[c], F[c]);
    double Nf, NF;
    if (!transpose) {
      double sd, sn;
      const double iv = 1.0 / cell_volume(L, i);
      flux_terms(L, opf, vf, i, j, k, sd, sn);
      Nf = (sd * vf[c] + sn) * iv;
      flux_terms(L, opF, vF, i, j, k, sd, sn);
      NF = (sd * vF[c] + sn) * iv;
      of[c] = q.a * vf[c] - Nf - q.b * vF[c];
      oF[c] = -q.d * vf[c] + q.e * vF[c] - NF;
    } else {
      double dT, nT;
      flux_terms_T(L, opf, vf, i, j, k, dT, nT);
      Nf = dT * vf[c] + nT;
      flux_terms_T(L, opF, vF, i, j, k, dT, nT);
      NF = dT * vF[c] + nT;
      of[c] = q.a * vf[c] - Nf - q.d * vF[c];
      oF[c] = -q.b * vf[c] + q.e * vF[c] - NF;
    }
  }
}

// nu = dt lam: the solution when transport is negligible against 1/dt
__global__ void k_adj_init(size_t n, double dt, const double* __restrict__ lf,
                           const double* __restrict__ lF, double* __restrict__ nf,
                           double* __restrict__ nF) {
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x) {
    nf[c] = dt * lf[c];
    nF[c] = dt * lF[c];
  }
}

// r = lam - (-J)^T nu (rounded to float into rout), max |r| and max |lam|
// over both fields
__global__ void k_adj_resid(AdjP p, const double* __restrict__ phi, const double* __restrict__ f,
                            const double* __restrict__ F, const double* __restrict__ lf,
                            const double* __restrict__ lF, const double* __restrict__ nf,
                            const double* __restrict__ nF, float2* __restrict__ rout,
                            unsigned long long* nrm) {
  const Level& L = p.L;
  const size_t n = L.ncell();
  const Op opf = op_of(p, 0, p.Df), opF = op_of(p, 1, p.DF);
  double mr = 0.0, mb = 0.0;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x) {
    int i, j, k;
    cell_ijk(L, c, i, j, k);
    const Kin q = kin_at(p, phi[c], f[c], F[c]);
    double dT, nT;
    flux_terms_T(L, opf, nf, i, j, k, dT, nT);
    const double rf = lf[c] - (q.a * nf[c] - (dT * nf[c] + nT) - q.d * nF[c]);
    flux_terms_T(L, opF, nF, i, j, k, dT, nT);
    const double rF = lF[c] - (-q.b * nf[c] + q.e * nF[c] - (dT * nF[c] + nT));
    rout[c] = make_float2((float)rf, (float)rF);
    double r = fmax(fabs(rf), fabs(rF));
    if (!(r <= 1e300)) r = INFINITY;   // NaN or Inf: never converged
    mr = fmax(mr, r);
    mb = fmax(mb, fmax(fabs(lf[c]), fabs(lF[c])));
  }
  mr = warp_max(mr);
  mb = warp_max(mb);
  if ((threadIdx.x & 31) == 0) {
    atomic_max_nonneg(&nrm[0], mr);
    atomic_max_nonneg(&nrm[1], mb);
  }
}

// Coefficients of the FP32 relaxation: per cell the inverse of the 2x2
// block [[A11, -d], [-b, A22]] of (-J)^T (A11 = a - dT_f, A22 = e - dT_F) as
// (A22, d, b, A11)/det, and the neighbour weights of N^T of both fields
// (W[q N + c] for f, W[(6 + q) N + c] for F).
__global__ void k_adj_coef(AdjP p, const double* __restrict__ phi, const double* __restrict__ f,
                           const double* __restrict__ F, float4* __restrict__ K,
                           float* __restrict__ W) {
  const Level& L = p.L;
  const size_t n = L.ncell();
  const Op opf = op_of(p, 0, p.Df), opF = op_of(p, 1, p.DF);
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x) {
    int i, j, k;
    cell_ijk(L, c, i, j, k);
    const Kin q = kin_at(p, phi[c], f[c], F[c]);
    double dTf, dTF, wf[6], wF[6];
    flux_weights_T(L, opf, i, j, k, dTf, wf);
    flux_weights_T(L, opF, i, j, k, dTF, wF);
    const double A11 = q.a - dTf, A22 = q.e - dTF;
    const double idet = 1.0 / (A11 * A22 - q.d * q.b);
    K[c] = make_float4((float)(A22 * idet), (float)(q.d * idet), (float)(q.b * idet),
                       (float)(A11 * idet));
#pragma unroll
    for (int m = 0; m < 6; ++m) {
      W[(size_t)m * n + c] = (float)wf[m];
      W[(size_t)(6 + m) * n + c] = (float)wF[m];
    }
  }
}

// One colour of the FP32 red-black Gauss-Seidel on (-J)^T e = r
__global__ void k_adj_csweep(Level L, const float4* __restrict__ K, const float* __restrict__ W,
                             const float2* __restrict__ r, float2* __restrict__ e, int color) {
  const int j = blockIdx.y, k = blockIdx.z;
  const int i = 2 * (blockIdx.x * blockDim.x + threadIdx.x) + ((j + k + color) & 1);
  if (i >= L.nx) return;
  const size_t n = L.ncell();
  const size_t c = cidx(L, i, j, k);
  const size_t sy = (size_t)L.nx, sz = (size_t)L.nx * L.ny;
  const bool has[6] = {i > 0, i + 1 < L.nx, j > 0, j + 1 < L.ny,
                       L.geom == SFX_CART3D && k > 0, L.geom == SFX_CART3D && k + 1 < L.nz};
  const size_t nb[6] = {c - 1, c + 1, c - sy, c + sy, c - sz, c + sz};
  const float2 rc = r[c];
  float sf = rc.x, sF = rc.y;
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    if (!has[m]) continue;
    const float2 v = e[nb[m]];
    sf += W[(size_t)m * n + c] * v.x;
    sF += W[(size_t)(6 + m) * n + c] * v.y;
  }
  const float4 q = K[c];
  e[c] = make_float2(q.x * sf + q.y * sF, q.z * sf + q.w * sF);
}

// nu += e
__global__ void k_adj_add(size_t n, const float2* __restrict__ e, double* __restrict__ nf,
                          double* __restrict__ nF) {
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x) {
    const float2 v = e[c];
    nf[c] += (double)v.x;
    nF[c] += (double)v.y;
  }
}

// lam0 = nu/dt (in place) and block partials of the four parameter terms
__global__ void k_adj_finish(AdjP p, const double* __restrict__ phi, const double* __restrict__ f,
                             const double* __restrict__ F, const double* __restrict__ nf,
                             const double* __restrict__ nF, double* __restrict__ lf,
                             double* __restrict__ lF, double* __restrict__ part) {
  const Level& L = p.L;
  const size_t n = L.ncell();
  const Op ohf = op_of(p, 0, 1.0), ohF = op_of(p, 1, 1.0);
  double s[4] = {0, 0, 0, 0}, e[4] = {0, 0, 0, 0};
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x) {
    int i, j, k;
    cell_ijk(L, c, i, j, k);
    const Kin q = kin_at(p, phi[c], f[c], F[c]);
    const double vf = nf[c], vF = nF[c];
    const double iv = 1.0 / cell_volume(L, i);
    double sd, sn;
    flux_terms(L, ohf, f, i, j, k, sd, sn);
    const double Nhf = (sd * f[c] + sn) * iv;
    flux_terms(L, ohF, F, i, j, k, sd, sn);
    const double NhF = (sd * F[c] + sn) * iv;
    const double t[4] = {(vf - vF) * F[c] * (q.finf - f[c]) / q.pe, -(vf - vF) * f[c],
                         vf * Nhf, vF * NhF};
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      double u, w;
      two_sum(s[m], t[m], u, w);
      s[m] = u;
      e[m] += w;
    }
    lf[c] = vf * p.inv_dt;
    lF[c] = vF * p.inv_dt;
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    block_sum_comp<kAdjThreads>(s[m], e[m]);
    if (threadIdx.x == 0) {
      const size_t o = 2 * ((size_t)m * gridDim.x + blockIdx.x);
      part[o] = s[m];
      part[o + 1] = e[m];
    }
  }
}

// One block per quantity: fixed-order combination of the block partials.
__global__ void k_adj_reduce(const double* __restrict__ part, int nblk, double* __restrict__ out) {
  const int m = blockIdx.x;
  double s = 0.0, e = 0.0;
  for (int q = threadIdx.x; q < nblk; q += blockDim.x) {
    const size_t o = 2 * ((size_t)m * nblk + q);
    double u, w;
    two_sum(s, part[o], u, w);
    s = u;
    e += part[o + 1] + w;
  }
  block_sum_comp<kAdjThreads>(s, e);
  if (threadIdx.x == 0) out[m] = s + e;
}

__global__ void k_f_from_gamma(size_t n, double inv_eps, const double* __restrict__ gamma,
                               const double* __restrict__ phi, double* __restrict__ f) {
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x) {
    const double p = phi[c];
    f[c] = gamma[c] * (p * (1.0 - p) * inv_eps);
  }
}

AdjP make_params(sfx_ctx* c, const sfx_params* pr, double dt) {
  AdjP p;
  p.L = c->lev[0].lv;
  p.Df = pr->Df;
  p.DF = pr->DF;
  p.inv_dt = 1.0 / dt;
  p.ka = pr->ka;
  p.kd = pr->kd;
  p.ginf = pr->gamma_inf;
  p.eps = pr->eps;
  p.eta = pr->eta;
  p.literal = pr->literal_upwind;
  const int nd = p.L.ndim();
  for (int d = 0; d < 3; ++d) {
    p.Bf[d] = d < nd ? c->adj.Bf[d] : nullptr;
    p.BF[d] = d < nd ? c->adj.BF[d] : nullptr;
  }
  return p;
}

sfx_status unit_drifts(sfx_ctx* c, const sfx_params* pr, const double* phi, cudaStream_t s) {
  return drift_faces64(c, phi, 1.0, 1.0, pr->eps, c->adj.Bf, c->adj.BF, s);
}

// The relaxation of one check as a graph, captured once per context and
// sweep count: every argument is context scratch, so it never goes stale.
// At 256^2 a colour sweep takes a few microseconds, and issuing the 2 S + 2
// launches one by one left the step bound by the host.
sfx_status relax_graph(sfx_ctx* c, const Level& L, int sweeps) {
  if (c->adj.relax && c->adj.relax_sweeps == sweeps) return SFX_OK;
  if (c->adj.relax) {
    cudaGraphExecDestroy(c->adj.relax);
    c->adj.relax = nullptr;
  }
  if (!c->adj.cap) SFX_CUDA(cudaStreamCreateWithFlags(&c->adj.cap, cudaStreamNonBlocking));
  cudaStream_t cs = c->adj.cap;
  const size_t n = L.ncell();
  dim3 blk(128), grd((unsigned)(((L.nx + 1) / 2 + 127) / 128), (unsigned)L.ny, (unsigned)L.nz);
  SFX_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  cudaMemsetAsync(c->adj.e, 0, n * sizeof(float2), cs);
  for (int q = 0; q < sweeps; ++q)
    for (int color = 0; color < 2; ++color)
      k_adj_csweep<<<grd, blk, 0, cs>>>(L, c->adj.K, c->adj.W, c->adj.r, c->adj.e, color);
  k_adj_add<<<blocks_for(n, kAdjThreads), kAdjThreads, 0, cs>>>(n, c->adj.e, c->adj.nf,
                                                                c->adj.nF);
  const cudaError_t le = cudaGetLastError();
  cudaGraph_t g = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(cs, &g);
  cudaError_t ie = cudaSuccess;
  cudaGraphExec_t ex = nullptr;
  if (le == cudaSuccess && ce == cudaSuccess) ie = cudaGraphInstantiate(&ex, g, 0);
  if (g) cudaGraphDestroy(g);
  SFX_CUDA(le);
  SFX_CUDA(ce);
  SFX_CUDA(ie);
  c->adj.relax = ex;
  c->adj.relax_sweeps = sweeps;
  return SFX_OK;
}

}  // namespace

sfx_status adj_ensure_scratch(sfx_ctx* c) {
  if (c->adj.ready) return SFX_OK;
  const Level& L = c->lev[0].lv;
  const size_t n = L.ncell();
  auto get = [&](size_t bytes, void** p) -> sfx_status {
    SFX_CUDA(cudaMalloc(p, bytes ? bytes : 8));
    c->allocations.push_back(*p);
    return SFX_OK;
  };
  sfx_status st;
  for (int d = 0; d < L.ndim(); ++d) {
    if ((st = get(L.nface(d) * sizeof(double), (void**)&c->adj.Bf[d])) != SFX_OK) return st;
    if ((st = get(L.nface(d) * sizeof(double), (void**)&c->adj.BF[d])) != SFX_OK) return st;
  }
  double** cells[4] = {&c->adj.nf, &c->adj.nF, &c->adj.sig, &c->adj.dm};
  for (double** q : cells)
    if ((st = get(n * sizeof(double), (void**)q)) != SFX_OK) return st;
  if ((st = get(3 * n * sizeof(double), (void**)&c->adj.force)) != SFX_OK) return st;
  if ((st = get(3 * n * sizeof(double), (void**)&c->adj.G)) != SFX_OK) return st;
  c->adj.nblk = std::min(blocks_for(n, kAdjThreads), 1024);
  if ((st = get((size_t)c->adj.nblk * 2 * 5 * sizeof(double), (void**)&c->adj.part)) != SFX_OK)
    return st;
  if ((st = get(8 * sizeof(double), (void**)&c->adj.d_out)) != SFX_OK) return st;
  if ((st = get(2 * sizeof(unsigned long long), (void**)&c->adj.d_nrm)) != SFX_OK) return st;
  if ((st = get(n * sizeof(float4), (void**)&c->adj.K)) != SFX_OK) return st;
  if ((st = get(12 * n * sizeof(float), (void**)&c->adj.W)) != SFX_OK) return st;
  if ((st = get(n * sizeof(float2), (void**)&c->adj.r)) != SFX_OK) return st;
  if ((st = get(n * sizeof(float2), (void**)&c->adj.e)) != SFX_OK) return st;
  SFX_CUDA(cudaMallocHost((void**)&c->adj.h_out, 8 * sizeof(double)));
  SFX_CUDA(cudaMallocHost((void**)&c->adj.h_nrm, 2 * sizeof(unsigned long long)));
  c->adj.ready = true;
  return SFX_OK;
}

sfx_status f_from_gamma(sfx_ctx* c, const double* gamma, const double* phi, double eps,
                        double* f, cudaStream_t s) {
  const size_t n = c->lev[0].lv.ncell();
  SFX_KERNEL(c, K_OTHER, k_f_from_gamma, blocks_for(n, 256), 256, s, n, 1.0 / eps, gamma, phi, f);
  SFX_LAUNCH_CHECK();
  return SFX_OK;
}

sfx_status adjoint_apply(sfx_ctx* c, const sfx_params* pr, const double* phi, const double* f,
                         const double* F, double dt, int transpose, const double* vf,
                         const double* vF, double* of, double* oF, cudaStream_t s) {
  sfx_status st = adj_ensure_scratch(c);
  if (st != SFX_OK) return st;
  if ((st = unit_drifts(c, pr, phi, s)) != SFX_OK) return st;
  const AdjP p = make_params(c, pr, dt);
  const size_t n = p.L.ncell();
  SFX_KERNEL(c, K_OTHER, k_adj_apply, blocks_for(n, 256), 256, s, p, phi, f, F, vf, vF,
             transpose, of, oF);
  SFX_LAUNCH_CHECK();
  return SFX_OK;
}

sfx_status adjoint_step(sfx_ctx* c, const sfx_params* pr, const double* phi, const double* f,
                        const double* F, double dt, double* lf, double* lF, double* dparams,
                        const sfx_solve_opts* o, sfx_step_stats* stats, cudaStream_t s) {
  sfx_status st = adj_ensure_scratch(c);
  if (st != SFX_OK) return st;
  if ((st = unit_drifts(c, pr, phi, s)) != SFX_OK) return st;
  const AdjP p = make_params(c, pr, dt);
  const Level& L = p.L;
  const size_t n = L.ncell();
  const int nb = blocks_for(n, kAdjThreads);
  double* nf = c->adj.nf;
  double* nF = c->adj.nF;
  SFX_KERNEL(c, K_SETUP, k_adj_init, nb, kAdjThreads, s, n, dt, lf, lF, nf, nF);
  SFX_KERNEL(c, K_SETUP, k_adj_coef, nb, kAdjThreads, s, p, phi, f, F, c->adj.K, c->adj.W);
  const int sweeps = std::max(1, o->nu1 + o->nu2);
  if ((st = relax_graph(c, L, sweeps)) != SFX_OK) return st;
  bool conv = false;
  double rel = INFINITY;
  int checks = 0, total_sweeps = 0;
  for (checks = 1; checks <= o->max_cycles; ++checks) {
    // FP64 residual of the current nu: the convergence test and the defect
    SFX_CUDA(cudaMemsetAsync(c->adj.d_nrm, 0, 2 * sizeof(unsigned long long), s));
    SFX_KERNEL(c, K_RESIDUAL, k_adj_resid, nb, kAdjThreads, s, p, phi, f, F, lf, lF, nf, nF,
               c->adj.r, c->adj.d_nrm);
    SFX_LAUNCH_CHECK();
    SFX_CUDA(cudaMemcpyAsync(c->adj.h_nrm, c->adj.d_nrm, 2 * sizeof(unsigned long long),
                             cudaMemcpyDeviceToHost, s));
    SFX_CUDA(cudaStreamSynchronize(s));
    double r, b;
    memcpy(&r, &c->adj.h_nrm[0], sizeof(double));
    memcpy(&b, &c->adj.h_nrm[1], sizeof(double));
    if (!std::isfinite(r)) return SFX_ERR_NONFINITE;
    rel = r / (b > 1e-300 ? b : 1e-300);
    if (b == 0.0 || rel <= o->tol) {
      conv = true;
      break;
    }
    if (checks == o->max_cycles) break;
    // FP32 relaxation of the defect equation from e = 0, then nu += e (one
    // graph launch; the profile counts its kernels and times it as a whole)
    prof_before(c, K_SMOOTH_FINE, s);
    SFX_CUDA(cudaGraphLaunch(c->adj.relax, s));
    prof_after(c, K_SMOOTH_FINE, s);
    c->prof.launches[K_SMOOTH_FINE] += 2 * sweeps - 1;
    c->prof.launches[K_OTHER] += 1;
    total_sweeps += sweeps;
  }
  const int nbf = c->adj.nblk;
  SFX_KERNEL(c, K_OTHER, k_adj_finish, nbf, kAdjThreads, s, p, phi, f, F, nf, nF, lf, lF,
             c->adj.part);
  SFX_KERNEL(c, K_OTHER, k_adj_reduce, 4, kAdjThreads, s, c->adj.part, nbf, c->adj.d_out);
  SFX_LAUNCH_CHECK();
  SFX_CUDA(cudaMemcpyAsync(c->adj.h_out, c->adj.d_out, 4 * sizeof(double),
                           cudaMemcpyDeviceToHost, s));
  SFX_CUDA(cudaStreamSynchronize(s));
  if (dparams)
    for (int m = 0; m < 4; ++m) dparams[m] += c->adj.h_out[m];
  if (stats) {
    stats->picard = std::min(checks, o->max_cycles);
    stats->vcycles = total_sweeps;
    stats->res_f = rel;
    stats->res_F = rel;
    stats->mass_f = 0.0;
    stats->mass_F = 0.0;
    stats->converged = conv ? 1 : 0;
  }
  return conv ? SFX_OK : SFX_ERR_NOT_CONVERGED;
}

}  // namespace sfx
