// C-ABI of libsfx: argument checks, the context (multigrid pyramid and work
// arrays) and dispatch to the kernels of the other translation units.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "sfx_internal.h"

namespace sfx {

static thread_local char g_cuda_err[256] = "";

sfx_status cuda_fail(cudaError_t e) {
  snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
  return SFX_ERR_CUDA;
}

void prof_before(sfx_ctx* c, int kind, cudaStream_t s) {
  Prof& P = c->prof;
  P.launches[kind]++;
  if (!P.on || P.used >= 8192) return;
  if (P.ev.size() < 2 * (P.used + 1)) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return;
    if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return; }
    P.ev.push_back(a);
    P.ev.push_back(b);
  }
  cudaEventRecord(P.ev[2 * P.used], s);
}

void prof_after(sfx_ctx* c, int kind, cudaStream_t s) {
  Prof& P = c->prof;
  if (!P.on || P.used >= 8192 || P.ev.size() < 2 * (P.used + 1)) return;
  cudaEventRecord(P.ev[2 * P.used + 1], s);
  if (P.kind.size() <= P.used) P.kind.push_back(kind);
  else P.kind[P.used] = kind;
  P.used++;
}

namespace {

template <typename T>
sfx_status dalloc(sfx_ctx* c, T** p, size_t n) {
  *p = nullptr;
  if (n == 0) n = 1;
  void* q = nullptr;
  SFX_CUDA(cudaMalloc(&q, n * sizeof(T)));
  c->allocations.push_back(q);
  *p = (T*)q;
  return SFX_OK;
}

bool grid_ok(const sfx_grid* g) {
  if (!g) return false;
  if (g->geom < SFX_PLANAR2D || g->geom > SFX_CART3D) return false;
  if (g->nx < 1 || g->ny < 1 || g->nz < 1) return false;
  if (g->geom != SFX_CART3D && g->nz != 1) return false;
  if (!(g->h > 0.0) || !std::isfinite(g->h)) return false;
  if ((size_t)g->nx * g->ny * g->nz > ((size_t)1 << 34)) return false;
  return true;
}

bool opts_ok(const sfx_solve_opts* o) {
  return o->tol > 0.0 && o->max_cycles >= 1 && o->nu1 >= 0 && o->nu2 >= 0 && o->vcycles >= 1 &&
         o->check_every >= 1 && o->coarse_sweeps >= 1 && o->mg_levels >= 0 &&
         o->nu1 + o->nu2 >= 1;
}

bool params_ok(const sfx_params* p) {
  return p && p->ka >= 0.0 && p->kd >= 0.0 && p->gamma_inf > 0.0 && p->Df >= 0.0 &&
         p->DF >= 0.0 && p->eps > 0.0 && p->eta >= 0.0 && p->eos >= 0 && p->eos <= 2 &&
         std::isfinite(p->ka) && std::isfinite(p->kd) && std::isfinite(p->Df) &&
         std::isfinite(p->DF) && std::isfinite(p->eps);
}

cudaStream_t S(void* s) { return (cudaStream_t)s; }

sfx_status build_levels(sfx_ctx* c) {
  Level L{c->grid.geom, c->grid.nx, c->grid.ny, c->grid.nz, c->grid.h};
  const bool is3 = L.geom == SFX_CART3D;
  for (;;) {
    LevelData D;
    D.lv = L;
    c->lev.push_back(D);
    bool even = L.nx % 2 == 0 && L.ny % 2 == 0 && (!is3 || L.nz % 2 == 0);
    if (!even || L.ncell() <= 64 || (int)c->lev.size() >= 16) break;
    Level Cc{L.geom, L.nx / 2, L.ny / 2, is3 ? L.nz / 2 : 1, 2.0 * L.h};
    if (Cc.nx < 2 || Cc.ny < 2 || (is3 && Cc.nz < 2)) break;
    L = Cc;
  }
  for (size_t l = 0; l < c->lev.size(); ++l) {
    LevelData& D = c->lev[l];
    const Level& V = D.lv;
    const int nd = V.ndim();
    sfx_status st;
    if (l > 0 && (st = dalloc(c, &D.a, V.ncell())) != SFX_OK) return st;
    if ((st = dalloc(c, &D.b, V.ncell())) != SFX_OK) return st;
    if ((st = dalloc(c, &D.lam, V.ncell())) != SFX_OK) return st;
    for (int d = 0; d < nd; ++d) {
      for (int fld = 0; fld < 2; ++fld)
        if ((st = dalloc(c, &D.B[fld][d], V.nface(d))) != SFX_OK) return st;
      if (l > 0 && (st = dalloc(c, &D.Bg[d], V.nface(d))) != SFX_OK) return st;
    }
  }
  return SFX_OK;
}

}  // namespace
}  // namespace sfx

using namespace sfx;

extern "C" {

const char* sfx_version(void) { return "libsfx 0.1 (sm_103a)"; }

const char* sfx_status_string(sfx_status s) {
  switch (s) {
    case SFX_OK: return "ok";
    case SFX_ERR_ARG: return "invalid argument";
    case SFX_ERR_NOT_CONVERGED: return "not converged";
    case SFX_ERR_NONFINITE: return "non-finite value in a residual";
    case SFX_ERR_TIMEOUT: return "device wait timed out";
    case SFX_ERR_CUDA: return "CUDA error";
    case SFX_ERR_WORKSPACE: return "workspace too small";
  }
  return "unknown status";
}

const char* sfx_last_cuda_error(void) { return g_cuda_err; }

void sfx_default_opts(sfx_solve_opts* o) {
  if (!o) return;
  o->tol = 1e-10;
  o->max_cycles = 200;
  o->nu1 = 2;
  o->nu2 = 2;
  o->mg_levels = 0;
  o->vcycles = 1;
  o->check_every = 1;
  o->coarse_sweeps = 40;
}

void sfx_ctx_destroy(sfx_ctx* c) {
  if (!c) return;
  for (cudaEvent_t e : c->prof.ev) cudaEventDestroy(e);
  for (cudaEvent_t e : c->f32.ev)
    if (e) cudaEventDestroy(e);
  for (void* p : c->allocations) cudaFree(p);
  if (c->h_norms) cudaFreeHost(c->h_norms);
  if (c->h_sums) cudaFreeHost(c->h_sums);
  if (c->adj.h_out) cudaFreeHost(c->adj.h_out);
  if (c->adj.h_nrm) cudaFreeHost(c->adj.h_nrm);
  if (c->adj.relax) cudaGraphExecDestroy(c->adj.relax);
  if (c->adj.cap) cudaStreamDestroy(c->adj.cap);
  delete c;
}

sfx_status sfx_ctx_create(const sfx_grid* grid, int precision, sfx_ctx** out) {
  if (!out) return SFX_ERR_ARG;
  *out = nullptr;
  if (!grid_ok(grid) || (precision != SFX_F64 && precision != SFX_F32)) return SFX_ERR_ARG;
  if (precision == SFX_F32) {
    // the FP32 kernels index cells, faces and the colour-packed work arrays
    // with 32-bit integers
    const size_t nx = grid->nx, ny = grid->ny, nz = grid->nz;
    const size_t most = std::max({(nx + 1) * ny * nz, nx * (ny + 1) * nz, nx * ny * (nz + 1),
                                  2 * ny * nz * ((nx + 1) / 2)});
    if (most >= ((size_t)1 << 31)) return SFX_ERR_ARG;
  }
  sfx_ctx* c = new sfx_ctx();
  c->grid = *grid;
  c->prec = precision;
  {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
        sms > 0)
      c->sm_count = sms;
  }
  sfx_status st = build_levels(c);
  size_t n = (size_t)grid->nx * grid->ny * grid->nz;
  if (st == SFX_OK) st = dalloc(c, &c->fstar, n);
  if (st == SFX_OK) st = dalloc(c, &c->Fstar, n);
  if (st == SFX_OK) st = dalloc(c, &c->chi0, n);
  if (st == SFX_OK) st = dalloc(c, &c->chi_tmp, n);
  c->n_partial_blocks = kTotalsBlocks;
  if (st == SFX_OK) st = dalloc(c, &c->partials, (size_t)2 * 8 * c->n_partial_blocks);
  if (st == SFX_OK) st = dalloc(c, &c->d_norms, 16);
  if (st == SFX_OK) st = dalloc(c, &c->d_sums, 8);
  if (st == SFX_OK && precision == SFX_F32) st = f32_ensure_scratch(c);
  if (st == SFX_OK) {
    c->d_flag = (int*)(c->d_norms + 7);
    cudaError_t e = cudaMallocHost(&c->h_norms, 16 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMallocHost(&c->h_sums, 8 * sizeof(double));
    if (e != cudaSuccess) st = cuda_fail(e);
  }
  if (st != SFX_OK) {
    sfx_ctx_destroy(c);
    return st;
  }
  *out = c;
  return SFX_OK;
}

sfx_status sfx_phase_field_build(sfx_ctx* c, const double* C, double* chi, void* phi,
                                 void* delta, int iters, double dtau, double eps, void* stream) {
  if (!c || !C || !chi || !phi || iters < 0 || !(dtau > 0.0) || !(eps > 0.0)) return SFX_ERR_ARG;
  return phase_field_build(c, C, chi, phi, delta, iters, dtau, eps, S(stream));
}

sfx_status sfx_phase_field_from_chi(sfx_ctx* c, const double* chi, double* phi, double* delta,
                                    double eps, void* stream) {
  if (!c || !chi || !phi || !(eps > 0.0) || phi == chi || delta == chi) return SFX_ERR_ARG;
  return phase_field_from_chi(c, chi, phi, delta, eps, S(stream));
}

sfx_status sfx_advect(sfx_ctx* c, const void* ux, const void* uy, const void* uz, double dt,
                      const void* xi, double bc_in, void* xi_out, void* stream) {
  if (!c || !ux || !uy || !xi || !xi_out || xi == xi_out || !(dt > 0.0)) return SFX_ERR_ARG;
  if (c->grid.geom == SFX_CART3D && !uz) return SFX_ERR_ARG;
  if (c->prec == SFX_F32)
    return advect32(c, (const float*)ux, (const float*)uy, (const float*)uz, dt,
                    (const float2*)xi, bc_in, (float2*)xi_out, S(stream));
  return advect(c, ux, uy, uz, dt, (const double*)xi, bc_in, (double*)xi_out, S(stream));
}

sfx_status sfx_mg_solve(sfx_ctx* c, double D, const double* Bx, const double* By,
                        const double* Bz, int literal_upwind, const double* lambda,
                        const double* b, double* a, const sfx_solve_opts* opts, int* cycles_out,
                        double* res_out, void* stream) {
  if (!c || !lambda || !b || !a || !(D >= 0.0)) return SFX_ERR_ARG;
  if (c->prec != SFX_F64) return SFX_ERR_ARG;
  sfx_solve_opts o;
  sfx_default_opts(&o);
  if (opts) o = *opts;
  if (!opts_ok(&o)) return SFX_ERR_ARG;
  return mg_solve(c, D, Bx, By, Bz, literal_upwind, lambda, b, a, &o, cycles_out, res_out,
                  S(stream));
}

sfx_status sfx_surfactant_step(sfx_ctx* c, const sfx_params* params, const void* phi,
                               const void* ux, const void* uy, const void* uz, void* f,
                               void* F, double dt, const sfx_solve_opts* opts,
                               sfx_step_stats* stats, void* stream) {
  if (!c || !params_ok(params) || !phi || !f || !F || f == F || !(dt > 0.0) ||
      !std::isfinite(dt))
    return SFX_ERR_ARG;
  if (ux && (!uy || (c->grid.geom == SFX_CART3D && !uz))) return SFX_ERR_ARG;
  sfx_solve_opts o;
  sfx_default_opts(&o);
  if (opts) o = *opts;
  if (!opts_ok(&o)) return SFX_ERR_ARG;
  if (c->prec == SFX_F32)
    return step_f32(c, params, (const double*)phi, (const float*)ux, (const float*)uy,
                    (const float*)uz, (float2*)f, (float2*)F, dt, &o, stats, S(stream));
  return surfactant_step(c, params, phi, ux, uy, uz, (double*)f, (double*)F, dt, &o, stats,
                         S(stream));
}

sfx_status sfx_totals(sfx_ctx* c, const void* const* fields, int n_fields, double* out,
                      void* stream) {
  if (!c || !fields || !out || n_fields < 1 || n_fields > 8) return SFX_ERR_ARG;
  for (int i = 0; i < n_fields; ++i)
    if (!fields[i]) return SFX_ERR_ARG;
  if (c->prec == SFX_F32) return totals32(c, fields, n_fields, out, S(stream));
  return totals(c, (const double* const*)fields, n_fields, out, S(stream));
}

sfx_status sfx_marangoni_force(sfx_ctx* c, const sfx_params* params, const void* f,
                               const void* phi, const void* C, int dm_mode, void* sigma,
                               void* force, void* stream) {
  if (!c || !params_ok(params) || !f || !phi || !force) return SFX_ERR_ARG;
  if (dm_mode != 0 && dm_mode != 1) return SFX_ERR_ARG;
  if (!C) return SFX_ERR_ARG;
  if (c->prec == SFX_F32)
    return marangoni32(c, params, (const float2*)f, (const double*)phi, (const float*)C, dm_mode,
                       (float*)sigma, (float*)force, S(stream));
  if (!sigma) return SFX_ERR_ARG;
  return marangoni(c, params, (const double*)f, phi, (const double*)C, dm_mode, (double*)sigma,
                   (double*)force, S(stream));
}

sfx_status sfx_acdi_step(sfx_ctx* c, const void* ux, const void* uy, const void* uz, double dt,
                         double zeta, double eps, int clip, double* phi, void* stream) {
  if (!c || !phi || !(dt > 0.0) || !std::isfinite(dt)) return SFX_ERR_ARG;
  if (!(eps > 0.0) || !(zeta >= 0.0) || !std::isfinite(eps) || !std::isfinite(zeta))
    return SFX_ERR_ARG;
  if (ux && (!uy || (c->grid.geom == SFX_CART3D && !uz))) return SFX_ERR_ARG;
  return acdi_step(c, ux, uy, uz, dt, zeta, eps, clip ? 1 : 0, phi, S(stream));
}

sfx_status sfx_capillary_force(sfx_ctx* c, const sfx_params* params, const double* phi,
                               const void* C, const void* sigma, void* kappa, void* force,
                               void* stream) {
  if (!c || !params_ok(params) || !phi || !C || !sigma || !force) return SFX_ERR_ARG;
  return capillary(c, params, phi, C, sigma, kappa, force, S(stream));
}

sfx_status sfx_vof_advect(sfx_ctx* c, const void* ux, const void* uy, const void* uz, double dt,
                          int order, double* C, void* stream) {
  if (!c || !ux || !uy || !C || !(dt > 0.0) || !std::isfinite(dt)) return SFX_ERR_ARG;
  if (c->grid.geom == SFX_AXISYM) return SFX_ERR_ARG;
  if (c->grid.geom == SFX_CART3D && !uz) return SFX_ERR_ARG;
  return vof_advect(c, ux, uy, uz, dt, order ? 1 : 0, C, S(stream));
}

sfx_status sfx_f_from_gamma(sfx_ctx* c, const double* gamma, const double* phi, double eps,
                            double* f, void* stream) {
  if (!c || !gamma || !phi || !f || !(eps > 0.0)) return SFX_ERR_ARG;
  return f_from_gamma(c, gamma, phi, eps, f, S(stream));
}

sfx_status sfx_marangoni_loss(sfx_ctx* c, const sfx_params* params, const double* f,
                              const double* phi, const double* C, int dm_mode, double* loss,
                              double* dloss_df, void* stream) {
  if (!c || !params_ok(params) || !f || !phi || !C || !loss) return SFX_ERR_ARG;
  if (dm_mode != 0 && dm_mode != 1) return SFX_ERR_ARG;
  return marangoni_loss(c, params, f, phi, C, dm_mode, loss, dloss_df, S(stream));
}

sfx_status sfx_adjoint_apply(sfx_ctx* c, const sfx_params* params, const double* phi,
                             const double* f, const double* F, double dt, int transpose,
                             const double* vf, const double* vF, double* out_f, double* out_F,
                             void* stream) {
  if (!c || !params_ok(params) || !phi || !f || !F || !vf || !vF || !out_f || !out_F ||
      !(dt > 0.0) || !std::isfinite(dt))
    return SFX_ERR_ARG;
  if (out_f == out_F || out_f == vf || out_f == vF || out_F == vf || out_F == vF)
    return SFX_ERR_ARG;
  return adjoint_apply(c, params, phi, f, F, dt, transpose ? 1 : 0, vf, vF, out_f, out_F,
                       S(stream));
}

sfx_status sfx_adjoint_step(sfx_ctx* c, const sfx_params* params, const double* phi,
                            const double* f, const double* F, double dt, double* lam_f,
                            double* lam_F, double* dparams, const sfx_solve_opts* opts,
                            sfx_step_stats* stats, void* stream) {
  if (!c || !params_ok(params) || !phi || !f || !F || !lam_f || !lam_F || lam_f == lam_F ||
      !(dt > 0.0) || !std::isfinite(dt))
    return SFX_ERR_ARG;
  sfx_solve_opts o;
  sfx_default_opts(&o);
  if (opts) o = *opts;
  if (!opts_ok(&o)) return SFX_ERR_ARG;
  return adjoint_step(c, params, phi, f, F, dt, lam_f, lam_F, dparams, &o, stats, S(stream));
}

sfx_status sfx_cfl_dt(sfx_ctx* c, const void* ux, const void* uy, const void* uz, double D,
                      double eps, double safety, double* dt_out, void* stream) {
  if (!c || !dt_out || !(D > 0.0) || !(eps > 0.0) || !(safety > 0.0)) return SFX_ERR_ARG;
  if (!ux || !uy || (c->grid.geom == SFX_CART3D && !uz)) return SFX_ERR_ARG;
  double umax = 0.0;
  sfx_status st = cfl_umax(c, ux, uy, uz, &umax, S(stream));
  if (st != SFX_OK) return st;
  const double h = c->grid.h;
  const int nd = c->grid.geom == SFX_CART3D ? 3 : 2;
  double dconv = h / (umax + D / eps);
  double ddiff = h * h / (2.0 * nd * D);
  *dt_out = safety * (dconv < ddiff ? dconv : ddiff);
  return SFX_OK;
}

sfx_status sfx_set_tuning(sfx_ctx* c, int key, int value) {
  if (!c) return SFX_ERR_ARG;
  if (key == SFX_TUNE_FUSED_SWEEP && (value == 0 || value == 1)) {
    c->f32.fused = value == 1;
    return SFX_OK;
  }
  if (key == SFX_TUNE_REUSE_DRIFT && (value == 0 || value == 1)) {
    c->f32.reuse_drift = value == 1;
    c->f32.drift_phi = nullptr;
    return SFX_OK;
  }
  if (key == SFX_TUNE_PREDICT && (value == 0 || value == 1)) {
    c->f32.predict = value == 1;
    c->f32.inc_valid = false;
    return SFX_OK;
  }
  if (key == SFX_TUNE_SWEEP_PLANES && (value == 1 || value == 2)) {
    c->f32.sweep_planes = value;
    return SFX_OK;
  }
  if (key == SFX_TUNE_TILED_SWEEP && (value == 0 || value == 1)) {
    c->f32.tiled = value == 1;
    return SFX_OK;
  }
  if (key == SFX_TUNE_F32_INCR_RESID && (value == 0 || value == 1)) {
    c->f32.incr_resid = value == 1;
    return SFX_OK;
  }
  if (key == SFX_TUNE_F32_SOR && (value == 0 || value == 1 || (value > 1000 && value < 2000))) {
    c->f32.sor = value;
    return SFX_OK;
  }
  if (key == SFX_TUNE_ADVECT_STAGED && (value == 0 || value == 1)) {
    c->f32.adv_staged = value == 1;
    return SFX_OK;
  }
  if (key == SFX_TUNE_F32_FAST_RESID && value >= 0 && value <= 16) {
    c->f32.fast_resid = value;
    return SFX_OK;
  }
  if (key == SFX_TUNE_TILED_ZCHUNK && (value == 0 || (value >= 4 && value <= 4096))) {
    c->f32.tiled_zchunk = value;
    return SFX_OK;
  }
  if (key == SFX_TUNE_F32_REDIST && (value == 0 || value == 1)) {
    c->f32.redist32 = value == 1;
    return SFX_OK;
  }
  if (key == SFX_TUNE_F32_SOLVER && value >= 0 && value <= 2) {
    c->f32.solver = value;
    c->f32.predicted = 0;
    return SFX_OK;
  }
  return SFX_ERR_ARG;
}

sfx_status sfx_df_pack(const double* in, void* out, size_t n, void* stream) {
  if ((!in || !out) && n) return SFX_ERR_ARG;
  return df_pack(in, out, n, S(stream));
}

sfx_status sfx_df_unpack(const void* in, double* out, size_t n, void* stream) {
  if ((!in || !out) && n) return SFX_ERR_ARG;
  return df_unpack(in, out, n, S(stream));
}

sfx_status sfx_profile(sfx_ctx* c, int on) {
  if (!c) return SFX_ERR_ARG;
  if (on) {
    for (int k = 0; k < K_COUNT; ++k) c->prof.launches[k] = 0;
    c->prof.work[0] = c->prof.work[1] = c->prof.work[2] = 0;
    c->prof.used = 0;
  }
  c->prof.on = on != 0;
  return SFX_OK;
}

sfx_status sfx_profile_work(sfx_ctx* c, int kind, long long* working) {
  if (!c || kind < 0 || kind >= K_COUNT || !working) return SFX_ERR_ARG;
  *working = kind == K_RESID_FAST ? c->prof.work[0]
             : kind == K_RESIDUAL ? c->prof.work[1]
             : kind == K_RESID_INCR ? c->prof.work[2] : -1;
  return SFX_OK;
}

sfx_status sfx_profile_read(sfx_ctx* c, int kind, long long* launches, double* total_ms,
                            long long* timed) {
  if (!c || kind < 0 || kind >= K_COUNT) return SFX_ERR_ARG;
  Prof& P = c->prof;
  if (launches) *launches = P.launches[kind];
  double ms = 0.0;
  long long nt = 0;
  for (size_t q = 0; q < P.used; ++q) {
    if (P.kind[q] != kind) continue;
    SFX_CUDA(cudaEventSynchronize(P.ev[2 * q + 1]));
    float e = 0.f;
    SFX_CUDA(cudaEventElapsedTime(&e, P.ev[2 * q], P.ev[2 * q + 1]));
    ms += e;
    ++nt;
  }
  if (total_ms) *total_ms = ms;
  if (timed) *timed = nt;
  return SFX_OK;
}

}  // extern "C"
