// Private host-side declarations of libsfx: the context and the launchers
// each translation unit provides.
#pragma once

#include <cuda_fp16.h>
#include <cmath>
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "sfx.h"
#include "sfx_common.cuh"

namespace sfx {

// Launch shape of the compensated FP64 totals: blocks of partial sums and
// threads per block.  sfx_totals and sfx_totals_noalloc both use it, so
// they reduce in the same order and return the same bits.
constexpr int kTotalsBlocks = 152 * 4;
constexpr int kTotalsThreads = 256;

// FP32 Newton solves (single-grid and batched) evaluate the residuals in
// FP32 until both relative residuals are below this, or for a set number
// of iterations, then in pair arithmetic.
constexpr float kFastResidSwitch = 1e-3f;

// Over-relaxation factor of the red updates of the FP32 Newton correction
// (relaxation without multigrid) for a field of diffusivity D on a grid of
// nd dimensions: black-then-red sweeps multiply a mode of Jacobi
// eigenvalue mu by 1 - omega (1 - mu^2) per sweep, whose largest value over
// mu^2 in [0, rho^2] is smallest at omega = 2/(2 - rho^2).  rho is bounded
// by a cell's neighbour weights over its diagonal, s/(1 + s) with
// s = dt (2 nd D/h^2 + sum over the faces of |B|/h), and the drift of a
// face is at most D |n_d|/eps (Sec. 2.3, |n| <= 1): the faces add at most
// 2 sqrt(nd) D/eps.  Single-grid and batched solves take it from here, so
// that they agree bit for bit.
inline float sor_omega(double D, double dt, double h, double eps, int nd) {
  const double sd = dt * (2.0 * nd * D / (h * h) + 2.0 * std::sqrt((double)nd) * D / (eps * h));
  const double rho = sd / (1.0 + sd);
  return (float)(2.0 / (2.0 - rho * rho));
}

// Device arrays of one multigrid level.  Level 0 (the fine grid) works on
// the caller's field; its coefficient arrays live here too.
struct LevelData {
  Level lv;
  double* a = nullptr;      // correction (coarse levels only)
  double* b = nullptr;      // right-hand side
  double* lam = nullptr;    // lambda (cell)
  double* B[2][3] = {};     // drift faces for the f (0) and F (1) problems
  double* Bg[3] = {};       // drift faces of a generic sfx_mg_solve call
};

// Kernel kinds counted (and, when profiling is on, timed with CUDA events
// on the launching stream) per context; values match sfx_kernel_kind.
enum Kind {
  K_SMOOTH_FINE = 0, K_SMOOTH_COARSE, K_RESTRICT, K_PROLONG, K_SETUP, K_RESIDUAL, K_ADVECT,
  K_TOTALS, K_FORCES, K_PHASE, K_OTHER, K_SMOOTH_TILED, K_RESID_FAST, K_RESID_INCR, K_COUNT
};

// One coarse level of the FP32 multigrid for the coupled Newton correction
// (plain cell layout; the fine level keeps the colour-packed arrays).
struct Mg32Level {
  float2* e = nullptr;      // correction (e_f, e_F)
  float2* r = nullptr;      // right-hand side of the correction equation
  float2* J = nullptr;      // exchange Jacobian (u, v), volume averages
  float2* B[3] = {};        // drift faces (B_f, B_F), area averages
};

// Coefficients of the correction equation that do not depend on the level.
struct Mg32Coef {
  float Df, DF, inv_dt, kd;
  int literal;
};

// Work arrays of SFX_F32 contexts (float drifts, double-float f*, F*).
struct F32Scratch {
  bool ready = false;
  float* Bf[3] = {};
  float* BF[3] = {};
  float2* B2[3] = {};     // (B_f, B_F) per face (the Newton residual pass)
  __half2* H2[3] = {};    // (B_f, B_F) per face in half precision (correction sweeps)
  float2* fstar = nullptr;
  float2* Fstar = nullptr;
  float* dsig = nullptr;   // sigma - sigma0
  int predicted = 0;       // Picard iterations to run before the first check
  float2* falt = nullptr;  // ping-pong partners of f and F for fused sweeps
  float2* Falt = nullptr;
  bool fused = true;       // one launch per red-black sweep
  int zchunk = 32;         // planes per block of the 3D fused sweep
  int solver = 1;          // 0: nonlinear pair sweeps; 1: coupled Newton
                           // defect correction; 2: Picard defect correction
  float4* rc = nullptr;    // r_f, r_F and the exchange Jacobian's u = c1 F,
                           // v = c1 (f_inf - f), colour-packed
  cudaEvent_t ev[2] = {nullptr, nullptr};
  bool reuse_drift = false;         // keep drift faces while phi and D's are unchanged
  const double* drift_phi = nullptr;
  float* phi32 = nullptr;           // folded float copy of phi
  int* flag = nullptr;              // convergence flag, iteration, prediction kept,
                                    // a tiled sweep that gave up waiting, residual
                                    // kind (0 FP32, else pair), FP32 passes so far
  int fast_resid = 2;               // FP32 residual passes at most per Newton solve
  bool adv_staged = true;           // 3D advection from shared-memory planes
  bool incr_resid = true;           // incremental FP32 residuals after a pair pass (tiled path)
  int sor = 1;                      // relaxation: 0 Gauss-Seidel, 1 over-relaxed red
                                    // updates (omega from the diffusion numbers),
                                    // 1001 .. 1999 omega_F = sor / 1000
  bool predict = true;              // start Newton from x* + last increment
  bool redist32 = false;            // redistance in FP32 (else FP64)
  int sweep_planes = 2;             // 3D correction sweep: planes per thread (1 or 2)
  std::vector<Mg32Level> mg;        // coarse levels of the correction's V-cycle (0 unused)
  const void* mg_faces_of = nullptr;  // drift faces the coarse faces were restricted from
  unsigned long long drift_epoch = 0, mg_epoch = ~0ull;  // rebuilds of the drift faces
  float predict_rho = 1.0f;         // reject a predicted start above this residual
  bool inc_valid = false;
  float* inc_f = nullptr;           // last step's implicit increments x - x*
  float* inc_F = nullptr;
  const void* inc_ptr[3] = {nullptr, nullptr, nullptr};   // f, F, phi of that step
  double inc_key[9] = {};           // dt and parameters of that step
  double drift_key[3] = {0, 0, 0};
  float *ef = nullptr, *eF = nullptr;   // corrections (Picard defect correction)
  float2* e2 = nullptr;                 // Newton corrections (e_f, e_F), colour-packed
  float *rf = nullptr, *rF = nullptr;   // residuals
  float *lf = nullptr, *lF = nullptr;   // diagonals of the linearised problems
  // tiled sweep of the Newton correction (3D, nx a multiple of 4): a second
  // correction buffer (the sweep reads one and writes the other), the
  // minus-side half drifts colour-packed by cell, and the tensor maps of
  // e2, e2b, rc and the three face arrays
  bool tiled = true;                    // use it where eligible (SFX_TUNE_TILED_SWEEP)
  bool tiled_ready = false;
  int tiled_zchunk = 0;                 // planes per block (0: chosen from the grid)
  float2* e2b = nullptr;
  __half2* Hm[3] = {};
  alignas(64) unsigned char tmaps[6][128] = {};
};

// Work arrays of the adjoint and of the Marangoni loss (FP64, either
// context precision), allocated on first use.
struct AdjScratch {
  bool ready = false;
  double* Bf[3] = {};             // drift faces of unit diffusivity, f problem
  double* BF[3] = {};             // and F problem
  double* nf = nullptr;           // adjoint unknowns nu_f, nu_F
  double* nF = nullptr;
  double* sig = nullptr;          // sigma of the loss
  double* force = nullptr;        // ndim x N
  double* dm = nullptr;           // delta_m per cell
  double* G = nullptr;            // dL/d(grad sigma), ndim x N
  double* part = nullptr;         // block partial sums, 5 quantities
  int nblk = 0;
  double* d_out = nullptr;        // 8 reduced values (device) and mirror
  double* h_out = nullptr;
  unsigned long long* d_nrm = nullptr;   // 2 max-norm slots and mirror
  unsigned long long* h_nrm = nullptr;
  float4* K = nullptr;            // FP32 relaxation: inverse 2x2 block per cell
  float* W = nullptr;             // 12 x N neighbour weights (6 per field)
  float2* r = nullptr;            // FP64 residual rounded to float
  float2* e = nullptr;            // correction (e_f, e_F)
  // the relaxation of one defect-correction check (e = 0, the colour
  // sweeps, nu += e) as a CUDA graph: one launch instead of 2 S + 2
  cudaStream_t cap = nullptr;     // private stream the graph is captured on
  cudaGraphExec_t relax = nullptr;
  int relax_sweeps = 0;           // S of the captured graph
};

struct Prof {
  bool on = false;
  long long launches[K_COUNT] = {};
  long long work[3] = {};        // residual passes that did work: FP32, pair, incremental
  std::vector<cudaEvent_t> ev;   // event pairs (start, end)
  std::vector<int> kind;         // kind of each recorded pair
  size_t used = 0;
};

}  // namespace sfx

struct sfx_ctx {
  sfx_grid grid;
  int prec = SFX_F64;
  int sm_count = 152;                // SMs of the context's device (grid sizing)
  std::vector<sfx::LevelData> lev;   // lev[0] = fine
  // fine-level scratch
  double* fstar = nullptr;
  double* Fstar = nullptr;
  double* chi0 = nullptr;
  double* chi_tmp = nullptr;
  double* sigma_tmp = nullptr;
  // reductions
  double* partials = nullptr;        // block partial sums (s, c) pairs
  int n_partial_blocks = 0;
  unsigned long long* d_norms = nullptr;  // 16 slots (device): 0..7 the FP64 solves and the
                                          // FP32 sweeps (7: d_flag), 8..15 the FP32 Newton
                                          // solve's two norm buffers
  unsigned long long* h_norms = nullptr;  // pinned mirror
  double* d_sums = nullptr;          // compensated totals (device)
  double* h_sums = nullptr;          // pinned mirror
  int* d_flag = nullptr;
  std::vector<void*> allocations;
  sfx::Prof prof;
  sfx::F32Scratch f32;
  sfx::AdjScratch adj;
  float* chi32 = nullptr;            // SFX_F32 redistancing: chi0, two iterates
  double* vofH = nullptr;            // VoF: indicator H, face fluxes Q
  double* vofQ = nullptr;
  double* acdi = nullptr;            // ACDI: phi*, r, psi, unit normals
};

namespace sfx {

// cuda error bookkeeping (sfx_api.cu)
sfx_status cuda_fail(cudaError_t e);
#define SFX_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return ::sfx::cuda_fail(e_);  \
  } while (0)
#define SFX_LAUNCH_CHECK() SFX_CUDA(cudaGetLastError())

// instrumentation around each kernel launch (sfx_api.cu)
void prof_before(sfx_ctx* c, int kind, cudaStream_t s);
void prof_after(sfx_ctx* c, int kind, cudaStream_t s);
#define SFX_KERNEL(c, kind, kern, grid, block, s, ...) \
  do {                                                 \
    ::sfx::prof_before(c, kind, s);                    \
    kern<<<grid, block, 0, s>>>(__VA_ARGS__);          \
    ::sfx::prof_after(c, kind, s);                     \
  } while (0)

// sfx_phase.cu
sfx_status phase_field_build(sfx_ctx* c, const double* C, double* chi, void* phi, void* delta,
                             int iters, double dtau, double eps, cudaStream_t s);
// FP32 multigrid of the coupled Newton correction (sfx_mg32.cu).
// mg32_prepare allocates levels 1 .. nlev-1 and restricts the drift faces
// (when they were rebuilt); mg32_cycle takes the fine correction after
// pre-smoothing, restricts its residual, runs the coarse V-cycle and adds
// the prolonged coarse correction to it (fine post-smoothing is the
// caller's).
sfx_status mg32_prepare(sfx_ctx* c, int nlev, cudaStream_t s);
sfx_status mg32_cycle(sfx_ctx* c, const Mg32Coef& k, int nlev, int nu1, int nu2,
                      int coarse_sweeps, const int* done, cudaStream_t s);
sfx_status phase_field_from_chi(sfx_ctx* c, const double* chi, double* phi, double* delta,
                                double eps, cudaStream_t s);
// sfx_advect.cu
sfx_status advect(sfx_ctx* c, const void* ux, const void* uy, const void* uz, double dt,
                  const double* xi, double bc_in, double* out, cudaStream_t s);
sfx_status cfl_umax(sfx_ctx* c, const void* ux, const void* uy, const void* uz, double* umax,
                    cudaStream_t s);
// sfx_solver.cu
sfx_status mg_solve(sfx_ctx* c, double D, const double* Bx, const double* By, const double* Bz,
                    int literal, const double* lam, const double* b, double* a,
                    const sfx_solve_opts* o, int* cycles, double* res, cudaStream_t s);
sfx_status surfactant_step(sfx_ctx* c, const sfx_params* p, const void* phi, const void* ux,
                           const void* uy, const void* uz, double* f, double* F, double dt,
                           const sfx_solve_opts* o, sfx_step_stats* st, cudaStream_t s);
// sfx_solver.cu: drift faces of both problems from a double phi
sfx_status drift_faces64(sfx_ctx* c, const double* phi, double Df, double DF, double eps,
                         double* const* Bf, double* const* BF, cudaStream_t s);
// sfx_acdi.cu
sfx_status acdi_step(sfx_ctx* c, const void* ux, const void* uy, const void* uz, double dt,
                     double zeta, double eps, int clip, double* phi, cudaStream_t s);
// sfx_capillary.cu
sfx_status capillary(sfx_ctx* c, const sfx_params* p, const double* phi, const void* C,
                     const void* sigma, void* kappa, void* force, cudaStream_t s);
// sfx_vof.cu
sfx_status vof_advect(sfx_ctx* c, const void* ux, const void* uy, const void* uz, double dt,
                      int order, double* C, cudaStream_t s);
// sfx_adjoint.cu
sfx_status adj_ensure_scratch(sfx_ctx* c);
sfx_status f_from_gamma(sfx_ctx* c, const double* gamma, const double* phi, double eps,
                        double* f, cudaStream_t s);
sfx_status adjoint_apply(sfx_ctx* c, const sfx_params* p, const double* phi, const double* f,
                         const double* F, double dt, int transpose, const double* vf,
                         const double* vF, double* of, double* oF, cudaStream_t s);
sfx_status adjoint_step(sfx_ctx* c, const sfx_params* p, const double* phi, const double* f,
                        const double* F, double dt, double* lf, double* lF, double* dparams,
                        const sfx_solve_opts* o, sfx_step_stats* st, cudaStream_t s);
// sfx_forces.cu
sfx_status marangoni_loss(sfx_ctx* c, const sfx_params* p, const double* f, const double* phi,
                          const double* C, int dm_mode, double* loss, double* grad,
                          cudaStream_t s);
sfx_status totals(sfx_ctx* c, const double* const* fields, int n, double* out, cudaStream_t s);
sfx_status marangoni(sfx_ctx* c, const sfx_params* p, const double* f, const void* phi,
                     const double* C, int dm_mode, double* sigma, double* force,
                     cudaStream_t s);

// sfx_f32.cu (SFX_F32 contexts: double-float state, FP32 arithmetic)
sfx_status f32_ensure_scratch(sfx_ctx* c);
sfx_status step_f32(sfx_ctx* c, const sfx_params* p, const double* phi, const float* ux,
                    const float* uy, const float* uz, float2* f, float2* F, double dt,
                    const sfx_solve_opts* o, sfx_step_stats* st, cudaStream_t s);
sfx_status advect32(sfx_ctx* c, const float* ux, const float* uy, const float* uz, double dt,
                    const float2* xi, double bc_in, float2* out, cudaStream_t s);
sfx_status totals32(sfx_ctx* c, const void* const* fields, int n, double* out, cudaStream_t s);
sfx_status marangoni32(sfx_ctx* c, const sfx_params* p, const float2* f, const double* phi,
                       const float* C, int dm_mode, float* sigma, float* force, cudaStream_t s);
sfx_status df_pack(const double* in, void* out, size_t n, cudaStream_t s);
sfx_status df_unpack(const void* in, double* out, size_t n, cudaStream_t s);

inline int blocks_for(size_t n, int threads) {
  size_t b = (n + threads - 1) / threads;
  if (b > 152 * 64) b = 152 * 64;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace sfx
