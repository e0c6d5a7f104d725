/*
 * libsfx: GB300 (sm_103a) library for the per-time-step coupled soluble-
 * surfactant update of the hybrid VoF / phase-field method
 * (arxiv 2605.27534) on uniform Cartesian blocks: 2D planar, axisymmetric
 * and 3D.
 *
 * Conventions shared by every call
 * --------------------------------
 * Layout.  Cell arrays hold nx*ny*nz values, x fastest: (k*ny + j)*nx + i.
 *   2D planar and axisymmetric grids have nz = 1; in the axisymmetric case x
 *   is the radius r (axis at r = 0) and y the axial coordinate z.
 *   Face-normal velocities: ux (nz, ny, nx+1), uy (nz, ny+1, nx),
 *   uz (nz+1, ny, nx) (3D only), x fastest.
 * Memory.  Every field pointer is a DEVICE pointer owned by the caller (e.g.
 *   a torch tensor), contiguous, of the element type named in each call.  The
 *   library owns only the opaque context and the scratch inside it (the
 *   multigrid pyramid and work arrays), allocated by sfx_ctx_create and freed
 *   by sfx_ctx_destroy.
 * Streams.  `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Work is enqueued on it in order.  Calls that report statistics
 *   or iterate to a tolerance synchronise with that stream before returning.
 * Errors.  Every call returns an sfx_status; nothing is thrown across the
 *   ABI.  sfx_status_string() names a status.  On SFX_ERR_ARG nothing was
 *   enqueued.  On SFX_ERR_NOT_CONVERGED the fields hold the last iterate and
 *   the stats are filled.  SFX_ERR_CUDA carries the CUDA error that
 *   sfx_last_cuda_error() returns.
 * Precision.  A context is created for SFX_F64 or SFX_F32.
 *   SFX_F64: every field is double.
 *   SFX_F32: the transported state (f, F and the advected xi) is stored as
 *   double-float pairs: two floats per cell, hi then lo, value hi + lo
 *   (about 48 significant bits; sfx_df_pack/sfx_df_unpack convert from/to
 *   double).  Velocities, VoF fraction, sigma and force are float.  The
 *   phase field phi (and delta) is double in both precisions: the unit
 *   normal n = grad phi/|grad phi| is undefined where phi is flat, and deep
 *   in the bulk its direction is set by variations of phi far below float
 *   resolution, so SFX_F32 takes the differences of phi in FP64 (once per
 *   phi) before working on a float copy of phi folded about 1/2 (phi where
 *   phi <= 1/2, phi - 1 elsewhere, so that phi and 1 - phi both keep full
 *   relative precision).  The per-iteration kernels use FP32 arithmetic
 *   only: residuals are formed from pair differences and applied as pair
 *   additions, so the totals keep ~1e-14 relative precision while the FP32
 *   coefficients put the solution within ~1e-7 of the FP64 operator's.
 *   Totals are reduced in FP64 across threads.
 */
#ifndef SFX_H
#define SFX_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SFX_OK = 0,
  SFX_ERR_ARG = 1,            /* null pointer, bad size or option */
  SFX_ERR_NOT_CONVERGED = 2,  /* tolerance not reached in max_cycles */
  SFX_ERR_NONFINITE = 3,      /* NaN or Inf met in a residual */
  SFX_ERR_TIMEOUT = 4,        /* a bounded device-side wait gave up */
  SFX_ERR_CUDA = 5,           /* a CUDA runtime call failed */
  SFX_ERR_WORKSPACE = 6       /* grid larger than the context was made for */
} sfx_status;

typedef enum { SFX_PLANAR2D = 0, SFX_AXISYM = 1, SFX_CART3D = 2 } sfx_geom;
typedef enum { SFX_F64 = 0, SFX_F32 = 1 } sfx_precision;
typedef enum { SFX_EOS_LANGMUIR = 0, SFX_EOS_LINEAR = 1, SFX_EOS_TANH = 2 } sfx_eos;

/* Uniform block (Sec. 3.2; App. A for 3D, App. B for axisymmetric). */
typedef struct {
  int geom;           /* sfx_geom */
  int nx, ny, nz;     /* cells; nz = 1 unless SFX_CART3D */
  double h;           /* cell size, > 0 */
} sfx_grid;

/* Physical parameters of Sec. 2.3-2.6 and App. C. */
typedef struct {
  double ka, kd;      /* adsorption rate r_a, desorption rate r_d, >= 0 */
  double gamma_inf;   /* saturation concentration Gamma_inf, > 0 */
  double Df, DF;      /* interfacial and bulk diffusivity, >= 0 */
  double eps;         /* phase-field width epsilon, > 0 (paper: 0.75 h) */
  double eta;         /* small constant in F/(phi + eta) (Sec. 2.6), >= 0 */
  double sigma0, E;   /* clean surface tension, Gibbs elasticity */
  int eos;            /* sfx_eos */
  int literal_upwind; /* 0: drift upwinded on its transport velocity -B;
                         1: face value as printed in Sec. 3.2 (for study) */
  double bc_F, bc_f;  /* inflow values used by the advection at walls */
} sfx_params;

/* Implicit solve controls (App. C Picard iteration, multigrid V-cycles). */
typedef struct {
  double tol;         /* stop when both relative nonlinear residuals
                         |b - L(a)|_inf / |b|_inf <= tol */
  int max_cycles;     /* cap on Picard iterations (each: nu V-cycles per field) */
  int nu1, nu2;       /* red-black Gauss-Seidel sweeps before / after the
                         coarse-grid correction */
  int mg_levels;      /* levels in the V-cycle (1 = smoother only; 0 = auto:
                         SFX_F64 every level; SFX_F32 relaxation alone when
                         max(Df, DF) dt/h^2 <= 1, else a V-cycle on the
                         Newton correction over the levels whose h <= 3 eps,
                         at least two) */
  int vcycles;        /* V-cycles per field per Picard iteration (>= 1) */
  int check_every;    /* Picard iterations between residual checks (>= 1) */
  int coarse_sweeps;  /* Gauss-Seidel sweeps on the coarsest level */
} sfx_solve_opts;

typedef struct {
  int picard;         /* Picard iterations taken */
  int vcycles;        /* V-cycles taken (both fields) */
  double res_f, res_F;/* final relative nonlinear residuals */
  double mass_f, mass_F; /* sum V f and sum V F after the step (FP64,
                            compensated) */
  int converged;
} sfx_step_stats;

typedef struct sfx_ctx sfx_ctx;

/* Library version and error text. */
const char* sfx_version(void);
const char* sfx_status_string(sfx_status s);
const char* sfx_last_cuda_error(void);

/* Context for one grid shape and precision: allocates the multigrid
   pyramid and work arrays on the current CUDA device (cudaMalloc).
   Returns SFX_ERR_ARG for a bad grid (for SFX_F32 also when a face array
   would reach 2^31 entries: its kernels index with 32-bit integers),
   SFX_ERR_CUDA if allocation fails. */
sfx_status sfx_ctx_create(const sfx_grid* grid, int precision, sfx_ctx** out);
void sfx_ctx_destroy(sfx_ctx* ctx);
/* Fill opts with the defaults used when a call gets opts = NULL. */
void sfx_default_opts(sfx_solve_opts* opts);

/* a1 + a2.  Phase field from the VoF fraction (Sec. 2.5):
   chi0 = 2h(C - 1/2), `iters` Jacobi steps of the Hamilton-Jacobi
   redistancing d chi/d tau + sign(chi0)(|grad chi| - 1) = 0 (first-order
   Godunov with the Russo-Smereka sub-cell fix) at pseudo-time step dtau,
   then phi = (1 - tanh(chi/(2 eps)))/2 and delta = phi (1 - phi)/eps.
   C, chi, phi, delta: double, in both precisions; the iterations are FP64
   unless an SFX_F32 context sets SFX_TUNE_F32_REDIST (FP32 iterate, chi
   within ~1e-7 h of the FP64 one).  delta may be NULL. */
sfx_status sfx_phase_field_build(sfx_ctx* ctx, const double* C, double* chi,
                                 void* phi, void* delta, int iters,
                                 double dtau, double eps, void* stream);

/* a2 alone.  The carrier from a given signed distance (Sec. 2.5):
   phi = (1 - tanh(chi/(2 eps)))/2 and delta = phi (1 - phi)/eps, chi > 0
   inside fluid 1.  For interfaces whose distance is known (an exact
   circle or sphere, or a distance computed elsewhere) instead of a VoF
   fraction.  chi, phi, delta: double cell arrays (device) in both
   precisions; delta may be NULL; no output may alias chi.  SFX_ERR_ARG on a
   null chi or phi, an output aliasing chi, or eps <= 0. */
sfx_status sfx_phase_field_from_chi(sfx_ctx* ctx, const double* chi, double* phi,
                                    double* delta, double eps, void* stream);

/* a3.  Explicit BCG advection xi* = xi - dt div(u xi) (Sec. 3.1) of one
   state field (double, or double-float pairs in SFX_F32 contexts) with face
   velocities u (context precision); bc_in is the value carried in through
   inflow walls.  xi_out must not alias xi. */
sfx_status sfx_advect(sfx_ctx* ctx, const void* ux, const void* uy,
                      const void* uz, double dt, const void* xi,
                      double bc_in, void* xi_out, void* stream);

/* a5.  Solve the generalised elliptic problem of Sec. 3.1
   div(alpha grad a + beta a) + lambda a = b with alpha = -D and beta = -B
   (B given on faces: Bx (nz,ny,nx+1), By (nz,ny+1,nx), Bz (nz+1,ny,nx) or
   NULL in 2D; wall faces are ignored) by multigrid V-cycles until
   |b - L(a)|_inf <= tol |b|_inf.  All arrays double (SFX_F64 contexts).
   a holds the initial guess and receives the solution. */
sfx_status sfx_mg_solve(sfx_ctx* ctx, double D, const double* Bx,
                        const double* By, const double* Bz, int literal_upwind,
                        const double* lambda, const double* b, double* a,
                        const sfx_solve_opts* opts, int* cycles_out,
                        double* res_out, void* stream);

/* a3'.  Geometric VoF advection of the volume fraction C (Sec. 2 tracks
   the interface with a geometric VoF method; the scheme is read as
   directionally split conservative PLIC advection): for each direction in
   turn (order 0: x, y, z; 1: reversed, alternate between steps), with face
   Courant numbers c_f = u_f dt/h,
     C <- C - (Q_+ - Q_-) + H (c_+ - c_-),
   Q_f the fluid of the upwind cell's PLIC reconstruction (Youngs normal)
   within |c_f| h of the face and H = [C > 1/2] at the start of the step.
   Conserves sum C exactly for divergence-free velocities; bounded for
   |c_f| <= 1/2.  Walls carry no flux.  C: double, in place; velocities in
   the context precision; SFX_F32 contexts evaluate the PLIC geometry of the
   fluxes in FP32 (fluxes to ~1e-7, C still conserved exactly).  Planar 2D and 3D (SFX_ERR_ARG for axisymmetric
   grids).  The context allocates two scratch arrays on first use. */
sfx_status sfx_vof_advect(sfx_ctx* ctx, const void* ux, const void* uy, const void* uz,
                          double dt, int order, double* C, void* stream);

/* a2 + a3 + a4 + a5 + a6.  One coupled surfactant step (Sec. 3.1 splitting;
   App. C source): explicit BCG advection of f and F when ux != NULL, then
   the fully implicit f/F system of App. C solved by Picard iteration, each
   half a multigrid solve of the Sec. 3.1 operator with the drifts
   B_f = -Df 2(0.5 - phi)/eps n and B_F = -DF (1 - phi)/eps n,
   n = grad phi/|grad phi| by centred differences, faded out where phi is
   flat: with q = |grad phi| / (phi (1 - phi)/eps), the ratio to the slope
   of the equilibrium tanh profile, n is scaled by clamp(q/1e-3 - 1, 0, 1)
   (0 for q <= 1e-3, the unit vector for q >= 2e-3), and n = 0 where
   |grad phi| < 1e-30.  f and F
   (state layout of the context) are updated in place; phi is double, the
   velocities are in the context precision.  SFX_F32 contexts solve the
   same system by coupled Newton defect correction (SFX_TUNE_F32_SOLVER):
   each iteration evaluates both residuals in pair arithmetic and relaxes
   the correction by nu1 + nu2 FP32 red-black sweeps with a 2x2 block solve
   per cell, or, when diffusion dominates (opts->mg_levels), by an FP32
   V-cycle: nu1 fine sweeps, the coarse levels (the same block smoother on
   re-discretised operators), nu2 fine sweeps.  stats may be NULL. */
sfx_status sfx_surfactant_step(sfx_ctx* ctx, const sfx_params* params,
                               const void* phi, const void* ux,
                               const void* uy, const void* uz, void* f,
                               void* F, double dt,
                               const sfx_solve_opts* opts,
                               sfx_step_stats* stats, void* stream);

/* a6.  Compensated totals sum V x of `n_fields` <= 8 state fields (double,
   or double-float pairs in SFX_F32 contexts; `fields` is a host array of
   device pointers) into out[i] (host memory).  Volumes: h^2 (planar), h^3
   (3D), pi (r+^2 - r-^2) h (axisymmetric).  Deterministic: fixed reduction
   order. */
sfx_status sfx_totals(sfx_ctx* ctx, const void* const* fields, int n_fields,
                      double* out, void* stream);

/* Largest n_fields that sfx_totals_noalloc accepts. */
#define SFX_NOALLOC_MAX_FIELDS 8

/* The totals of sfx_totals (same launch shape and reduction order, so the
   same bits) without a context and without allocating.  For callers that may not allocate device
   memory: programs whose device memory belongs to another allocator, and
   code that must avoid the device-wide synchronisation of cudaMalloc and
   cudaFree.  The paper has no counterpart; this is a service of the
   library.
   Scratch: a fixed file-scope device array of 2 x SFX_NOALLOC_MAX_FIELDS x
   608 + SFX_NOALLOC_MAX_FIELDS doubles (about 78 KB) that every GPU which
   loads the library keeps until the process exits.  The first call on a
   device looks up the array's device address (cudaGetSymbolAddress) with
   that device current; make that first call before any stream capture.
   Every call shares the array and leaves its contents behind; each call
   writes every slot before reading it.  Calls whose GPU work overlaps (for
   instance on two unordered streams) race on the array.
   grid: host pointer, as for sfx_ctx_create.  fields: host array of
   n_fields device pointers to double cell arrays.  out: host array of
   n_fields doubles, written after the call synchronises with `stream`.
   Returns SFX_ERR_WORKSPACE when n_fields > SFX_NOALLOC_MAX_FIELDS,
   SFX_ERR_ARG for a bad grid or null pointer, SFX_ERR_CUDA on a CUDA
   failure.  Calls no cudaMalloc, cudaFree or allocating library routine. */
sfx_status sfx_totals_noalloc(const sfx_grid* grid, const double* const* fields,
                              int n_fields, double* out, void* stream);

/* a7 + a8.  EOS and Marangoni force (Sec. 2.3-2.4):
   Gamma = f/delta_phi where delta_phi >= 1e-3/eps (else 0); sigma(Gamma)
   by params->eos, evaluated in double; force = delta_m (I - n n) grad sigma
   with centred grad sigma, n from phi, and delta_m the PLIC interface area
   per cell volume (dm_mode 1; Youngs normal) or |grad C| (dm_mode 0).
   phi is double.  SFX_F64: f, C, sigma, force double.  SFX_F32: f
   double-float pairs, C, sigma, force float (sigma may be NULL); the
   Langmuir logarithm is
   taken in double once Gamma/Gamma_inf > 1/2, and the gradient is taken of
   sigma - sigma0.  force holds ndim arrays of N cells, component-major. */
sfx_status sfx_marangoni_force(sfx_ctx* ctx, const sfx_params* params,
                               const void* f, const void* phi,
                               const void* C, int dm_mode, void* sigma,
                               void* force, void* stream);

/* One step of the ACDI phase-field equation (Sec. 2.5):
     d phi/dt + div(u phi) = div(zeta {eps grad phi
                               - 1/4 (1 - tanh^2(psi/(2 eps))) grad psi/|grad psi|}),
     psi = eps ln((phi + 1e-6)/(1 - phi + 1e-6)).
   The advective part is the BCG step of sfx_advect (skipped when ux is
   NULL; inflow faces carry phi = 1); the regularisation is explicit, in
   flux form, with central face fluxes: eps (phi_R - phi_L)/h, and the mean
   of the two cells' unit normals of psi (centred differences; 0 where
   |grad psi| < 0.1, i.e. where phi saturates and psi is flat to round-off)
   times 1 - tanh^2 of the face mean of psi/(2 eps).  Wall faces carry no
   flux.
   The paper takes zeta = 1.1 max|u| and eps = 0.75 h.  With veps the
   scheme's phi saturates towards -veps and 1 + veps and overshoots [0, 1]
   by O(veps) there; psi is formed from phi clipped to [0, 1].  clip = 1
   clips the result to [0, 1] (what the surfactant step needs: it divides
   by phi + eta); clip = 0 keeps the overshoots and conserves sum V phi
   exactly.  phi: double, in place, in both precisions; ux, uy, uz: face velocities in the context
   precision (uz NULL in 2D).  Stable for zeta eps dt/h^2 <= 1/(2 ndim) and
   the BCG Courant limit.  The context allocates (3 + ndim) N doubles of
   scratch on first use.  SFX_ERR_ARG on a null phi, dt <= 0, eps <= 0 or
   zeta < 0. */
sfx_status sfx_acdi_step(sfx_ctx* ctx, const void* ux, const void* uy,
                         const void* uz, double dt, double zeta, double eps,
                         int clip, double* phi, void* stream);

/* Capillary force (Sec. 2.4, curvature of Sec. 2.2):
     F_cap = sigma kappa delta_s n,  kappa = -div n,  delta_s = |grad C|,
   n = grad phi/|grad phi| at cell centres (centred differences, 0 where
   phi is flat), div n in flux form over the cell's faces with each face
   taking the mean of its two cells' normal components (the axisymmetric
   face areas add the hoop term n_r/r), no normal component on wall faces,
   zero area on the axis; grad C centred with zero-gradient ghosts.  sigma
   is any cell field, normally the EOS output of sfx_marangoni_force.
   params: only eps is used.  phi is double.  SFX_F64: C, sigma, kappa,
   force double, FP64 arithmetic.  SFX_F32: C, sigma, kappa, force float;
   the differences of phi are taken in FP64 and the rest in FP32 (kappa is
   a difference of unit vectors over h, so its rounding grows as 2^-24/h).
   kappa (may be NULL) receives the curvature; force holds ndim arrays of N
   cells, component-major.  Caller-owned device arrays; SFX_ERR_ARG on a
   null argument. */
sfx_status sfx_capillary_force(sfx_ctx* ctx, const sfx_params* params,
                               const double* phi, const void* C,
                               const void* sigma, void* kappa, void* force,
                               void* stream);

/* a9.  Time step of Sec. 3.3: safety * min(h/(umax + D/eps),
   h^2/(2 N_d D)), with umax the largest |face velocity| (reduced on the
   device from ux, uy, uz in the context precision).  Host result. */
sfx_status sfx_cfl_dt(sfx_ctx* ctx, const void* ux, const void* uy,
                      const void* uz, double D, double eps, double safety,
                      double* dt_out, void* stream);

/* Tuning knobs (same results, different schedules).  Returns SFX_ERR_ARG
   for an unknown key or value. */
typedef enum {
  SFX_TUNE_FUSED_SWEEP = 0, /* SFX_F32, solver 0: 1 (default) = one launch
                               per red-black sweep through shared-memory
                               tiles; 0 = one launch per colour.  Bitwise
                               equal. */
  SFX_TUNE_F32_SOLVER = 1,  /* SFX_F32: 1 (default) = coupled Newton defect
                               correction: one pair-arithmetic pass
                               evaluates both residuals and the pointwise
                               2x2 exchange Jacobian, then nu1 + nu2 FP32
                               red-black sweeps with a 2x2 solve per cell
                               relax the correction; 2 = the same with the
                               fields linearised alternately (Picard);
                               0 = nonlinear red-black sweeps on the pair
                               state.  Same fixed point, same test. */
  SFX_TUNE_REUSE_DRIFT = 2, /* SFX_F32: 1 = keep the drift faces and the
                               folded float copy of phi of the last step
                               while phi's pointer, Df, DF and eps are
                               unchanged (for a static interface; after
                               writing phi in place, set the knob again to
                               force a rebuild); 0 (default) = rebuild them
                               every step. */
  SFX_TUNE_F32_REDIST = 4,  /* SFX_F32: 1 = iterate the redistancing of
                               sfx_phase_field_build in FP32 (2D: eight
                               Jacobi steps per launch in shared memory);
                               chi within ~1e-7 h of the FP64 iterate, but
                               where |grad chi| is small (the front of the
                               redistanced band) the direction of grad phi,
                               and with it the drift, follows chi's float
                               rounding: with F = 1 inside a 256^3 sphere
                               the step then moves by 5e-5.  0 (default) =
                               FP64 redistancing as in SFX_F64 contexts. */
  SFX_TUNE_SWEEP_PLANES = 5, /* SFX_F32, 3D: z-planes each thread of the
                               Newton correction's colour launches updates,
                               1 or 2 (default: two independent cells'
                               loads in flight per thread; 5 % faster at
                               256^3).  With tiled sweeps the one colour
                               launch left, which adds the corrections to
                               the state, always takes one (8 % faster).
                               Bitwise equal. */
  SFX_TUNE_TILED_SWEEP = 6, /* SFX_F32 Newton solver, 3D grids with nx a
                               multiple of 4, relaxation without the V-cycle
                               (mg_levels < 2): 1 (default) = sweeps 1 .. S-1
                               of an iteration as one launch each (black,
                               then red), marching through z-planes staged in
                               shared memory by tensor copies, the last black
                               colour as a colour launch; 0 = one launch per
                               colour.  Bitwise equal.  A staging wait that
                               gives up (after 1 s) ends the step with
                               SFX_ERR_TIMEOUT. */
  SFX_TUNE_TILED_ZCHUNK = 7, /* z-planes per block of the tiled sweep, 4 ..
                               4096, or 0 (default): chosen from the grid
                               and the SM count to fill the last wave of
                               blocks (37 at 256^3 on 152 SMs). */
  SFX_TUNE_F32_INCR_RESID = 10, /* SFX_F32 Newton solver on the tiled path:
                               1 (default) = after a pair residual pass
                               whose relative residuals are below 1e5 tol,
                               the residuals of the next iterates are formed
                               in FP32 from the previous ones and the
                               correction just added (linear terms and a
                               product of the correction, rounded to ~1e-6
                               of the pair residual, so the chain stays
                               below a tenth of the tolerance; the relative
                               test keeps the scales |b| of the pair pass,
                               since the chain reads neither the state nor
                               x*); 0 = a pair
                               pass at every iteration after the FP32
                               ones. */
  SFX_TUNE_F32_SOR = 11,    /* SFX_F32 Newton solver, relaxation without
                               multigrid (also a batch's, through
                               sfx_batch_set_tuning): 1 (default) = every
                               red update after the first is over-relaxed,
                               e <- e + omega (e_GS - e), per field with
                               omega = 2/(2 - rho^2), rho = s/(1 + s),
                               s = dt (2 d D/h^2 + 2 sqrt(d) D/(eps h)) on
                               a d-dimensional grid (a row-sum bound on the
                               Jacobi radius with the drift bounded by
                               D/eps per face; the minimax factor of
                               black-then-red sweeps is rho^2/(2 - rho^2)
                               per sweep instead of rho^2); 1001 .. 1999 =
                               omega of F set to value/1000 (f as for 1);
                               0 = Gauss-Seidel.  The converged state is
                               the same fixed point. */
  SFX_TUNE_ADVECT_STAGED = 9, /* SFX_F32, 3D: 1 (default) = the BCG step of
                               f and F from z-planes staged in shared
                               memory (values rounded once, neighbours past
                               a wall clamped in the staging); 0 = the
                               tiles that gather from global memory.
                               Bitwise equal. */
  SFX_TUNE_F32_FAST_RESID = 8, /* SFX_F32 Newton solver: at most this many
                               iterations per solve (0 .. 16, default 2)
                               evaluate the residuals in FP32 instead of
                               pair arithmetic (about 1e-7 of the scale
                               instead of 1e-14), switching to the pair
                               pass once both relative residuals are below
                               1e-3; only a pair residual can pass the
                               tolerance test, so the converged state is
                               the same fixed point; 0 = pair residuals
                               only. */
  SFX_TUNE_PREDICT = 3      /* SFX_F32 Newton solver: 1 (default) = start
                               the iteration from x* plus the previous
                               step's implicit increment x - x* when the
                               step continues the same problem (same f, F
                               and phi buffers, dt and parameters; the last
                               step converged), restarting from x* when
                               the predicted start's relative residuals
                               exceed 1; 0 = start from x*.  Same fixed
                               point and test; the iterate differs within
                               the tolerance. */
} sfx_tune_key;
sfx_status sfx_set_tuning(sfx_ctx* ctx, int key, int value);

/* Conversions between double arrays and the double-float pairs of SFX_F32
   contexts (n cells; device pointers; enqueued on stream). */
sfx_status sfx_df_pack(const double* in, void* out, size_t n, void* stream);
sfx_status sfx_df_unpack(const void* in, double* out, size_t n, void* stream);

/* a10.  Discrete adjoint of the no-flow coupled step (App. C), FP64 in
   either context precision; every array below is double.  A step solves
   R(x1; x0, theta) = 0 for x1 = (f, F) with the App. C residuals
     R_f = (f^n - f)/dt + N_f f + q,  R_F = (F^n - F)/dt + N_F F - q,
     q = k_a F (f_inf - f)/(phi + eta) - k_d f,
   N the Sec. 3.1-3.2 flux divergence of each field.  With J = dR/dx1 at the
   state after the step, a loss gradient lam1 = dL/dx1 pulls back as
     (-J)^T nu = lam1,  dL/dx0 = nu/dt,  dL/dtheta += (dR/dtheta)^T nu,
   theta = (k_a, k_d, D_f, D_F) (Sec. 2.3 / App. C parameters).  The paper
   has no adjoint: this is the exact derivative of its discrete step. */

/* f = Gamma delta_phi, delta_phi = phi (1 - phi)/eps (Sec. 2.3).  The map
   is diagonal, so the same call takes dL/df to dL/dGamma. */
sfx_status sfx_f_from_gamma(sfx_ctx* ctx, const double* gamma, const double* phi, double eps,
                            double* f, void* stream);
/* L = sum_c V_c |F_Ma,c|^2 of the sfx_marangoni_force field (FP64), and,
   when dloss_df != NULL, dL/df per cell.  Waits for stream. */
sfx_status sfx_marangoni_loss(sfx_ctx* ctx, const sfx_params* params, const double* f,
                              const double* phi, const double* C, int dm_mode, double* loss,
                              double* dloss_df, void* stream);
/* out = (-J) v, or (-J)^T v when transpose != 0, at the state (f, F) after
   a step of size dt (for checks of the adjoint).  Outputs must not alias
   inputs. */
sfx_status sfx_adjoint_apply(sfx_ctx* ctx, const sfx_params* params, const double* phi,
                             const double* f, const double* F, double dt, int transpose,
                             const double* vf, const double* vF, double* out_f, double* out_F,
                             void* stream);
/* One adjoint step.  f, F: the state after the forward step; lam_f, lam_F:
   in dL/d(f, F) after the step, out dL/d(f, F) before it (in place);
   dparams (host, 4 doubles, may be NULL): the step's dL/d(k_a, k_d, D_f,
   D_F) is added.  The transposed system is solved by defect correction:
   each check evaluates the FP64 residual r = lam1 - (-J)^T nu, and until
   max|r| <= tol max|lam1| the correction of (-J)^T e = r is relaxed by
   nu1 + nu2 FP32 red-black Gauss-Seidel sweeps (2x2 solve per cell, on
   coefficients computed once per step from the FP64 operator) and added to
   nu; after max_cycles checks SFX_ERR_NOT_CONVERGED (outputs written).
   stats (may be NULL): picard = checks, vcycles = sweeps, res_f = res_F =
   the final relative residual.  The relaxation of a check runs as one CUDA
   graph launch, captured on the context's first call (and again when
   nu1 + nu2 changes) on a stream the context owns.  Waits for stream. */
sfx_status sfx_adjoint_step(sfx_ctx* ctx, const sfx_params* params, const double* phi,
                            const double* f, const double* F, double dt, double* lam_f,
                            double* lam_F, double* dparams, const sfx_solve_opts* opts,
                            sfx_step_stats* stats, void* stream);

/* Batched SFX_F32 step over many independent axisymmetric blocks
   (Sec. 4.3 runs series of drop cases with different Bi and Da; each one is
   a small (r, z) block).  Every instance has its own size, h, dt and
   parameters; all their fields are packed back to back in shared arrays:
   instance i's cells start at cell_off[i] (its own layout is the
   axisymmetric one above: nx = nr, ny = nz), its radial faces at
   rface_off[i] ((nz, nr+1) each) and its axial faces at zface_off[i]
   ((nz+1, nr) each); sfx_batch_layout returns the offsets.  Each step does,
   per instance, what sfx_surfactant_step does in an SFX_F32 context with
   the coupled Newton solver: drift faces (Sec. 2.3), BCG advection
   (Sec. 3.1) when velocities are given, then App. C's coupled implicit
   system solved by Newton defect correction until both relative residuals
   are <= tol.  An instance that meets the tolerance stops iterating at once
   while the others go on.  The whole step is one CUDA graph launch, captured
   on the first call and again when a pointer, tol or the schedule changes;
   it never synchronises with the host.  The library owns the batch (the
   descriptors, the scratch and the graph). */
typedef struct {
  int nr, nz;           /* cells in r and z, >= 1 */
  double h, dt;         /* cell size and time step, > 0 */
  sfx_params params;    /* as for sfx_surfactant_step (sigma0, E, eos unused) */
} sfx_batch_instance;
typedef struct sfx_batch sfx_batch;

/* Copies the n >= 1 descriptors; SFX_ERR_ARG on a bad size or parameter. */
sfx_status sfx_batch_create(const sfx_batch_instance* inst, int n, sfx_batch** out);
/* The same with the geometry of every instance: SFX_AXISYM (as
   sfx_batch_create; nr x nz rings) or SFX_PLANAR2D (nr x nz planar cells of
   unit depth, e.g. the flat-interface columns of Sec. 4.3); totals are then
   sum h^2 x.  SFX_ERR_ARG for another geometry. */
sfx_status sfx_batch_create_geom(const sfx_batch_instance* inst, int n, int geom,
                                 sfx_batch** out);
void sfx_batch_destroy(sfx_batch* b);
/* Totals of the packed arrays and, when the array pointers are not NULL,
   the n offsets of each instance (host arrays of n size_t). */
sfx_status sfx_batch_layout(const sfx_batch* b, size_t* n_cells, size_t* n_rfaces,
                            size_t* n_zfaces, size_t* cell_off, size_t* rface_off,
                            size_t* zface_off);
/* Schedule: threads per block (128, 256 or 512), red-black sweeps per
   Newton iteration (1..16) and the iteration budget (1..200).  Defaults
   256, 3, 8.  An instance that has not converged within the budget keeps
   its last iterate and is reported by sfx_batch_stats. */
sfx_status sfx_batch_set_schedule(sfx_batch* b, int block, int sweeps, int max_iters);
/* Solver tuning of a batch, keys and values as sfx_set_tuning:
   SFX_TUNE_F32_FAST_RESID (0 .. 16, default 2; each instance counts its
   own FP32 residual passes and switches to pair residuals on its own, the
   rule of the single-grid solve) and SFX_TUNE_F32_SOR (default 1; omega
   per instance from its parameters, as a single-grid context computes it).
   SFX_ERR_ARG for another key or a value out of range. */
sfx_status sfx_batch_set_tuning(sfx_batch* b, int key, int value);
/* One step of every instance.  phi: phase field (double, packed cells);
   ur, uz: face velocities (float, packed radial / axial faces), both NULL
   for no advection; f, F: double-float pairs (packed cells), updated in
   place.  Enqueued on stream; returns without waiting. */
sfx_status sfx_batch_step(sfx_batch* b, const void* phi, const void* ur, const void* uz,
                          void* f, void* F, double tol, void* stream);
/* on != 0: phi is static (a fixed interface).  Its folded copy and the
   drift faces are then built once, outside the step graph, on the next
   step and whenever the phi pointer changes; after writing phi in place,
   call again to force a rebuild.  on = 0 (default): every step rebuilds
   them inside the graph. */
sfx_status sfx_batch_reuse_phi(sfx_batch* b, int on);
/* Per-instance results of the last step (host arrays of n, any may be
   NULL): Newton iterations, final relative residuals, compensated totals
   sum V f and sum V F (FP64) and whether the tolerance was met.  Waits for
   stream. */
sfx_status sfx_batch_stats(sfx_batch* b, int* iters, float* res_f, float* res_F,
                           double* mass_f, double* mass_F, int* converged, void* stream);
/* Work counters per instance (host arrays of n, may be NULL): residual
   passes and correction sweep groups (sweeps x 2 colours) run since the
   batch was created or last reset (reset != 0 zeroes them after reading).
   Waits for stream. */
sfx_status sfx_batch_work(sfx_batch* b, long long* resid_passes, long long* sweep_groups,
                          int reset, void* stream);
/* Autotuner: runs one step of every candidate schedule (tiles of 128, 256
   or 512 packed cells per block, 2, 3 or 4 sweeps) on scratch copies of f
   and F (which stay unchanged),
   gives each the smallest iteration budget under which every instance
   converged (plus one spare), times it and keeps the fastest schedule.
   Since a step's iterations end on the device once every instance has
   converged, the budget kept is only a cap: twice the probed one, at least
   16 (at most 200; 200 when no candidate converged every instance within
   40 iterations).  chosen (3 ints, may be NULL) receives block, sweeps and
   budget.  Allocates the two scratch copies (cudaMalloc) and releases
   them, and its events, on every return; on an error the previous schedule
   is restored.  Waits for stream. */
sfx_status sfx_batch_autotune(sfx_batch* b, const void* phi, const void* ur, const void* uz,
                              const void* f, const void* F, double tol, void* stream,
                              int* chosen);

/* Instrumentation (not part of the method).  Kernel kinds: */
typedef enum {
  SFX_K_SMOOTH_FINE = 0,  /* red-black Gauss-Seidel colour sweep, fine level */
  SFX_K_SMOOTH_COARSE,    /* colour sweeps and the coarsest-level solve */
  SFX_K_RESTRICT,         /* residual restriction */
  SFX_K_PROLONG,          /* prolongation and correction */
  SFX_K_SETUP,            /* App. C coefficients, drift faces, restrictions */
  SFX_K_RESIDUAL,         /* residual norms (convergence checks) */
  SFX_K_ADVECT,           /* BCG advection */
  SFX_K_TOTALS,           /* compensated totals */
  SFX_K_FORCES,           /* EOS and Marangoni force */
  SFX_K_PHASE,            /* redistancing and phase field */
  SFX_K_OTHER,
  SFX_K_SMOOTH_TILED,     /* tiled red-black sweep (both colours), fine level */
  SFX_K_RESID_FAST,       /* FP32 residual passes of the FP32 Newton solve */
  SFX_K_RESID_INCR,       /* incremental FP32 residual passes of that solve */
  SFX_K_COUNT
} sfx_kernel_kind;

/* on != 0: reset the per-kind launch counters and start bracketing every
   kernel launch of this context with CUDA events recorded on the launching
   stream (at most 8192 launches are timed per run); on = 0: stop. */
sfx_status sfx_profile(sfx_ctx* ctx, int on);
/* Launches of `kind` since the last sfx_profile(ctx, 1), the summed
   event-timed duration in ms and how many launches were timed.  Waits for
   the recorded events.  Any output pointer may be NULL. */
sfx_status sfx_profile_read(sfx_ctx* ctx, int kind, long long* launches,
                            double* total_ms, long long* timed);
/* Of the launches of `kind` since the last sfx_profile(ctx, 1), those that
   did work, where the library can tell: the residual passes of the FP32
   Newton solve (SFX_K_RESIDUAL, SFX_K_RESID_FAST, SFX_K_RESID_INCR), of
   which each iteration launches every kind and all but one return at once,
   counted from the residual
   kind recorded with the iteration's norms (iterations whose norms the
   solve read); -1 for the other kinds.  SFX_ERR_ARG on a bad kind. */
sfx_status sfx_profile_work(sfx_ctx* ctx, int kind, long long* working);

#ifdef __cplusplus
}
#endif
#endif /* SFX_H */
