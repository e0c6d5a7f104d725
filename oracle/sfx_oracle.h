/*
 * FP64 CPU oracle for the coupled soluble-surfactant step of the hybrid
 * VoF / phase-field method (arxiv 2605.27534).
 *
 * TEST INFRASTRUCTURE ONLY.  This oracle exists to check the CUDA library
 * against the paper.  It is plain, serial, double-precision C that follows
 * the paper's equations in the paper's order.  Only the tests, the smoke
 * check and the CPU-baseline leg of the benchmark may load it; the product
 * path never calls it.  It shares no code, header, table or constant with
 * the CUDA library.
 *
 * Layout: cell-centred arrays, x fastest: index (k*ny + j)*nx + i.
 *   2D planar: nz = 1, x/y.  Axisymmetric: nz = 1, x = r (axis at x = 0),
 *   y = z (axial).  3D: x/y/z.
 * Face-normal velocities: ux[nz][ny][nx+1], uy[nz][ny+1][nx],
 *   uz[nz+1][ny][nx] (3D only).
 *
 * Parity-unpinned functions (no closed form or independent check fixes
 * them; they are checked only against convergence under refinement):
 *   orc_marangoni with dm_mode = 1 in 3D (plane-cube area).
 */
#ifndef SFX_ORACLE_H
#define SFX_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_PLANAR = 0, ORC_AXI = 1, ORC_3D = 2 };
enum { ORC_EOS_LANGMUIR = 0, ORC_EOS_LINEAR = 1, ORC_EOS_TANH = 2 };

typedef struct {
  int geom;           /* ORC_PLANAR, ORC_AXI, ORC_3D */
  int nx, ny, nz;     /* nz = 1 unless 3D */
  double h;           /* uniform cell size */
} orc_grid;

typedef struct {
  double ka, kd;      /* adsorption rate r_a, desorption rate r_d (Sec. 2.6) */
  double gamma_inf;   /* saturation concentration Gamma_inf */
  double Df, DF;      /* interfacial and bulk diffusivities */
  double eps;         /* phase-field width epsilon (Sec. 2.5) */
  double eta;         /* small constant added to phi in F/phi (Sec. 2.6) */
  double sigma0, E;   /* EOS: clean tension and Gibbs elasticity (Sec. 2.3) */
  int eos;            /* ORC_EOS_* */
  int literal_upwind; /* 1: face value taken as printed in Sec. 3.2 (left if
                         B > 0); 0: upwind for the transport velocity -B */
  double bc_F, bc_f;  /* inflow (Dirichlet) values for advection */
} orc_params;

typedef struct {
  double tol;         /* Picard stop: relative nonlinear residual */
  int max_picard;
  int max_sweeps;     /* Gauss-Seidel sweep cap per linear solve */
} orc_opts;

typedef struct {
  int picard;         /* Picard iterations taken */
  int sweeps;         /* total Gauss-Seidel sweeps */
  double res_f, res_F;/* final relative nonlinear residuals */
  double mass_f, mass_F; /* sum V f, sum V F after the step */
  int converged;
} orc_stats;

/* threads of the build: omp_get_max_threads() in the OpenMP build, else 1 */
int orc_threads(void);

/* cell volume and face areas (Sec. 3.2, App. A, App. B) */
double orc_cell_volume(const orc_grid* g, int i, int j, int k);

/* a1: signed distance from the VoF fraction by Hamilton-Jacobi iterations
   (Sec. 2.5).  chi0 = 2h(C - 1/2); iters Jacobi steps with pseudo-time dtau. */
void orc_redistance(const orc_grid* g, const double* C, int iters, double dtau,
                    double* chi);
/* a2: phi = (1 - tanh(chi / 2 eps)) / 2 and delta = phi (1 - phi) / eps */
void orc_phase_field(const orc_grid* g, const double* chi, double eps,
                     double* phi, double* delta);
/* a1 + a2 together, as the library call does */
void orc_phase_field_build(const orc_grid* g, const double* C, int iters,
                           double dtau, double eps, double* chi, double* phi,
                           double* delta);

/* unit normal n = grad(phi)/|grad(phi)| at cell centres, centred
   differences, zero-gradient walls; n = 0 where |grad phi| < 1e-30.
   n has 2 (or 3) arrays of N values: n[d*N + c].  Where phi is flat the
   normal fades out: n is scaled by min(max(q/ORC_NORMAL_KAPPA - 1, 0), 1),
   q = |grad phi| / (phi (1 - phi)/eps). */
#define ORC_NORMAL_KAPPA 1e-3
void orc_normals(const orc_grid* g, const double* phi, double eps, double* n);

/* anti-diffusive face drift B at every face of the grid (Sec. 2.6, App. C):
   which = 0 -> B_f = -Df * 2(0.5 - phi)/eps n ; which = 1 -> B_F = -DF (1 - phi)/eps n,
   face value = mean of the two cell values (Sec. 3.2).  Walls get 0. */
void orc_face_drift(const orc_grid* g, const orc_params* p, const double* phi,
                    int which, double* Bx, double* By, double* Bz);

/* a5: generic operator L(a) = div(alpha grad a + beta a) + lambda a with
   alpha = -D, beta = -B (Sec. 3.1); writes L(a) per cell. */
void orc_apply_operator(const orc_grid* g, double D, const double* Bx,
                        const double* By, const double* Bz, int literal_upwind,
                        const double* lambda, const double* a, double* out);
/* a5: solve L(a) = b by Gauss-Seidel to relative residual tol; returns the
   sweep count (negative if the cap was hit). */
int orc_elliptic_solve(const orc_grid* g, double D, const double* Bx,
                       const double* By, const double* Bz, int literal_upwind,
                       const double* lambda, const double* b, double* a,
                       double tol, int max_sweeps, double* rel_res);

/* a3: explicit BCG advection xi* = xi - dt div(u xi) (Sec. 3.1). */
void orc_advect_bcg(const orc_grid* g, const double* ux, const double* uy,
                    const double* uz, double dt, const double* xi,
                    double bc_in, double* xi_star);

/* a3': one step of directionally split conservative PLIC advection of the
   volume fraction C (in place), direction order 0 (x, y, z) or 1
   (reversed); planar 2D and 3D grids. */
void orc_vof_advect(const orc_grid* g, const double* ux, const double* uy,
                    const double* uz, double dt, int order, double* C);

/* a4: coupled implicit source step of App. C for (f, F), Picard on the
   two elliptic problems.  fstar/Fstar are the post-advection fields; f and F
   are overwritten with the new state. */
void orc_coupled_implicit(const orc_grid* g, const orc_params* p,
                          const double* phi, const double* fstar,
                          const double* Fstar, double dt, const orc_opts* o,
                          double* f, double* F, orc_stats* st);

/* the whole step: a3 (if ux != NULL) then a4, then a6 totals. */
void orc_surfactant_step(const orc_grid* g, const orc_params* p,
                         const double* phi, const double* ux, const double* uy,
                         const double* uz, double dt, const orc_opts* o,
                         double* f, double* F, orc_stats* st);

/* nonlinear residuals of App. C (relative infinity norms) for a given state */
void orc_coupled_residual(const orc_grid* g, const orc_params* p,
                          const double* phi, const double* fstar,
                          const double* Fstar, double dt, const double* f,
                          const double* F, double* rf, double* rF,
                          double* res_f, double* res_F);

/* a6: compensated totals sum V x */
double orc_total(const orc_grid* g, const double* x);

/* a7: EOS sigma(Gamma), Gamma = f/delta where delta >= 1e-3/eps else 0 */
void orc_eos(const orc_grid* g, const orc_params* p, const double* f,
             const double* phi, double* gamma, double* sigma);
/* a8: Marangoni force F_Ma = delta_m (I - n n) grad sigma (Sec. 2.4).
   dm_mode 0: delta_m = |grad C| (centred); 1: PLIC area / cell volume. */
void orc_marangoni(const orc_grid* g, const orc_params* p, const double* f,
                   const double* phi, const double* C, int dm_mode,
                   double* sigma, double* force);

/* PLIC helpers (exposed for pinning): fraction of the unit cell below the
   plane m.x = alpha, and the interface area inside the unit cell. */
double orc_plic_volume(int dim, const double* m, double alpha);
double orc_plic_area(int dim, const double* m, double C);

/* One step of the ACDI phase-field equation (Sec. 2.5): BCG advection of
   phi (skipped when ux is NULL), then the explicit central regularisation
   flux with velocity scale zeta and width eps; clip = 1 clips the result
   to [0, 1]; phi_out may not alias phi. */
void orc_acdi_step(const orc_grid* g, const double* ux, const double* uy,
                   const double* uz, double dt, double zeta, double eps, int clip,
                   const double* phi, double* phi_out);

/* Capillary force F_cap = sigma kappa delta_s n, kappa = -div n (flux
   form over the faces), delta_s = |grad C| (Sec. 2.2, 2.4).  force holds
   ndim component arrays; kappa (may be NULL) receives the curvature. */
void orc_capillary(const orc_grid* g, const double* phi, const double* C,
                   const double* sigma, double eps, double* kappa,
                   double* force);

/* a9: time step from the CFL criterion of Sec. 3.3 */
double orc_cfl_dt(int ndim, double h, double umax, double D, double eps,
                  double safety);

#ifdef __cplusplus
}
#endif
#endif
