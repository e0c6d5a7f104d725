/*
 * FP64 CPU oracle for the coupled soluble-surfactant step of the hybrid
 * VoF / phase-field method (arxiv 2605.27534).
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the
 * benchmark's CPU-baseline leg to check and time the CUDA library.  The
 * product path never loads it.  Plain serial double precision; every loop
 * follows the paper's formula directly, with no blocking or fusion.
 *
 * Readings of points the paper leaves open are marked READING and listed in
 * the design notes of the repository.
 */
#ifdef _OPENMP
#include <omp.h>
#endif
#include "sfx_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define PI_D 3.14159265358979323846

/* ------------------------------------------------------------------ grid */

static int ndim_of(const orc_grid* g) { return g->geom == ORC_3D ? 3 : 2; }
static size_t ncell_of(const orc_grid* g) {
  return (size_t)g->nx * g->ny * g->nz;
}
static size_t idx(const orc_grid* g, int i, int j, int k) {
  return ((size_t)k * g->ny + j) * g->nx + i;
}
static int extent(const orc_grid* g, int d) {
  return d == 0 ? g->nx : (d == 1 ? g->ny : g->nz);
}

/* Cell volume: h^2 (planar, unit depth), h^3 (3D), and the exact ring
   volume pi (r+^2 - r-^2) dz of App. B with r- = i h, r+ = (i+1) h. */
/* threads the order-independent loops run on (1 in the serial build) */
int orc_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

double orc_cell_volume(const orc_grid* g, int i, int j, int k) {
  (void)j; (void)k;
  double h = g->h;
  if (g->geom == ORC_PLANAR) return h * h;
  if (g->geom == ORC_3D) return h * h * h;
  return PI_D * (double)(2 * i + 1) * h * h * h;
}

/* Area of the face on the minus side of cell (i,j,k) in direction d:
   planar h, 3D h^2; axisymmetric radial face 2 pi r dz at r = i h (zero on
   the axis) and axial face pi (r+^2 - r-^2)  (App. B). */
static double face_area(const orc_grid* g, int d, int i, int j, int k) {
  (void)j; (void)k;
  double h = g->h;
  if (g->geom == ORC_PLANAR) return h;
  if (g->geom == ORC_3D) return h * h;
  if (d == 0) return 2.0 * PI_D * (i * h) * h;
  return PI_D * (double)(2 * i + 1) * h * h;
}

/* neighbour of (i,j,k) shifted by s in direction d; returns 0 outside */
static int shift(const orc_grid* g, int d, int s, int* i, int* j, int* k) {
  int c[3] = {*i, *j, *k};
  c[d] += s;
  if (c[d] < 0 || c[d] >= extent(g, d)) return 0;
  *i = c[0]; *j = c[1]; *k = c[2];
  return 1;
}

/* value of a cell field at the neighbour, or at the cell itself outside the
   domain (zero-gradient wall; symmetry on the axis) */
static double nb_or_self(const orc_grid* g, const double* x, int i, int j,
                         int k, int d, int s) {
  int a = i, b = j, c = k;
  if (!shift(g, d, s, &a, &b, &c)) return x[idx(g, i, j, k)];
  return x[idx(g, a, b, c)];
}

/* face arrays: direction d has extent+1 faces along d */
static size_t face_idx(const orc_grid* g, int d, int i, int j, int k) {
  int fx = g->nx + (d == 0), fy = g->ny + (d == 1);
  return ((size_t)k * fy + j) * fx + i;
}
static size_t nface_of(const orc_grid* g, int d) {
  return (size_t)(g->nx + (d == 0)) * (g->ny + (d == 1)) * (g->nz + (d == 2));
}

/* Neumaier compensated sum helper */
typedef struct { double s, c; } ksum;
static void kadd(ksum* a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
  else a->c += (x - t) + a->s;
  a->s = t;
}

/* ---------------------------------------------------- a1/a2: phase field */

/* Godunov upwind |grad chi| for the sign s of chi0 (first-order HJ). */
static double godunov_grad(const orc_grid* g, const double* chi, int i, int j,
                           int k, double s) {
  double h = g->h, acc = 0.0;
  double c0 = chi[idx(g, i, j, k)];
  for (int d = 0; d < ndim_of(g); ++d) {
    double a = (c0 - nb_or_self(g, chi, i, j, k, d, -1)) / h; /* backward */
    double b = (nb_or_self(g, chi, i, j, k, d, +1) - c0) / h; /* forward */
    double t;
    if (s > 0) {
      double ap = a > 0 ? a : 0, bm = b < 0 ? b : 0;
      t = ap * ap > bm * bm ? ap * ap : bm * bm;
    } else {
      double am = a < 0 ? a : 0, bp = b > 0 ? b : 0;
      t = am * am > bp * bp ? am * am : bp * bp;
    }
    acc += t;
  }
  return sqrt(acc);
}

/* READING: chi0 = 2h(C - 1/2) (positive inside fluid 1), first-order
   Godunov pseudo-time steps, and the Russo-Smereka sub-cell fix in cells
   whose chi0 changes sign against a face neighbour (Sec. 2.5). */
void orc_redistance(const orc_grid* g, const double* C, int iters, double dtau,
                    double* chi) {
  size_t n = ncell_of(g);
  double h = g->h;
  double* chi0 = (double*)malloc(n * sizeof(double));
  double* nxt = (double*)malloc(n * sizeof(double));
  for (size_t c = 0; c < n; ++c) chi0[c] = 2.0 * h * (C[c] - 0.5);
  memcpy(chi, chi0, n * sizeof(double));
  for (int it = 0; it < iters; ++it) {
    for (int k = 0; k < g->nz; ++k)
      for (int j = 0; j < g->ny; ++j)
        for (int i = 0; i < g->nx; ++i) {
          size_t c = idx(g, i, j, k);
          double s0 = chi0[c];
          double s = s0 > 0 ? 1.0 : (s0 < 0 ? -1.0 : 0.0);
          int near = 0;
          for (int d = 0; d < ndim_of(g) && !near; ++d)
            for (int sh = -1; sh <= 1; sh += 2) {
              int a = i, b = j, cc = k;
              if (shift(g, d, sh, &a, &b, &cc) &&
                  s0 * chi0[idx(g, a, b, cc)] < 0) near = 1;
            }
          if (near) {
            /* sub-cell fix: relax towards the distance D = h chi0/|dchi0| */
            double acc = 0.0;
            for (int d = 0; d < ndim_of(g); ++d) {
              double m = nb_or_self(g, chi0, i, j, k, d, -1);
              double p = nb_or_self(g, chi0, i, j, k, d, +1);
              double q = fabs(p - m) * 0.5;
              if (fabs(p - s0) > q) q = fabs(p - s0);
              if (fabs(s0 - m) > q) q = fabs(s0 - m);
              acc += q * q;
            }
            double dchi = sqrt(acc);
            if (dchi < 1e-300) dchi = 1e-300;
            double Dist = h * s0 / dchi;
            nxt[c] = chi[c] - (dtau / h) * (s * fabs(chi[c]) - Dist);
          } else {
            nxt[c] = chi[c] - dtau * s * (godunov_grad(g, chi, i, j, k, s) - 1.0);
          }
        }
    memcpy(chi, nxt, n * sizeof(double));
  }
  free(chi0);
  free(nxt);
}

/* phi = (1 - tanh(chi/(2 eps)))/2 (Sec. 2.5), delta = phi(1-phi)/eps (Sec. 2.6) */
void orc_phase_field(const orc_grid* g, const double* chi, double eps,
                     double* phi, double* delta) {
  size_t n = ncell_of(g);
  for (size_t c = 0; c < n; ++c) {
    double p = 0.5 * (1.0 - tanh(chi[c] / (2.0 * eps)));
    phi[c] = p;
    if (delta) delta[c] = p * (1.0 - p) / eps;
  }
}

void orc_phase_field_build(const orc_grid* g, const double* C, int iters,
                           double dtau, double eps, double* chi, double* phi,
                           double* delta) {
  orc_redistance(g, C, iters, dtau, chi);
  orc_phase_field(g, chi, eps, phi, delta);
}

/* n = grad phi / |grad phi| with centred differences (Sec. 2.6).
   READING: the paper leaves n undefined where phi is flat.  Beyond the
   redistancing band phi is flat up to variations many orders below its
   own profile slope, and there the direction of grad phi is set by those
   variations (by round-off at the last few bits).  With
   q = |grad phi| / (phi (1 - phi)/eps), the ratio to the slope of the
   equilibrium profile, n is scaled by w = min(max(q/ORC_NORMAL_KAPPA - 1,
   0), 1): n = 0 where q <= ORC_NORMAL_KAPPA, the unit vector where
   q >= 2 ORC_NORMAL_KAPPA, and a linear ramp between, so that n (and the
   step) depends continuously on phi; n = 0 where |grad phi| < 1e-30. */
void orc_normals(const orc_grid* g, const double* phi, double eps, double* n) {
  size_t N = ncell_of(g);
  int D = ndim_of(g);
#pragma omp parallel for collapse(2)
  for (int k = 0; k < g->nz; ++k)
    for (int j = 0; j < g->ny; ++j)
      for (int i = 0; i < g->nx; ++i) {
        size_t c = idx(g, i, j, k);
        double gp[3] = {0, 0, 0}, m2 = 0;
        for (int d = 0; d < D; ++d) {
          gp[d] = (nb_or_self(g, phi, i, j, k, d, +1) -
                   nb_or_self(g, phi, i, j, k, d, -1)) / (2.0 * g->h);
          m2 += gp[d] * gp[d];
        }
        double m = sqrt(m2);
        double slope = phi[c] * (1.0 - phi[c]) / eps;
        double w = 0.0;
        if (m >= 1e-30) {
          w = m / (ORC_NORMAL_KAPPA * slope) - 1.0;
          if (w > 1.0) w = 1.0;
          if (!(w > 0.0)) w = 0.0;
        }
        for (int d = 0; d < D; ++d) n[d * N + c] = w > 0.0 ? w * (gp[d] / m) : 0.0;
      }
}

/* B_f = -Df 2(0.5-phi)/eps n, B_F = -DF (1-phi)/eps n (App. C); face value
   is the mean of the two adjacent cell values (Sec. 3.2). */
void orc_face_drift(const orc_grid* g, const orc_params* p, const double* phi,
                    int which, double* Bx, double* By, double* Bz) {
  size_t N = ncell_of(g);
  int D = ndim_of(g);
  double* n = (double*)malloc((size_t)D * N * sizeof(double));
  double* Bc = (double*)malloc((size_t)D * N * sizeof(double));
  orc_normals(g, phi, p->eps, n);
  for (size_t c = 0; c < N; ++c) {
    double s = which == 0 ? -p->Df * 2.0 * (0.5 - phi[c]) / p->eps
                          : -p->DF * (1.0 - phi[c]) / p->eps;
    for (int d = 0; d < D; ++d) Bc[d * N + c] = s * n[d * N + c];
  }
  double* out[3] = {Bx, By, Bz};
  for (int d = 0; d < D; ++d) {
    int fx = g->nx + (d == 0), fy = g->ny + (d == 1), fz = g->nz + (d == 2);
    for (int k = 0; k < fz; ++k)
      for (int j = 0; j < fy; ++j)
        for (int i = 0; i < fx; ++i) {
          int pos = d == 0 ? i : (d == 1 ? j : k);
          size_t f = face_idx(g, d, i, j, k);
          if (pos == 0 || pos == extent(g, d)) { out[d][f] = 0.0; continue; }
          int li = i, lj = j, lk = k;
          if (d == 0) li--; else if (d == 1) lj--; else lk--;
          out[d][f] = 0.5 * (Bc[d * N + idx(g, li, lj, lk)] +
                             Bc[d * N + idx(g, i, j, k)]);
        }
  }
  free(n);
  free(Bc);
}

/* ------------------------------------------------- a5: elliptic operator */

/* Face quantity G = D da/dn + B a_up written as G = cL a_L + cR a_R.
   Centred diffusive flux; first-order upwind B flux (Sec. 3.2).
   READING: the printed rule takes the left value when B > 0; the transport
   velocity of div(B xi) on the right-hand side is -B, so the upwind value is
   the left one when B < 0.  literal = 1 selects the printed rule. */
static void face_coeffs(double D, double h, double B, int literal, double* cL,
                        double* cR) {
  *cL = -D / h;
  *cR = D / h;
  int left = literal ? (B > 0) : (B < 0);
  if (left) *cL += B;
  else *cR += B;
}

static const double* face_arr(const double* Bx, const double* By,
                              const double* Bz, int d) {
  return d == 0 ? Bx : (d == 1 ? By : Bz);
}

/* L(a) at one cell, and its diagonal d L(a)_c / d a_c:
   L(a)_c = lambda_c a_c - (1/V_c) sum_d (A+ G+ - A- G-)  (Sec. 3.1-3.2). */
static void cell_operator(const orc_grid* g, double D, const double* Bx,
                          const double* By, const double* Bz, int literal,
                          const double* lambda, const double* a, int i, int j,
                          int k, double* Lc, double* diag) {
  size_t c = idx(g, i, j, k);
  double V = orc_cell_volume(g, i, j, k);
  double flux = 0.0, dflux = 0.0;
  for (int d = 0; d < ndim_of(g); ++d) {
    const double* B = face_arr(Bx, By, Bz, d);
    /* plus face: this cell is the left cell */
    int pi_ = i, pj = j, pk = k;
    if (shift(g, d, +1, &pi_, &pj, &pk)) {
      int fi = i + (d == 0), fj = j + (d == 1), fk = k + (d == 2);
      double A = face_area(g, d, fi, fj, fk);
      double cL, cR;
      face_coeffs(D, g->h, B[face_idx(g, d, fi, fj, fk)], literal, &cL, &cR);
      flux += A * (cL * a[c] + cR * a[idx(g, pi_, pj, pk)]);
      dflux += A * cL;
    }
    /* minus face: this cell is the right cell */
    int mi = i, mj = j, mk = k;
    if (shift(g, d, -1, &mi, &mj, &mk)) {
      double A = face_area(g, d, i, j, k);
      double cL, cR;
      face_coeffs(D, g->h, B[face_idx(g, d, i, j, k)], literal, &cL, &cR);
      flux -= A * (cL * a[idx(g, mi, mj, mk)] + cR * a[c]);
      dflux -= A * cR;
    }
  }
  *Lc = lambda[c] * a[c] - flux / V;
  *diag = lambda[c] - dflux / V;
}

void orc_apply_operator(const orc_grid* g, double D, const double* Bx,
                        const double* By, const double* Bz, int literal_upwind,
                        const double* lambda, const double* a, double* out) {
#pragma omp parallel for collapse(2)
  for (int k = 0; k < g->nz; ++k)
    for (int j = 0; j < g->ny; ++j)
      for (int i = 0; i < g->nx; ++i) {
        double Lc, dg;
        cell_operator(g, D, Bx, By, Bz, literal_upwind, lambda, a, i, j, k,
                      &Lc, &dg);
        out[idx(g, i, j, k)] = Lc;
      }
}

static double rel_residual(const orc_grid* g, double D, const double* Bx,
                           const double* By, const double* Bz, int literal,
                           const double* lambda, const double* b,
                           const double* a) {
  double rmax = 0.0, bmax = 0.0;
  int nan = 0;
  /* the maxima do not depend on the order: the OpenMP build of the oracle
     (a CPU baseline over all host cores) gives the same value */
#pragma omp parallel for collapse(2) reduction(max : rmax, bmax) reduction(| : nan)
  for (int k = 0; k < g->nz; ++k)
    for (int j = 0; j < g->ny; ++j)
      for (int i = 0; i < g->nx; ++i) {
        size_t c = idx(g, i, j, k);
        double Lc, dg;
        cell_operator(g, D, Bx, By, Bz, literal, lambda, a, i, j, k, &Lc, &dg);
        double r = fabs(b[c] - Lc);
        if (r != r) nan = 1;
        else if (r > rmax) rmax = r;
        if (fabs(b[c]) > bmax) bmax = fabs(b[c]);
      }
  if (nan) return NAN;
  return rmax / (bmax > 1e-300 ? bmax : 1e-300);
}

/* Lexicographic Gauss-Seidel: a_c += (b_c - L(a)_c) / diag_c.  The paper
   solves these problems by multigrid; the converged answer does not depend
   on the solver, and plain Gauss-Seidel is the simplest one to check. */
int orc_elliptic_solve(const orc_grid* g, double D, const double* Bx,
                       const double* By, const double* Bz, int literal_upwind,
                       const double* lambda, const double* b, double* a,
                       double tol, int max_sweeps, double* rel_res) {
  double res = rel_residual(g, D, Bx, By, Bz, literal_upwind, lambda, b, a);
  double best = res;
  int stall = 0, sweeps = 0;
  while (res > tol && sweeps < max_sweeps) {
    for (int k = 0; k < g->nz; ++k)
      for (int j = 0; j < g->ny; ++j)
        for (int i = 0; i < g->nx; ++i) {
          size_t c = idx(g, i, j, k);
          double Lc, dg;
          cell_operator(g, D, Bx, By, Bz, literal_upwind, lambda, a, i, j, k,
                        &Lc, &dg);
          a[c] += (b[c] - Lc) / dg;
        }
    ++sweeps;
    res = rel_residual(g, D, Bx, By, Bz, literal_upwind, lambda, b, a);
    /* stop at the round-off floor: 50 sweeps without a 0.1 % improvement */
    if (res < best * (1.0 - 1e-3)) { best = res; stall = 0; }
    else if (++stall >= 50) break;
  }
  if (rel_res) *rel_res = res;
  return res <= tol ? sweeps : -sweeps;
}

/* ------------------------------------------------------ a3: BCG advection */

/* monotonised-central limited difference (van Leer), in value units */
static double mc_slope(double xm, double x0, double xp) {
  double dl = x0 - xm, dr = xp - x0;
  if (dl * dr <= 0.0) return 0.0;
  double dc = 0.5 * (xp - xm);
  double m = fabs(dc);
  if (2.0 * fabs(dl) < m) m = 2.0 * fabs(dl);
  if (2.0 * fabs(dr) < m) m = 2.0 * fabs(dr);
  return dc > 0 ? m : -m;
}

static const double* vel_arr(const double* ux, const double* uy,
                             const double* uz, int d) {
  return d == 0 ? ux : (d == 1 ? uy : uz);
}

/* Time-centred face value of the BCG predictor (Sec. 3.1): the upwind cell
   value extrapolated to the face over half a step along the normal, minus
   half a step of transverse upwind advection.  Face (fi,fj,fk) in direction
   d lies between cell (f - e_d) and cell f. */
static double bcg_face_value(const orc_grid* g, const double* ux,
                             const double* uy, const double* uz, double dt,
                             const double* xi, double bc_in, int d, int fi,
                             int fj, int fk, double u) {
  int pos = d == 0 ? fi : (d == 1 ? fj : fk);
  int n = extent(g, d);
  double sgn = u > 0 ? 1.0 : -1.0;
  /* upwind cell */
  int ui = fi, uj = fj, uk = fk;
  if (u > 0) {
    if (pos == 0) return bc_in; /* inflow through the minus wall */
    if (d == 0) ui--; else if (d == 1) uj--; else uk--;
  } else {
    if (pos == n) return bc_in; /* inflow through the plus wall */
  }
  size_t U = idx(g, ui, uj, uk);
  double x0 = xi[U];
  double cour = u * dt / g->h;
  double slope = mc_slope(nb_or_self(g, xi, ui, uj, uk, d, -1), x0,
                          nb_or_self(g, xi, ui, uj, uk, d, +1));
  double val = x0 + 0.5 * (sgn - cour) * slope;
  for (int t = 0; t < ndim_of(g); ++t) {
    if (t == d) continue;
    const double* vt = vel_arr(ux, uy, uz, t);
    int ai = ui + (t == 0), aj = uj + (t == 1), ak = uk + (t == 2);
    double vbar = 0.5 * (vt[face_idx(g, t, ui, uj, uk)] +
                         vt[face_idx(g, t, ai, aj, ak)]);
    double dx = vbar > 0 ? x0 - nb_or_self(g, xi, ui, uj, uk, t, -1)
                         : nb_or_self(g, xi, ui, uj, uk, t, +1) - x0;
    val -= 0.5 * dt * vbar * dx / g->h;
  }
  return val;
}

void orc_advect_bcg(const orc_grid* g, const double* ux, const double* uy,
                    const double* uz, double dt, const double* xi,
                    double bc_in, double* xi_star) {
#pragma omp parallel for collapse(2)
  for (int k = 0; k < g->nz; ++k)
    for (int j = 0; j < g->ny; ++j)
      for (int i = 0; i < g->nx; ++i) {
        double V = orc_cell_volume(g, i, j, k);
        double div = 0.0;
        for (int d = 0; d < ndim_of(g); ++d) {
          const double* u = vel_arr(ux, uy, uz, d);
          /* minus face */
          double um = u[face_idx(g, d, i, j, k)];
          if (um != 0.0)
            div -= face_area(g, d, i, j, k) * um *
                   bcg_face_value(g, ux, uy, uz, dt, xi, bc_in, d, i, j, k, um);
          /* plus face */
          int pi_ = i + (d == 0), pj = j + (d == 1), pk = k + (d == 2);
          double up = u[face_idx(g, d, pi_, pj, pk)];
          if (up != 0.0)
            div += face_area(g, d, pi_, pj, pk) * up *
                   bcg_face_value(g, ux, uy, uz, dt, xi, bc_in, d, pi_, pj, pk,
                                  up);
        }
        size_t c = idx(g, i, j, k);
        xi_star[c] = xi[c] - dt * div / V;
      }
}

/* ------------------------------------------ a4: coupled implicit source */

typedef struct {
  double *Bfx, *Bfy, *Bfz, *BFx, *BFy, *BFz;
  double *lam, *rhs, *pe, *finf;
} coupled_ws;

static void coupled_ws_init(const orc_grid* g, const orc_params* p,
                            const double* phi, coupled_ws* w) {
  size_t N = ncell_of(g);
  w->Bfx = (double*)calloc(nface_of(g, 0), sizeof(double));
  w->Bfy = (double*)calloc(nface_of(g, 1), sizeof(double));
  w->Bfz = (double*)calloc(g->geom == ORC_3D ? nface_of(g, 2) : 1, sizeof(double));
  w->BFx = (double*)calloc(nface_of(g, 0), sizeof(double));
  w->BFy = (double*)calloc(nface_of(g, 1), sizeof(double));
  w->BFz = (double*)calloc(g->geom == ORC_3D ? nface_of(g, 2) : 1, sizeof(double));
  w->lam = (double*)malloc(N * sizeof(double));
  w->rhs = (double*)malloc(N * sizeof(double));
  w->pe = (double*)malloc(N * sizeof(double));
  w->finf = (double*)malloc(N * sizeof(double));
  orc_face_drift(g, p, phi, 0, w->Bfx, w->Bfy, w->Bfz);
  orc_face_drift(g, p, phi, 1, w->BFx, w->BFy, w->BFz);
  for (size_t c = 0; c < N; ++c) {
    /* READING: the small constant of Sec. 2.6 is added to phi: F/(phi+eta) */
    w->pe[c] = phi[c] + p->eta;
    /* f_inf = Gamma_inf delta_phi with delta_phi = phi(1-phi)/eps */
    w->finf[c] = p->gamma_inf * phi[c] * (1.0 - phi[c]) / p->eps;
  }
}

static void coupled_ws_free(coupled_ws* w) {
  free(w->Bfx); free(w->Bfy); free(w->Bfz);
  free(w->BFx); free(w->BFy); free(w->BFz);
  free(w->lam); free(w->rhs); free(w->pe); free(w->finf);
}

/* App. C coefficients of the f problem for a given F:
   lambda_f = 1/dt + r_d + r_a F/phi,  b_f = f_star/dt + r_a (F/phi) f_inf */
static void f_problem(const orc_grid* g, const orc_params* p, coupled_ws* w,
                      const double* fstar, const double* F, double dt) {
  size_t N = ncell_of(g);
#pragma omp parallel for
  for (size_t c = 0; c < N; ++c) {
    double Fs = F[c] / w->pe[c];
    w->lam[c] = 1.0 / dt + p->kd + p->ka * Fs;
    w->rhs[c] = fstar[c] / dt + p->ka * Fs * w->finf[c];
  }
}

/* App. C coefficients of the F problem for a given f:
   lambda_F = 1/dt + r_a (f_inf - f)/phi,  b_F = F_star/dt + r_d f */
static void F_problem(const orc_grid* g, const orc_params* p, coupled_ws* w,
                      const double* Fstar, const double* f, double dt) {
  size_t N = ncell_of(g);
#pragma omp parallel for
  for (size_t c = 0; c < N; ++c) {
    w->lam[c] = 1.0 / dt + p->ka * (w->finf[c] - f[c]) / w->pe[c];
    w->rhs[c] = Fstar[c] / dt + p->kd * f[c];
  }
}

void orc_coupled_residual(const orc_grid* g, const orc_params* p,
                          const double* phi, const double* fstar,
                          const double* Fstar, double dt, const double* f,
                          const double* F, double* rf, double* rF,
                          double* res_f, double* res_F) {
  size_t N = ncell_of(g);
  coupled_ws w;
  coupled_ws_init(g, p, phi, &w);
  double* La = (double*)malloc(N * sizeof(double));
  double mx, mb;

  f_problem(g, p, &w, fstar, F, dt);
  orc_apply_operator(g, p->Df, w.Bfx, w.Bfy, w.Bfz, p->literal_upwind, w.lam, f, La);
  mx = 0; mb = 0;
  for (size_t c = 0; c < N; ++c) {
    double r = w.rhs[c] - La[c];
    if (rf) rf[c] = r;
    if (fabs(r) > mx) mx = fabs(r);
    if (fabs(w.rhs[c]) > mb) mb = fabs(w.rhs[c]);
  }
  if (res_f) *res_f = mx / (mb > 1e-300 ? mb : 1e-300);

  F_problem(g, p, &w, Fstar, f, dt);
  orc_apply_operator(g, p->DF, w.BFx, w.BFy, w.BFz, p->literal_upwind, w.lam, F, La);
  mx = 0; mb = 0;
  for (size_t c = 0; c < N; ++c) {
    double r = w.rhs[c] - La[c];
    if (rF) rF[c] = r;
    if (fabs(r) > mx) mx = fabs(r);
    if (fabs(w.rhs[c]) > mb) mb = fabs(w.rhs[c]);
  }
  if (res_F) *res_F = mx / (mb > 1e-300 ? mb : 1e-300);
  free(La);
  coupled_ws_free(&w);
}

/* READING: App. C calls the system fully implicit without naming the
   iteration.  Picard: solve the f problem with the latest F, then the F
   problem with the new f, until both nonlinear residuals are below tol. */
void orc_coupled_implicit(const orc_grid* g, const orc_params* p,
                          const double* phi, const double* fstar,
                          const double* Fstar, double dt, const orc_opts* o,
                          double* f, double* F, orc_stats* st) {
  size_t N = ncell_of(g);
  coupled_ws w;
  coupled_ws_init(g, p, phi, &w);
  memcpy(f, fstar, N * sizeof(double));
  memcpy(F, Fstar, N * sizeof(double));
  double tol_lin = 0.1 * o->tol;
  int it = 0, sweeps = 0, conv = 0;
  double rf = 1, rF = 1, rr;
  for (it = 1; it <= o->max_picard; ++it) {
    f_problem(g, p, &w, fstar, F, dt);
    int s = orc_elliptic_solve(g, p->Df, w.Bfx, w.Bfy, w.Bfz, p->literal_upwind,
                               w.lam, w.rhs, f, tol_lin, o->max_sweeps, &rr);
    sweeps += s < 0 ? -s : s;
    F_problem(g, p, &w, Fstar, f, dt);
    s = orc_elliptic_solve(g, p->DF, w.BFx, w.BFy, w.BFz, p->literal_upwind,
                           w.lam, w.rhs, F, tol_lin, o->max_sweeps, &rr);
    sweeps += s < 0 ? -s : s;
    orc_coupled_residual(g, p, phi, fstar, Fstar, dt, f, F, NULL, NULL, &rf, &rF);
    if (rf <= o->tol && rF <= o->tol) { conv = 1; break; }
  }
  if (st) {
    st->picard = it > o->max_picard ? o->max_picard : it;
    st->sweeps = sweeps;
    st->res_f = rf;
    st->res_F = rF;
    st->converged = conv;
  }
  coupled_ws_free(&w);
}

void orc_surfactant_step(const orc_grid* g, const orc_params* p,
                         const double* phi, const double* ux, const double* uy,
                         const double* uz, double dt, const orc_opts* o,
                         double* f, double* F, orc_stats* st) {
  size_t N = ncell_of(g);
  double* fs = (double*)malloc(N * sizeof(double));
  double* Fs = (double*)malloc(N * sizeof(double));
  if (ux) {
    orc_advect_bcg(g, ux, uy, uz, dt, f, p->bc_f, fs);
    orc_advect_bcg(g, ux, uy, uz, dt, F, p->bc_F, Fs);
  } else {
    memcpy(fs, f, N * sizeof(double));
    memcpy(Fs, F, N * sizeof(double));
  }
  orc_coupled_implicit(g, p, phi, fs, Fs, dt, o, f, F, st);
  if (st) {
    st->mass_f = orc_total(g, f);
    st->mass_F = orc_total(g, F);
  }
  free(fs);
  free(Fs);
}

/* ------------------------------------------------------------ a6: totals */

double orc_total(const orc_grid* g, const double* x) {
  ksum s = {0, 0};
  for (int k = 0; k < g->nz; ++k)
    for (int j = 0; j < g->ny; ++j)
      for (int i = 0; i < g->nx; ++i)
        kadd(&s, orc_cell_volume(g, i, j, k) * x[idx(g, i, j, k)]);
  return s.s + s.c;
}

/* --------------------------------------------------------- a7/a8: forces */

/* READING: Gamma = f/delta_phi where delta_phi >= 1e-3/eps, else 0. */
void orc_eos(const orc_grid* g, const orc_params* p, const double* f,
             const double* phi, double* gamma, double* sigma) {
  size_t N = ncell_of(g);
  for (size_t c = 0; c < N; ++c) {
    double del = phi[c] * (1.0 - phi[c]) / p->eps;
    double G = del >= 1e-3 / p->eps ? f[c] / del : 0.0;
    double x = G / p->gamma_inf;
    double s;
    if (p->eos == ORC_EOS_LANGMUIR) {
      /* sigma = sigma0 (1 + E ln(1 - Gamma/Gamma_inf))  (Sec. 2.3, Sec. 5) */
      if (x > 1.0 - 1e-12) x = 1.0 - 1e-12;
      s = p->sigma0 * (1.0 + p->E * log1p(-x));
    } else if (p->eos == ORC_EOS_LINEAR) {
      s = p->sigma0 * (1.0 - p->E * x);      /* Sec. 2.3 linear limit */
    } else {
      s = p->sigma0 * (1.0 - tanh(p->E * x)); /* Sec. 6 */
    }
    if (gamma) gamma[c] = G;
    sigma[c] = s;
  }
}

/* Volume of the unit cube below the plane m.x = a, for m >= 0 with
   sum m = 1 (Scardovelli & Zaleski 2000), and its derivative in a.  The
   cubic of that paper is evaluated region by region in expanded form, so
   components near zero lose no precision (the region whose width equals a
   tiny component is simply empty).  By symmetry V(a) = 1 - V(1 - a), so
   only a <= 1/2 is evaluated directly.  m is sorted ascending here. */
static void sort_asc(double* m, int n) {
  for (int i = 1; i < n; ++i)
    for (int j = i; j > 0 && m[j] < m[j - 1]; --j) {
      double t = m[j]; m[j] = m[j - 1]; m[j - 1] = t;
    }
}

/* value (want_derivative = 0) or derivative (1) for a <= 1/2 */
static double plic_half(int dim, const double* m, double a, int want_derivative) {
  if (a <= 0.0) return 0.0;
  if (dim == 2) {
    double m1 = m[0], m2 = m[1];           /* m1 <= m2, m1 + m2 = 1 */
    if (a < m1)                            /* corner triangle */
      return want_derivative ? a / (m1 * m2) : a * a / (2.0 * m1 * m2);
    return want_derivative ? 1.0 / m2 : (a - 0.5 * m1) / m2; /* trapezoid */
  }
  double m1 = m[0], m2 = m[1], m3 = m[2];  /* ascending, sum 1 */
  double v, dv;
  if (a < m1) {                            /* corner tetrahedron */
    v = a * a * a / (6.0 * m1 * m2 * m3);
    dv = a * a / (2.0 * m1 * m2 * m3);
  } else if (a < m2) {                     /* wedge along the m1 axis */
    v = (a * a - a * m1 + m1 * m1 / 3.0) / (2.0 * m2 * m3);
    dv = (2.0 * a - m1) / (2.0 * m2 * m3);
  } else if (a < m3 && a < m1 + m2) {      /* two corners cut */
    double u = a - m2;
    v = (3.0 * a * a - 3.0 * a * m1 + m1 * m1) / (6.0 * m2 * m3) -
        u * u * u / (6.0 * m1 * m2 * m3);
    dv = (2.0 * a - m1) / (2.0 * m2 * m3) - u * u / (2.0 * m1 * m2 * m3);
  } else if (m3 >= m1 + m2) {              /* plane spans the m3 direction */
    v = (a - 0.5 * (m1 + m2)) / m3;
    dv = 1.0 / m3;
  } else {                                 /* m3 <= a < m1 + m2 */
    double u = a - m2, w = a - m3;
    v = (3.0 * a * a - 3.0 * a * m1 + m1 * m1) / (6.0 * m2 * m3) -
        (u * u * u + w * w * w) / (6.0 * m1 * m2 * m3);
    dv = (2.0 * a - m1) / (2.0 * m2 * m3) - (u * u + w * w) / (2.0 * m1 * m2 * m3);
  }
  return want_derivative ? dv : v;
}

static double plic_vol_pos(int dim, const double* m, double a) {
  double ms[3] = {m[0], m[1], dim == 3 ? m[2] : 0.0};
  sort_asc(ms, dim);
  if (a <= 0.0) return 0.0;
  if (a >= 1.0) return 1.0;
  if (a <= 0.5) return plic_half(dim, ms, a, 0);
  return 1.0 - plic_half(dim, ms, 1.0 - a, 0);
}

static double plic_dvol_pos(int dim, const double* m, double a) {
  double ms[3] = {m[0], m[1], dim == 3 ? m[2] : 0.0};
  sort_asc(ms, dim);
  if (a <= 0.0 || a >= 1.0) return 0.0;
  return plic_half(dim, ms, a <= 0.5 ? a : 1.0 - a, 1);
}

static void plic_normalise(int dim, const double* m, double* mp, double* l2) {
  double s = 0, q = 0;
  for (int d = 0; d < dim; ++d) { s += fabs(m[d]); q += m[d] * m[d]; }
  for (int d = 0; d < dim; ++d) mp[d] = s > 0 ? fabs(m[d]) / s : 0;
  *l2 = s > 0 ? sqrt(q) / s : 0;
}

double orc_plic_volume(int dim, const double* m, double alpha) {
  double mp[3], l2;
  plic_normalise(dim, m, mp, &l2);
  return plic_vol_pos(dim, mp, alpha);
}

/* interface area inside the unit cell for volume fraction C: find alpha by
   bisection on the monotone volume function, then area = |m| dV/dalpha */
double orc_plic_area(int dim, const double* m, double C) {
  if (!(C > 0.0 && C < 1.0)) return 0.0;
  double mp[3], l2;
  plic_normalise(dim, m, mp, &l2);
  if (l2 == 0) return 0.0;
  double lo = 0.0, hi = 1.0;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (plic_vol_pos(dim, mp, mid) < C) lo = mid; else hi = mid;
  }
  return l2 * plic_dvol_pos(dim, mp, 0.5 * (lo + hi));
}

/* Youngs normal of the fluid-1 region: minus the (1,2,1)-weighted gradient
   of C over the 3x3(x3) block, zero-gradient walls */
static void youngs_normal(const orc_grid* g, const double* C, int i, int j,
                          int k, double* m) {
  int D = ndim_of(g);
  for (int d = 0; d < 3; ++d) m[d] = 0.0;
  int kr = D == 3 ? 1 : 0;
  for (int dk = -kr; dk <= kr; ++dk)
    for (int dj = -1; dj <= 1; ++dj)
      for (int di = -1; di <= 1; ++di) {
        int a = i + di, b = j + dj, c = k + dk;
        a = a < 0 ? 0 : (a >= g->nx ? g->nx - 1 : a);
        b = b < 0 ? 0 : (b >= g->ny ? g->ny - 1 : b);
        c = c < 0 ? 0 : (c >= g->nz ? g->nz - 1 : c);
        double w = (di == 0 ? 2.0 : 1.0) * (dj == 0 ? 2.0 : 1.0) *
                   (D == 3 ? (dk == 0 ? 2.0 : 1.0) : 1.0);
        double v = C[idx(g, a, b, c)];
        m[0] -= w * di * v;
        m[1] -= w * dj * v;
        if (D == 3) m[2] -= w * dk * v;
      }
}

void orc_marangoni(const orc_grid* g, const orc_params* p, const double* f,
                   const double* phi, const double* C, int dm_mode,
                   double* sigma, double* force) {
  size_t N = ncell_of(g);
  int D = ndim_of(g);
  double* n = (double*)malloc((size_t)D * N * sizeof(double));
  orc_eos(g, p, f, phi, NULL, sigma);
  orc_normals(g, phi, p->eps, n);
  for (int k = 0; k < g->nz; ++k)
    for (int j = 0; j < g->ny; ++j)
      for (int i = 0; i < g->nx; ++i) {
        size_t c = idx(g, i, j, k);
        double gs[3] = {0, 0, 0}, nd = 0;
        for (int d = 0; d < D; ++d) {
          gs[d] = (nb_or_self(g, sigma, i, j, k, d, +1) -
                   nb_or_self(g, sigma, i, j, k, d, -1)) / (2.0 * g->h);
          nd += n[d * N + c] * gs[d];
        }
        double dm;
        if (dm_mode == 0) {
          double q = 0;
          for (int d = 0; d < D; ++d) {
            double gc = (nb_or_self(g, C, i, j, k, d, +1) -
                         nb_or_self(g, C, i, j, k, d, -1)) / (2.0 * g->h);
            q += gc * gc;
          }
          dm = sqrt(q);
        } else {
          /* READING: delta_m = A_f / V_c with the PLIC area; in the
             axisymmetric case both use the cell-centre radius, so the ratio
             equals the planar one (unit-cell area / h). */
          /* READING: interface cells are those with 1e-6 < C < 1 - 1e-6;
             fractions closer to 0 or 1 are round-off of empty or full cells */
          double m[3];
          youngs_normal(g, C, i, j, k, m);
          dm = (C[c] > 1e-6 && C[c] < 1.0 - 1e-6) ? orc_plic_area(D, m, C[c]) / g->h : 0.0;
        }
        for (int d = 0; d < D; ++d)
          force[d * N + c] = dm * (gs[d] - n[d * N + c] * nd);
      }
  free(n);
}

/* ------------------------------------------------ ACDI transport of phi */

/* One step of the ACDI phase-field equation (Sec. 2.5):
     d phi/dt + div(u phi) = div(zeta {eps grad phi
                                - 1/4 (1 - tanh^2(psi/(2 eps))) grad psi/|grad psi|}),
     psi = eps ln((phi + veps)/(1 - phi + veps)),  veps = 1e-6.
   READING: the paper gives the model but not its discretisation.  The
   advective part is the explicit BCG step of Sec. 3.1 (the step of f and
   F; inflow faces carry phi = 1, fluid 2); the regularisation is explicit
   (forward Euler) on the advected phi* in flux form with the central face
   fluxes of Jain (2022): on the face between cells L and R along d,
     a_f = zeta [eps (phi*_R - phi*_L)/h
                 - 1/4 (1 - tanh^2(psi_f/(2 eps))) nbar_f],
   psi_f = (psi_L + psi_R)/2 and nbar_f the mean of the two cells' d
   components of n = grad psi/|grad psi| (centred differences with
   zero-gradient ghosts).  Wall faces carry no flux, the axis face has zero
   area:
     phi = phi* + dt/V_c sum_f (+-) A_f a_f.
   READING: Sec. 2.5 defines the normal as grad psi/|grad psi| only.  Where
   phi saturates (1 - phi or phi far below veps) psi is flat to round-off
   and the direction of its gradient is set by the last bits of phi, while
   1 - tanh^2 there is ~4 veps, not 0: the regularisation would then move
   phi by ~zeta veps dt/h per step in a direction set by round-off.  As for
   the normal of the surfactant drifts, n = 0 where |grad psi| is below
   ORC_ACDI_KAPPA times its equilibrium value 1 (psi is a signed distance
   at equilibrium), or below 1e-30.
   READING: with veps the model's phi saturates towards -veps and 1 + veps,
   and the explicit step overshoots [0, 1] by O(veps) where phi saturates;
   past 1 + veps the logarithm of psi has no value.  psi is formed from phi*
   clipped to [0, 1]; with clip = 1 the result is clipped to [0, 1] as well
   (the paper requires phi in [0, 1], and the surfactant step divides by
   phi + eta, eta = veps), with clip = 0 it keeps the overshoots and sum V
   phi is conserved exactly.  |grad psi| falls below 0.1 only where
   veps dominates psi (phi or 1 - phi below ~0.1 veps); a threshold of 1e-3
   still left cells whose normal turned by 1e-6 under a 1e-15 change of
   phi. */
#define ORC_ACDI_KAPPA 0.1
void orc_acdi_step(const orc_grid* g, const double* ux, const double* uy,
                   const double* uz, double dt, double zeta, double eps, int clip,
                   const double* phi, double* phi_out) {
  const double veps = 1e-6;
  size_t N = ncell_of(g);
  int D = ndim_of(g);
  double* ps = (double*)malloc(N * sizeof(double));
  double* psi = (double*)malloc(N * sizeof(double));
  double* n = (double*)malloc((size_t)D * N * sizeof(double));
  if (ux)
    orc_advect_bcg(g, ux, uy, uz, dt, phi, 1.0, ps);
  else
    memcpy(ps, phi, N * sizeof(double));
  for (size_t c = 0; c < N; ++c) {
    double pc = ps[c] < 0.0 ? 0.0 : (ps[c] > 1.0 ? 1.0 : ps[c]);
    psi[c] = eps * log((pc + veps) / (1.0 - pc + veps));
  }
  for (int k = 0; k < g->nz; ++k)
    for (int j = 0; j < g->ny; ++j)
      for (int i = 0; i < g->nx; ++i) {
        size_t c = idx(g, i, j, k);
        double gp[3] = {0, 0, 0}, m2 = 0;
        for (int d = 0; d < D; ++d) {
          gp[d] = (nb_or_self(g, psi, i, j, k, d, +1) -
                   nb_or_self(g, psi, i, j, k, d, -1)) / (2.0 * g->h);
          m2 += gp[d] * gp[d];
        }
        double m = sqrt(m2);
        int flat = m < 1e-30 || m < ORC_ACDI_KAPPA;
        for (int d = 0; d < D; ++d) n[(size_t)d * N + c] = flat ? 0.0 : gp[d] / m;
      }
  for (int k = 0; k < g->nz; ++k)
    for (int j = 0; j < g->ny; ++j)
      for (int i = 0; i < g->nx; ++i) {
        size_t c = idx(g, i, j, k);
        double div = 0.0;
        for (int d = 0; d < D; ++d) {
          for (int s = -1; s <= 1; s += 2) {
            int a = i, b = j, e = k;
            if (!shift(g, d, s, &a, &b, &e)) continue;   /* wall or axis face */
            size_t o = idx(g, a, b, e);
            /* L and R along +d */
            size_t cL = s < 0 ? o : c, cR = s < 0 ? c : o;
            double A = s < 0 ? face_area(g, d, i, j, k) : face_area(g, d, a, b, e);
            double psif = 0.5 * (psi[cL] + psi[cR]);
            double t = tanh(psif / (2.0 * eps));
            double nbar = 0.5 * (n[(size_t)d * N + cL] + n[(size_t)d * N + cR]);
            double af = zeta * (eps * (ps[cR] - ps[cL]) / g->h - 0.25 * (1.0 - t * t) * nbar);
            div += s * A * af;
          }
        }
        double v = ps[c] + dt * div / orc_cell_volume(g, i, j, k);
        if (clip) v = v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v);
        phi_out[c] = v;
      }
  free(ps);
  free(psi);
  free(n);
}

/* ------------------------------------------------------ capillary force */

/* Capillary force F_cap = sigma kappa delta_s n (Sec. 2.4) with the mean
   curvature kappa = -div n (Sec. 2.2) and delta_s = |grad C|.
   READING: n is the cell-centred unit normal of orc_normals (grad phi /
   |grad phi|, zero where phi is flat).  div n is taken in flux form over
   the faces of the cell, (1/V_c) sum_f (+-) A_f nbar_f, nbar_f the mean of
   the two adjacent cells' normal components along the face normal: on a
   planar grid this is the centred difference, on the axisymmetric grid the
   face areas add the hoop term n_r/r.  A wall face carries no normal
   component (walls are symmetry planes, so the interface meets them at a
   right angle); the axis face has zero area.  grad C is centred with
   zero-gradient ghosts, as delta_m = |grad C| of the Marangoni force.
   sigma is any cell field (the EOS output); kappa may be NULL. */
void orc_capillary(const orc_grid* g, const double* phi, const double* C,
                   const double* sigma, double eps, double* kappa,
                   double* force) {
  size_t N = ncell_of(g);
  int D = ndim_of(g);
  double* n = (double*)malloc((size_t)D * N * sizeof(double));
  orc_normals(g, phi, eps, n);
  for (int k = 0; k < g->nz; ++k)
    for (int j = 0; j < g->ny; ++j)
      for (int i = 0; i < g->nx; ++i) {
        size_t c = idx(g, i, j, k);
        double div = 0.0;
        for (int d = 0; d < D; ++d) {
          const double* nd = n + (size_t)d * N;
          for (int s = -1; s <= 1; s += 2) {
            int a = i, b = j, e = k;
            if (!shift(g, d, s, &a, &b, &e)) continue;   /* wall or axis face */
            /* the face between the cell and its neighbour: minus face of
               the cell (s = -1) or of the neighbour (s = +1) */
            double A = s < 0 ? face_area(g, d, i, j, k) : face_area(g, d, a, b, e);
            double nbar = 0.5 * (nd[c] + nd[idx(g, a, b, e)]);
            div += s * A * nbar;
          }
        }
        double kap = -div / orc_cell_volume(g, i, j, k);
        double q = 0.0;
        for (int d = 0; d < D; ++d) {
          double gc = (nb_or_self(g, C, i, j, k, d, +1) -
                       nb_or_self(g, C, i, j, k, d, -1)) / (2.0 * g->h);
          q += gc * gc;
        }
        double ds = sqrt(q);
        if (kappa) kappa[c] = kap;
        for (int d = 0; d < D; ++d)
          force[(size_t)d * N + c] = sigma[c] * kap * ds * n[(size_t)d * N + c];
      }
  free(n);
}

/* --------------------------------------------------------------- a9: CFL */

/* dt = safety * min(h / (|u|max + D/eps), h^2 / (2 N_d D))  (Sec. 3.3) */
double orc_cfl_dt(int ndim, double h, double umax, double D, double eps,
                  double safety) {
  double dc = h / (umax + D / eps);
  double dd = h * h / (2.0 * ndim * D);
  return safety * (dc < dd ? dc : dd);
}

/* -------------------------------------------- a3': VoF advection of C */

/* READING: the paper tracks c with a geometric VoF method (Sec. 2) and does
   not spell out the scheme.  Directionally split conservative PLIC
   advection (Weymouth & Yue 2010) is taken: for each direction d in turn,
   with face Courant numbers c_f = u_f dt/h,
     C <- C - (Q_+ - Q_-) + H (c_+ - c_-),
   Q_f the volume fraction crossing face f (the fluid of the upwind cell's
   PLIC reconstruction within |c_f| h of the face, signed with u_f) and
   H = 1 where the cell's C at the start of the step exceeds 1/2, else 0.
   The order of the directions alternates from step to step.  Youngs
   normal, alpha from the Scardovelli-Zaleski volume by bisection.  Walls
   carry no flux (u.n = 0 there).  Planar 2D and 3D. */

/* Fraction of the unit cell's fluid {m.x <= kappa} (volume fraction Cv)
   lying in the slab a <= x_d <= b.  With n = |m|/sum|m| and coordinates
   reflected where m < 0 the fluid is {n.z <= alpha}, V(n, alpha) = Cv; the
   fluid with z_d <= t is t V(n', alpha') for the box scaled by t along d. */
static double plic_below(int dim, const double* n, double alpha, int d, double t) {
  if (t <= 0.0) return 0.0;
  double np[3], s = 0.0;
  for (int e = 0; e < dim; ++e) {
    np[e] = e == d ? n[e] * t : n[e];
    s += np[e];
  }
  if (s <= 0.0) return 0.0;
  for (int e = 0; e < dim; ++e) np[e] /= s;
  return t * plic_vol_pos(dim, np, alpha / s);
}

static double plic_slab(int dim, const double* m, double Cv, int d, double a, double b) {
  if (Cv <= 0.0) return 0.0;
  if (Cv >= 1.0) return b - a;
  double n[3], l2;
  plic_normalise(dim, m, n, &l2);
  if (l2 == 0.0) return Cv * (b - a);     /* no direction: spread uniformly */
  double lo = 0.0, hi = 1.0;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (plic_vol_pos(dim, n, mid) < Cv) lo = mid; else hi = mid;
  }
  double alpha = 0.5 * (lo + hi);
  double ra = a, rb = b;
  if (m[d] < 0.0) { ra = 1.0 - b; rb = 1.0 - a; }
  return plic_below(dim, n, alpha, d, rb) - plic_below(dim, n, alpha, d, ra);
}

void orc_vof_advect(const orc_grid* g, const double* ux, const double* uy,
                    const double* uz, double dt, int order, double* C) {
  size_t N = ncell_of(g);
  int D = ndim_of(g);
  double* H = (double*)malloc(N * sizeof(double));
  for (size_t c = 0; c < N; ++c) H[c] = C[c] > 0.5 ? 1.0 : 0.0;
  const double* U[3] = {ux, uy, uz};
  for (int s = 0; s < D; ++s) {
    int d = order ? D - 1 - s : s;
    size_t nf = nface_of(g, d);
    double* Q = (double*)calloc(nf, sizeof(double));
    int fx = g->nx + (d == 0), fy = g->ny + (d == 1), fz = g->nz + (d == 2);
    for (int k = 0; k < fz; ++k)
      for (int j = 0; j < fy; ++j)
        for (int i = 0; i < fx; ++i) {
          int pos = d == 0 ? i : (d == 1 ? j : k);
          if (pos == 0 || pos == extent(g, d)) continue;   /* walls */
          size_t f = face_idx(g, d, i, j, k);
          double cf = U[d][f] * dt / g->h;
          if (cf == 0.0) continue;
          int li = i, lj = j, lk = k;
          if (d == 0) li--; else if (d == 1) lj--; else lk--;
          int ui = cf > 0 ? li : i, uj = cf > 0 ? lj : j, uk = cf > 0 ? lk : k;
          double m[3];
          youngs_normal(g, C, ui, uj, uk, m);
          double cu = C[idx(g, ui, uj, uk)];
          Q[f] = cf > 0 ? plic_slab(D, m, cu, d, 1.0 - cf, 1.0)
                        : -plic_slab(D, m, cu, d, 0.0, -cf);
        }
    for (int k = 0; k < g->nz; ++k)
      for (int j = 0; j < g->ny; ++j)
        for (int i = 0; i < g->nx; ++i) {
          size_t c = idx(g, i, j, k);
          int pi_ = i + (d == 0), pj = j + (d == 1), pk = k + (d == 2);
          size_t fm = face_idx(g, d, i, j, k), fp = face_idx(g, d, pi_, pj, pk);
          double cm = U[d][fm] * dt / g->h, cp = U[d][fp] * dt / g->h;
          C[c] = C[c] - (Q[fp] - Q[fm]) + H[c] * (cp - cm);
        }
    free(Q);
  }
  free(H);
}
