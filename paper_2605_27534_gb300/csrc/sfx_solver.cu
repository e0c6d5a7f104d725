// Generalised elliptic operator of Sec. 3.1-3.2 (App. A in 3D, App. B in
// axisymmetric form), its red-black Gauss-Seidel multigrid solver, and the
// App. C coupled implicit source step solved by Picard iteration.
//
//   L(a) = div(alpha grad a + beta a) + lambda a,  alpha = -D, beta = -B
//
// written per cell as L(a)_c = (lambda_c - S_d/V_c) a_c - S_n/V_c with the
// face quantity G = D (a_R - a_L)/h + B a_up = cL a_L + cR a_R and
//   S_d = sum_+ A cL - sum_- A cR,   S_n = sum_+ A cR a_+ - sum_- A cL a_-.
// The drift is upwinded on its transport velocity -B (a_up = a_L when
// B < 0); `literal` selects the face value printed in Sec. 3.2 instead.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "sfx_internal.h"
#include "sfx_op64.cuh"

namespace sfx {
namespace {

constexpr int kMaxLevels = 16;

// One colour of a red-black Gauss-Seidel sweep: a_c = (b_c + S_n/V)/(lam - S_d/V)
__global__ void k_rbgs(Level L, Op op, const double* __restrict__ b, double* __restrict__ a,
                       int color) {
  int j = blockIdx.y, k = blockIdx.z;
  int i = 2 * (blockIdx.x * blockDim.x + threadIdx.x) + ((j + k + color) & 1);
  if (i >= L.nx) return;
  double sd, sn;
  flux_terms(L, op, a, i, j, k, sd, sn);
  size_t c = cidx(L, i, j, k);
  double iv = 1.0 / cell_volume(L, i);
  a[c] = (b[c] + sn * iv) / (op.lam[c] - sd * iv);
}

// ---------------------------------------------------------- V-cycle tail
// The coarse levels of a V-cycle are too small to fill the GPU: each of
// their sweeps, restrictions and prolongations would be a launch whose
// cost is its latency.  Every level from the first one with at most
// kTailCells cells down to the coarsest runs in one block instead
// (__syncthreads between phases), with the per-cell arithmetic of the
// multi-launch path (k_rbgs, k_resid_restrict, k_prolong_add): red-black
// updates within a colour are independent, so the result is the same.
// One SM's FP64 pipe bounds a phase: at 4096 cells (64^2) a phase took
// longer in one block than as a launch over the whole GPU (the 512^2
// FP64 vortex step went from 9.4 to 12.3 ms), at 1024 cells the two are
// about even, so the tail starts there.
constexpr int kTailCells = 1024;
constexpr int kMaxTail = 8;

struct TailLevels {
  int n;                  // levels in the tail; T.L[n - 1] is the coarsest
  Level L[kMaxTail];
  Op op[kMaxTail];
  double* a[kMaxTail];    // a[0]: the correction of the tail's first level
  double* b[kMaxTail];    // b[0]: its right-hand side; b[t >= 1] are written
  int nu1, nu2, coarse_sweeps;
};

__device__ void tail_smooth(const Level& L, const Op& op, const double* b, double* a,
                            int sweeps) {
  const int hx = (L.nx + 1) / 2;
  const int nwork = hx * L.ny * L.nz;
  for (int it = 0; it < sweeps; ++it)
    for (int color = 0; color < 2; ++color) {
      for (int w = threadIdx.x; w < nwork; w += blockDim.x) {
        const int ih = w % hx, j = (w / hx) % L.ny, k = w / (hx * L.ny);
        const int i = 2 * ih + ((j + k + color) & 1);
        if (i >= L.nx) continue;
        double sd, sn;
        flux_terms(L, op, a, i, j, k, sd, sn);
        const size_t c = cidx(L, i, j, k);
        const double iv = 1.0 / cell_volume(L, i);
        a[c] = (b[c] + sn * iv) / (op.lam[c] - sd * iv);
      }
      __syncthreads();
    }
}

// The coarsest level's many sweeps: from shared memory when it fits (its
// a, b, lambda and drift faces are staged once; flux_terms reads them
// through the same generic pointers), else from global memory.
constexpr int kSmemCells = 512;
constexpr int kSmemFaces = 768;   // a face array of <= 512 cells, extents >= 2

__device__ void coarsest_sweeps(const Level& L, const Op& op, const double* b, double* a,
                                int sweeps) {
  __shared__ double sa[kSmemCells], sb[kSmemCells], sl[kSmemCells];
  __shared__ double sB[3][kSmemFaces];
  const int n = (int)L.ncell();
  const int nd = L.ndim();
  bool fits = n <= kSmemCells;
  for (int d = 0; d < nd; ++d) fits = fits && (int)L.nface(d) <= kSmemFaces;
  if (!fits) {
    tail_smooth(L, op, b, a, sweeps);
    return;
  }
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    sa[c] = a[c];
    sb[c] = b[c];
    sl[c] = op.lam[c];
  }
  Op so = op;
  so.lam = sl;
  for (int d = 0; d < 3; ++d) {
    if (d >= nd || !op.B[d]) {
      so.B[d] = d < nd ? nullptr : op.B[d];
      continue;
    }
    const int nf = (int)L.nface(d);
    for (int f = threadIdx.x; f < nf; f += blockDim.x) sB[d][f] = op.B[d][f];
    so.B[d] = sB[d];
  }
  __syncthreads();
  tail_smooth(L, so, sb, sa, sweeps);
  for (int c = threadIdx.x; c < n; c += blockDim.x) a[c] = sa[c];
  __syncthreads();
}

__global__ void __launch_bounds__(1024) k_vcycle_tail(TailLevels T) {
  for (int t = 0; t + 1 < T.n; ++t) {
    const Level& Lf = T.L[t];
    const Level& Lc = T.L[t + 1];
    tail_smooth(Lf, T.op[t], T.b[t], T.a[t], T.nu1);
    const int n = (int)Lc.ncell();
    const int kz = Lf.geom == SFX_CART3D ? 2 : 1;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
      const int I = c % Lc.nx, J = (c / Lc.nx) % Lc.ny, K = c / (Lc.nx * Lc.ny);
      double acc = 0.0;
      for (int dk = 0; dk < kz; ++dk)
        for (int dj = 0; dj < 2; ++dj)
          for (int di = 0; di < 2; ++di) {
            const int i = 2 * I + di, j = 2 * J + dj, k = kz == 2 ? 2 * K + dk : 0;
            double sd, sn;
            flux_terms(Lf, T.op[t], T.a[t], i, j, k, sd, sn);
            const size_t f = cidx(Lf, i, j, k);
            const double V = cell_volume(Lf, i);
            acc += V * T.b[t][f] - ((T.op[t].lam[f] * V - sd) * T.a[t][f] - sn);
          }
      T.b[t + 1][c] = acc / cell_volume(Lc, I);
      T.a[t + 1][c] = 0.0;
    }
    __syncthreads();
  }
  const int last = T.n - 1;
  coarsest_sweeps(T.L[last], T.op[last], T.b[last], T.a[last], T.coarse_sweeps);
  for (int t = T.n - 2; t >= 0; --t) {
    const Level& Lc = T.L[t + 1];
    const Level& Lf = T.L[t];
    const bool is3 = Lf.geom == SFX_CART3D;
    const double* ec = T.a[t + 1];
    const int n = (int)Lf.ncell();
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
      const int i = c % Lf.nx, j = (c / Lf.nx) % Lf.ny, k = c / (Lf.nx * Lf.ny);
      const int I = i >> 1, J = j >> 1, K = k >> 1;
      const int I2 = min(max(I + ((i & 1) ? 1 : -1), 0), Lc.nx - 1);
      const int J2 = min(max(J + ((j & 1) ? 1 : -1), 0), Lc.ny - 1);
      double v;
      if (!is3) {
        v = 0.5625 * ec[cidx(Lc, I, J, 0)] + 0.1875 * ec[cidx(Lc, I2, J, 0)] +
            0.1875 * ec[cidx(Lc, I, J2, 0)] + 0.0625 * ec[cidx(Lc, I2, J2, 0)];
      } else {
        const int K2 = min(max(K + ((k & 1) ? 1 : -1), 0), Lc.nz - 1);
        v = 0.421875 * ec[cidx(Lc, I, J, K)] +
            0.140625 * (ec[cidx(Lc, I2, J, K)] + ec[cidx(Lc, I, J2, K)] + ec[cidx(Lc, I, J, K2)]) +
            0.046875 * (ec[cidx(Lc, I2, J2, K)] + ec[cidx(Lc, I2, J, K2)] + ec[cidx(Lc, I, J2, K2)]) +
            0.015625 * ec[cidx(Lc, I2, J2, K2)];
      }
      T.a[t][c] += v;
    }
    __syncthreads();
    tail_smooth(Lf, T.op[t], T.b[t], T.a[t], T.nu2);
  }
}

// Coarsest level alone: all sweeps inside one block.
__global__ void __launch_bounds__(1024) k_coarse_solve(Level L, Op op, const double* __restrict__ b,
                                                       double* a, int sweeps) {
  coarsest_sweeps(L, op, b, a, sweeps);
}

// Volume-weighted restriction of the residual b - L(a) to the coarse grid.
__global__ void k_resid_restrict(Level Lf, Level Lc, Op op, const double* __restrict__ b,
                                 const double* __restrict__ a, double* __restrict__ rc) {
  size_t n = Lc.ncell();
  int kz = Lf.geom == SFX_CART3D ? 2 : 1;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x) {
    int I = (int)(c % Lc.nx), J = (int)((c / Lc.nx) % Lc.ny), K = (int)(c / ((size_t)Lc.nx * Lc.ny));
    double acc = 0.0;
    for (int dk = 0; dk < kz; ++dk)
      for (int dj = 0; dj < 2; ++dj)
        for (int di = 0; di < 2; ++di) {
          int i = 2 * I + di, j = 2 * J + dj, k = kz == 2 ? 2 * K + dk : 0;
          double sd, sn;
          flux_terms(Lf, op, a, i, j, k, sd, sn);
          size_t f = cidx(Lf, i, j, k);
          double V = cell_volume(Lf, i);
          acc += V * b[f] - ((op.lam[f] * V - sd) * a[f] - sn);
        }
    rc[c] = acc / cell_volume(Lc, I);
  }
}

// Volume-weighted restriction of a cell coefficient.
__global__ void k_restrict_cells(Level Lf, Level Lc, const double* __restrict__ xf,
                                 double* __restrict__ xc) {
  size_t n = Lc.ncell();
  int kz = Lf.geom == SFX_CART3D ? 2 : 1;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x) {
    int I = (int)(c % Lc.nx), J = (int)((c / Lc.nx) % Lc.ny), K = (int)(c / ((size_t)Lc.nx * Lc.ny));
    double acc = 0.0;
    for (int dk = 0; dk < kz; ++dk)
      for (int dj = 0; dj < 2; ++dj)
        for (int di = 0; di < 2; ++di) {
          int i = 2 * I + di, j = 2 * J + dj, k = kz == 2 ? 2 * K + dk : 0;
          acc += cell_volume(Lf, i) * xf[cidx(Lf, i, j, k)];
        }
    xc[c] = acc / cell_volume(Lc, I);
  }
}

// Area-weighted restriction of face drifts in direction d.
__global__ void k_restrict_faces(Level Lf, Level Lc, int d, const double* __restrict__ Bf,
                                 double* __restrict__ Bc) {
  size_t n = Lc.nface(d);
  int fx = Lc.nx + (d == 0), fy = Lc.ny + (d == 1);
  bool is3 = Lf.geom == SFX_CART3D;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n;
       q += (size_t)gridDim.x * blockDim.x) {
    int I = (int)(q % fx), J = (int)((q / fx) % fy), K = (int)(q / ((size_t)fx * fy));
    int pos = d == 0 ? I : (d == 1 ? J : K);
    if (pos == 0 || pos == Lc.extent(d)) { Bc[q] = 0.0; continue; }
    double num = 0.0, den = 0.0;
    // the 2 (2D) or 4 (3D) fine faces covering this coarse face
    for (int t1 = 0; t1 < 2; ++t1)
      for (int t2 = 0; t2 < (is3 ? 2 : 1); ++t2) {
        int i = 2 * I, j = 2 * J, k = is3 ? 2 * K : 0;
        if (d == 0) { j += t1; k += t2; }
        else if (d == 1) { i += t1; k += t2; }
        else { i += t1; j += t2; }
        double A = face_area(Lf, d, i);
        num += A * Bf[fidx(Lf, d, i, j, k)];
        den += A;
      }
    Bc[q] = num / den;
  }
}

// a_fine += bilinear / trilinear interpolation of the coarse correction
// (weights 3/4 parent, 1/4 neighbour per direction; mirrored at walls).
__global__ void k_prolong_add(Level Lc, Level Lf, const double* __restrict__ ec,
                              double* __restrict__ af) {
  size_t n = Lf.ncell();
  bool is3 = Lf.geom == SFX_CART3D;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(c % Lf.nx), j = (int)((c / Lf.nx) % Lf.ny), k = (int)(c / ((size_t)Lf.nx * Lf.ny));
    int I = i >> 1, J = j >> 1, K = k >> 1;
    int I2 = min(max(I + ((i & 1) ? 1 : -1), 0), Lc.nx - 1);
    int J2 = min(max(J + ((j & 1) ? 1 : -1), 0), Lc.ny - 1);
    double v;
    if (!is3) {
      v = 0.5625 * ec[cidx(Lc, I, J, 0)] + 0.1875 * ec[cidx(Lc, I2, J, 0)] +
          0.1875 * ec[cidx(Lc, I, J2, 0)] + 0.0625 * ec[cidx(Lc, I2, J2, 0)];
    } else {
      int K2 = min(max(K + ((k & 1) ? 1 : -1), 0), Lc.nz - 1);
      v = 0.421875 * ec[cidx(Lc, I, J, K)] +
          0.140625 * (ec[cidx(Lc, I2, J, K)] + ec[cidx(Lc, I, J2, K)] + ec[cidx(Lc, I, J, K2)]) +
          0.046875 * (ec[cidx(Lc, I2, J2, K)] + ec[cidx(Lc, I2, J, K2)] + ec[cidx(Lc, I, J2, K2)]) +
          0.015625 * ec[cidx(Lc, I2, J2, K2)];
    }
    af[c] += v;
  }
}

// |b - L(a)|_inf and |b|_inf into norms[slot], norms[slot+1]; NaN -> flag.
__global__ void k_resid_norm(Level L, Op op, const double* __restrict__ b,
                             const double* __restrict__ a, unsigned long long* norms, int slot,
                             int* flag) {
  size_t n = L.ncell();
  double rmax = 0.0, bmax = 0.0;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(c % L.nx), j = (int)((c / L.nx) % L.ny), k = (int)(c / ((size_t)L.nx * L.ny));
    double sd, sn;
    flux_terms(L, op, a, i, j, k, sd, sn);
    double iv = 1.0 / cell_volume(L, i);
    double r = b[c] - ((op.lam[c] - sd * iv) * a[c] - sn * iv);
    if (!isfinite(r)) { atomicOr(flag, 1); r = 0.0; }
    rmax = fmax(rmax, fabs(r));
    bmax = fmax(bmax, fabs(b[c]));
  }
  rmax = warp_max(rmax);
  bmax = warp_max(bmax);
  if ((threadIdx.x & 31) == 0) {
    atomic_max_nonneg(&norms[slot], rmax);
    atomic_max_nonneg(&norms[slot + 1], bmax);
  }
}

// ------------------------------------------------------------ App. C terms
struct Kin {
  double ka, kd, ginf, eps, eta, inv_dt;
};

// f problem: lambda_f = 1/dt + r_d + r_a F/(phi+eta),
//            b_f = f_star/dt + r_a F/(phi+eta) Gamma_inf phi(1-phi)/eps
template <typename P>
__global__ void k_setup_f(size_t n, Kin q, const P* __restrict__ phi, const double* __restrict__ F,
                          const double* __restrict__ fstar, double* __restrict__ lam,
                          double* __restrict__ b) {
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x) {
    double p = (double)phi[c];
    double Fs = F[c] / (p + q.eta);
    lam[c] = q.inv_dt + q.kd + q.ka * Fs;
    b[c] = fstar[c] * q.inv_dt + q.ka * Fs * (q.ginf * p * (1.0 - p) / q.eps);
  }
}

// F problem: lambda_F = 1/dt + r_a (f_inf - f)/(phi+eta), b_F = F_star/dt + r_d f
template <typename P>
__global__ void k_setup_F(size_t n, Kin q, const P* __restrict__ phi, const double* __restrict__ f,
                          const double* __restrict__ Fstar, double* __restrict__ lam,
                          double* __restrict__ b) {
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x) {
    double p = (double)phi[c];
    double finf = q.ginf * p * (1.0 - p) / q.eps;
    lam[c] = q.inv_dt + q.ka * (finf - f[c]) / (p + q.eta);
    b[c] = Fstar[c] * q.inv_dt + q.kd * f[c];
  }
}

// Both nonlinear residuals of App. C at the current (f, F):
// norms[0..3] = |r_f|, |b_f|, |r_F|, |b_F| (infinity norms).
template <typename P>
__global__ void k_coupled_resid(Level L, Kin q, Op opf, Op opF, const P* __restrict__ phi,
                                const double* __restrict__ f, const double* __restrict__ F,
                                const double* __restrict__ fstar,
                                const double* __restrict__ Fstar, unsigned long long* norms,
                                int* flag) {
  size_t n = L.ncell();
  double m[4] = {0, 0, 0, 0};
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(c % L.nx), j = (int)((c / L.nx) % L.ny), k = (int)(c / ((size_t)L.nx * L.ny));
    double p = (double)phi[c];
    double pe = p + q.eta, finf = q.ginf * p * (1.0 - p) / q.eps;
    double iv = 1.0 / cell_volume(L, i);
    double sd, sn;
    // f residual with the current F
    double Fs = F[c] / pe;
    double lam = q.inv_dt + q.kd + q.ka * Fs;
    double b = fstar[c] * q.inv_dt + q.ka * Fs * finf;
    flux_terms(L, opf, f, i, j, k, sd, sn);
    double r = b - ((lam - sd * iv) * f[c] - sn * iv);
    if (!isfinite(r)) { atomicOr(flag, 1); r = 0.0; }
    m[0] = fmax(m[0], fabs(r));
    m[1] = fmax(m[1], fabs(b));
    // F residual with the current f
    lam = q.inv_dt + q.ka * (finf - f[c]) / pe;
    b = Fstar[c] * q.inv_dt + q.kd * f[c];
    flux_terms(L, opF, F, i, j, k, sd, sn);
    r = b - ((lam - sd * iv) * F[c] - sn * iv);
    if (!isfinite(r)) { atomicOr(flag, 1); r = 0.0; }
    m[2] = fmax(m[2], fabs(r));
    m[3] = fmax(m[3], fabs(b));
  }
  for (int s = 0; s < 4; ++s) {
    double v = warp_max(m[s]);
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(&norms[s], v);
  }
}

// Face drifts of both problems in direction d (App. C):
//   B_f = -Df 2(0.5 - phi)/eps n,  B_F = -DF (1 - phi)/eps n,
// face value = mean of the two adjacent cell values; walls 0.
template <typename P>
__global__ void k_drift_faces(Level L, int d, const P* __restrict__ phi, double Df, double DF,
                              double eps, double* __restrict__ Bf, double* __restrict__ BF) {
  size_t n = L.nface(d);
  int fx = L.nx + (d == 0), fy = L.ny + (d == 1);
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n;
       q += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(q % fx), j = (int)((q / fx) % fy), k = (int)(q / ((size_t)fx * fy));
    int pos = d == 0 ? i : (d == 1 ? j : k);
    if (pos == 0 || pos == L.extent(d)) { Bf[q] = 0.0; BF[q] = 0.0; continue; }
    int li = i - (d == 0), lj = j - (d == 1), lk = k - (d == 2);
    double pL = (double)phi[cidx(L, li, lj, lk)], pR = (double)phi[cidx(L, i, j, k)];
    double nL = normal_comp(L, phi, li, lj, lk, d, eps), nR = normal_comp(L, phi, i, j, k, d, eps);
    Bf[q] = 0.5 * ((-Df * 2.0 * (0.5 - pL) / eps) * nL + (-Df * 2.0 * (0.5 - pR) / eps) * nR);
    BF[q] = 0.5 * ((-DF * (1.0 - pL) / eps) * nL + (-DF * (1.0 - pR) / eps) * nR);
  }
}

__global__ void k_zero(size_t n, double* x) {
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x)
    x[c] = 0.0;
}

// ------------------------------------------------------------- host side
struct Hier {
  int nlev;
  double D;
  int literal;
  const double* B[kMaxLevels][3];
  const double* lam[kMaxLevels];
};

Op op_at(const Hier& H, int l) {
  Op o;
  o.D = H.D;
  o.literal = H.literal;
  for (int d = 0; d < 3; ++d) o.B[d] = H.B[l][d];
  o.lam = H.lam[l];
  return o;
}

sfx_status smooth(sfx_ctx* c, int kind, const Level& L, const Op& op, const double* b, double* a,
                  int sweeps, cudaStream_t s) {
  dim3 blk(128), grd((unsigned)(((L.nx + 1) / 2 + 127) / 128), (unsigned)L.ny, (unsigned)L.nz);
  for (int it = 0; it < sweeps; ++it)
    for (int color = 0; color < 2; ++color)
      SFX_KERNEL(c, kind, k_rbgs, grd, blk, s, L, op, b, a, color);
  SFX_LAUNCH_CHECK();
  return SFX_OK;
}

sfx_status coarse_solve(sfx_ctx* c, const Level& L, const Op& op, const double* b, double* a,
                        int sweeps, cudaStream_t s) {
  if (L.ncell() <= 8192) {
    SFX_KERNEL(c, K_SMOOTH_COARSE, k_coarse_solve, 1, 1024, s, L, op, b, a, sweeps);
    SFX_LAUNCH_CHECK();
    return SFX_OK;
  }
  return smooth(c, K_SMOOTH_COARSE, L, op, b, a, sweeps, s);
}

sfx_status vcycle(sfx_ctx* c, const Hier& H, int l, double* a, const double* b,
                  const sfx_solve_opts* o, cudaStream_t s) {
  const Level& L = c->lev[l].lv;
  Op op = op_at(H, l);
  if (l >= 1 && l < H.nlev - 1 && L.ncell() <= (size_t)kTailCells && H.nlev - l <= kMaxTail) {
    // this level and every coarser one in one block
    TailLevels T{};
    T.n = H.nlev - l;
    for (int t = 0; t < T.n; ++t) {
      T.L[t] = c->lev[l + t].lv;
      T.op[t] = op_at(H, l + t);
      T.a[t] = t == 0 ? a : c->lev[l + t].a;
      T.b[t] = t == 0 ? const_cast<double*>(b) : c->lev[l + t].b;
    }
    T.nu1 = o->nu1;
    T.nu2 = o->nu2;
    T.coarse_sweeps = o->coarse_sweeps;
    SFX_KERNEL(c, K_SMOOTH_COARSE, k_vcycle_tail, 1, 1024, s, T);
    SFX_LAUNCH_CHECK();
    return SFX_OK;
  }
  if (l == H.nlev - 1) return coarse_solve(c, L, op, b, a, o->coarse_sweeps, s);
  const int kind = l == 0 ? K_SMOOTH_FINE : K_SMOOTH_COARSE;
  sfx_status st = smooth(c, kind, L, op, b, a, o->nu1, s);
  if (st != SFX_OK) return st;
  LevelData& C = c->lev[l + 1];
  const Level& Lc = C.lv;
  SFX_KERNEL(c, K_RESTRICT, k_resid_restrict, blocks_for(Lc.ncell(), 256), 256, s, L, Lc, op, b, a, C.b);
  SFX_KERNEL(c, K_OTHER, k_zero, blocks_for(Lc.ncell(), 256), 256, s, Lc.ncell(), C.a);
  SFX_LAUNCH_CHECK();
  st = vcycle(c, H, l + 1, C.a, C.b, o, s);
  if (st != SFX_OK) return st;
  SFX_KERNEL(c, K_PROLONG, k_prolong_add, blocks_for(L.ncell(), 256), 256, s, Lc, L, C.a, a);
  SFX_LAUNCH_CHECK();
  return smooth(c, kind, L, op, b, a, o->nu2, s);
}

int levels_to_use(sfx_ctx* c, const sfx_solve_opts* o) {
  int built = (int)c->lev.size();
  if (o->mg_levels <= 0) return built;
  return std::min(o->mg_levels, built);
}

sfx_status restrict_lambda(sfx_ctx* c, int nlev, cudaStream_t s) {
  for (int l = 1; l < nlev; ++l) {
    const Level& Lf = c->lev[l - 1].lv;
    const Level& Lc = c->lev[l].lv;
    SFX_KERNEL(c, K_SETUP, k_restrict_cells, blocks_for(Lc.ncell(), 256), 256, s, Lf, Lc, c->lev[l - 1].lam,
                                                                 c->lev[l].lam);
  }
  SFX_LAUNCH_CHECK();
  return SFX_OK;
}

sfx_status read_norms(sfx_ctx* c, cudaStream_t s, double* out4, bool* nonfinite) {
  // slots 0..3: norms; slot 7 holds the non-finite flag (d_flag aliases it)
  SFX_CUDA(cudaMemcpyAsync(c->h_norms, c->d_norms, 8 * sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, s));
  SFX_CUDA(cudaStreamSynchronize(s));
  for (int i = 0; i < 4; ++i) {
    unsigned long long u = c->h_norms[i];
    double v;
    memcpy(&v, &u, sizeof(double));
    out4[i] = v;
  }
  int hflag = 0;
  memcpy(&hflag, &c->h_norms[7], sizeof(int));
  *nonfinite = hflag != 0;
  return SFX_OK;
}

sfx_status clear_norms(sfx_ctx* c, cudaStream_t s) {
  SFX_CUDA(cudaMemsetAsync(c->d_norms, 0, 8 * sizeof(unsigned long long), s));
  return SFX_OK;
}

double rel(double r, double b) { return r / (b > 1e-300 ? b : 1e-300); }

template <typename P>
sfx_status step_impl(sfx_ctx* c, const sfx_params* p, const P* phi, const void* ux,
                     const void* uy, const void* uz, double* f, double* F, double dt,
                     const sfx_solve_opts* o, sfx_step_stats* stats, cudaStream_t s) {
  const Level& L = c->lev[0].lv;
  const size_t n = L.ncell();
  const int nlev = levels_to_use(c, o);
  const int nd = L.ndim();
  // drift faces of both problems at every level (phi is fixed over the step)
  for (int d = 0; d < nd; ++d)
    SFX_KERNEL(c, K_SETUP, k_drift_faces<P>, blocks_for(L.nface(d), 256), 256, s, 
        L, d, phi, p->Df, p->DF, p->eps, c->lev[0].B[0][d], c->lev[0].B[1][d]);
  for (int l = 1; l < nlev; ++l)
    for (int fld = 0; fld < 2; ++fld)
      for (int d = 0; d < nd; ++d)
        SFX_KERNEL(c, K_SETUP, k_restrict_faces, blocks_for(c->lev[l].lv.nface(d), 256), 256, s, 
            c->lev[l - 1].lv, c->lev[l].lv, d, c->lev[l - 1].B[fld][d], c->lev[l].B[fld][d]);
  SFX_LAUNCH_CHECK();
  // a3: explicit advection, then start the implicit solve from (f*, F*)
  if (ux) {
    sfx_status st = advect(c, ux, uy, uz, dt, f, p->bc_f, c->fstar, s);
    if (st != SFX_OK) return st;
    st = advect(c, ux, uy, uz, dt, F, p->bc_F, c->Fstar, s);
    if (st != SFX_OK) return st;
    SFX_CUDA(cudaMemcpyAsync(f, c->fstar, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    SFX_CUDA(cudaMemcpyAsync(F, c->Fstar, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  } else {
    SFX_CUDA(cudaMemcpyAsync(c->fstar, f, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    SFX_CUDA(cudaMemcpyAsync(c->Fstar, F, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  Kin q{p->ka, p->kd, p->gamma_inf, p->eps, p->eta, 1.0 / dt};
  Hier Hf{}, HF{};
  Hf.nlev = HF.nlev = nlev;
  Hf.D = p->Df;
  HF.D = p->DF;
  Hf.literal = HF.literal = p->literal_upwind;
  for (int l = 0; l < nlev; ++l) {
    for (int d = 0; d < 3; ++d) {
      Hf.B[l][d] = d < nd ? c->lev[l].B[0][d] : nullptr;
      HF.B[l][d] = d < nd ? c->lev[l].B[1][d] : nullptr;
    }
    Hf.lam[l] = HF.lam[l] = c->lev[l].lam;
  }
  double* lam0 = c->lev[0].lam;
  double* b0 = c->lev[0].b;
  int it = 0, cycles = 0;
  bool conv = false;
  double nrm[4] = {0, 0, 0, 0};
  const int nb = blocks_for(n, 256);
  for (it = 1; it <= o->max_cycles; ++it) {
    SFX_KERNEL(c, K_SETUP, k_setup_f<P>, nb, 256, s, n, q, phi, F, c->fstar, lam0, b0);
    SFX_LAUNCH_CHECK();
    sfx_status st = restrict_lambda(c, nlev, s);
    if (st != SFX_OK) return st;
    for (int v = 0; v < o->vcycles; ++v) {
      st = vcycle(c, Hf, 0, f, b0, o, s);
      if (st != SFX_OK) return st;
      ++cycles;
    }
    SFX_KERNEL(c, K_SETUP, k_setup_F<P>, nb, 256, s, n, q, phi, f, c->Fstar, lam0, b0);
    SFX_LAUNCH_CHECK();
    st = restrict_lambda(c, nlev, s);
    if (st != SFX_OK) return st;
    for (int v = 0; v < o->vcycles; ++v) {
      st = vcycle(c, HF, 0, F, b0, o, s);
      if (st != SFX_OK) return st;
      ++cycles;
    }
    if (it % o->check_every == 0 || it == o->max_cycles) {
      st = clear_norms(c, s);
      if (st != SFX_OK) return st;
      SFX_KERNEL(c, K_RESIDUAL, k_coupled_resid<P>, blocks_for(n, 256), 256, s, L, q, op_at(Hf, 0), op_at(HF, 0), phi,
                                                            f, F, c->fstar, c->Fstar, c->d_norms,
                                                            c->d_flag);
      SFX_LAUNCH_CHECK();
      bool bad = false;
      st = read_norms(c, s, nrm, &bad);
      if (st != SFX_OK) return st;
      if (bad) {
        if (stats) stats->converged = 0;
        return SFX_ERR_NONFINITE;
      }
      if (rel(nrm[0], nrm[1]) <= o->tol && rel(nrm[2], nrm[3]) <= o->tol) {
        conv = true;
        break;
      }
    }
  }
  if (stats) {
    stats->picard = std::min(it, o->max_cycles);
    stats->vcycles = cycles;
    stats->res_f = rel(nrm[0], nrm[1]);
    stats->res_F = rel(nrm[2], nrm[3]);
    stats->converged = conv ? 1 : 0;
    const double* fl[2] = {f, F};
    double m[2];
    sfx_status st = totals(c, fl, 2, m, s);
    if (st != SFX_OK) return st;
    stats->mass_f = m[0];
    stats->mass_F = m[1];
  }
  return conv ? SFX_OK : SFX_ERR_NOT_CONVERGED;
}

}  // namespace

sfx_status drift_faces64(sfx_ctx* c, const double* phi, double Df, double DF, double eps,
                         double* const* Bf, double* const* BF, cudaStream_t s) {
  const Level& L = c->lev[0].lv;
  for (int d = 0; d < L.ndim(); ++d)
    SFX_KERNEL(c, K_SETUP, k_drift_faces<double>, blocks_for(L.nface(d), 256), 256, s, L, d, phi,
               Df, DF, eps, Bf[d], BF[d]);
  SFX_LAUNCH_CHECK();
  return SFX_OK;
}

sfx_status surfactant_step(sfx_ctx* c, const sfx_params* p, const void* phi, const void* ux,
                           const void* uy, const void* uz, double* f, double* F, double dt,
                           const sfx_solve_opts* o, sfx_step_stats* st, cudaStream_t s) {
  if (c->prec == SFX_F64)
    return step_impl<double>(c, p, (const double*)phi, ux, uy, uz, f, F, dt, o, st, s);
  return step_impl<float>(c, p, (const float*)phi, ux, uy, uz, f, F, dt, o, st, s);
}

sfx_status mg_solve(sfx_ctx* c, double D, const double* Bx, const double* By, const double* Bz,
                    int literal, const double* lam, const double* b, double* a,
                    const sfx_solve_opts* o, int* cycles_out, double* res_out, cudaStream_t s) {
  const int nlev = levels_to_use(c, o);
  const int nd = c->lev[0].lv.ndim();
  const double* Bin[3] = {Bx, By, nd == 3 ? Bz : nullptr};
  Hier H{};
  H.nlev = nlev;
  H.D = D;
  H.literal = literal;
  for (int d = 0; d < 3; ++d) H.B[0][d] = Bin[d];
  H.lam[0] = lam;
  // coarse coefficients: restrict lambda and the face drifts
  for (int l = 1; l < nlev; ++l) {
    const Level& Lf = c->lev[l - 1].lv;
    const Level& Lc = c->lev[l].lv;
    SFX_KERNEL(c, K_SETUP, k_restrict_cells, blocks_for(Lc.ncell(), 256), 256, s, Lf, Lc, H.lam[l - 1],
                                                                 c->lev[l].lam);
    H.lam[l] = c->lev[l].lam;
    for (int d = 0; d < 3; ++d) {
      if (H.B[l - 1][d] == nullptr) { H.B[l][d] = nullptr; continue; }
      SFX_KERNEL(c, K_SETUP, k_restrict_faces, blocks_for(Lc.nface(d), 256), 256, s, Lf, Lc, d, H.B[l - 1][d],
                                                                    c->lev[l].Bg[d]);
      H.B[l][d] = c->lev[l].Bg[d];
    }
  }
  SFX_LAUNCH_CHECK();
  const Level& L = c->lev[0].lv;
  int cyc = 0;
  double nrm[4] = {0, 0, 0, 0};
  bool conv = false;
  for (cyc = 0; cyc <= o->max_cycles; ++cyc) {
    if (cyc % o->check_every == 0 || cyc == o->max_cycles) {
      sfx_status st = clear_norms(c, s);
      if (st != SFX_OK) return st;
      SFX_KERNEL(c, K_RESIDUAL, k_resid_norm, blocks_for(L.ncell(), 256), 256, s, L, op_at(H, 0), b, a, c->d_norms, 0,
                                                              c->d_flag);
      SFX_LAUNCH_CHECK();
      bool bad = false;
      st = read_norms(c, s, nrm, &bad);
      if (st != SFX_OK) return st;
      if (bad) return SFX_ERR_NONFINITE;
      if (rel(nrm[0], nrm[1]) <= o->tol) { conv = true; break; }
    }
    if (cyc == o->max_cycles) break;
    sfx_status st = vcycle(c, H, 0, a, b, o, s);
    if (st != SFX_OK) return st;
  }
  if (cycles_out) *cycles_out = cyc;
  if (res_out) *res_out = rel(nrm[0], nrm[1]);
  return conv ? SFX_OK : SFX_ERR_NOT_CONVERGED;
}

}  // namespace sfx
