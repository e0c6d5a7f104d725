// PLIC geometry in a unit cell (FP64): the Scardovelli-Zaleski volume below
// a plane, its slope (interface area), the plane offset for a given volume,
// the fluid volume in a slab of the cell (geometric VoF fluxes), and the
// Youngs normal of a volume-fraction field.
#pragma once

#include "sfx_common.cuh"

namespace sfx {

// ------------------------------------------------------------- PLIC area
// Fraction of the unit cube below the plane m.x = a (m >= 0, sum m = 1;
// Scardovelli & Zaleski 2000) and its slope dV/da.  The cubic is expanded
// per region so that near-zero components cost no precision; V(a) =
// 1 - V(1 - a) folds a into [0, 1/2].  `q` holds the components in
// ascending order (q[0] = 0 in 2D).
struct VolSlope {
  double v, dv;
};

__device__ inline VolSlope plic_lower_half(const double* q, bool three_d, double a) {
  VolSlope r{0.0, 0.0};
  if (a <= 0.0) return r;
  if (!three_d) {
    const double lo = q[1], hi = q[2];
    if (a < lo) {
      r.v = 0.5 * a * a / (lo * hi);
      r.dv = a / (lo * hi);
    } else {
      r.v = (a - 0.5 * lo) / hi;
      r.dv = 1.0 / hi;
    }
    return r;
  }
  const double p = q[0], s = q[1], t = q[2];
  const double inv_st = 1.0 / (s * t);
  if (a < p) {
    r.v = a * a * a * inv_st / (6.0 * p);
    r.dv = 0.5 * a * a * inv_st / p;
  } else if (a < s) {
    r.v = 0.5 * (a * (a - p) + p * p / 3.0) * inv_st;
    r.dv = (a - 0.5 * p) * inv_st;
  } else if (t >= p + s) {
    if (a < p + s) {
      double u = a - s;
      r.v = (a * a - a * p + p * p / 3.0) * 0.5 * inv_st - u * u * u * inv_st / (6.0 * p);
      r.dv = (a - 0.5 * p) * inv_st - 0.5 * u * u * inv_st / p;
    } else {
      r.v = (a - 0.5 * (p + s)) / t;
      r.dv = 1.0 / t;
    }
  } else {
    double u = a - s, w = fmax(a - t, 0.0);
    r.v = (a * a - a * p + p * p / 3.0) * 0.5 * inv_st - (u * u * u + w * w * w) * inv_st / (6.0 * p);
    r.dv = (a - 0.5 * p) * inv_st - 0.5 * (u * u + w * w) * inv_st / p;
  }
  return r;
}

__device__ inline VolSlope plic_volume(const double* q, bool three_d, double a) {
  if (a <= 0.0) return VolSlope{0.0, 0.0};
  if (a >= 1.0) return VolSlope{1.0, 0.0};
  if (a <= 0.5) return plic_lower_half(q, three_d, a);
  VolSlope r = plic_lower_half(q, three_d, 1.0 - a);
  r.v = 1.0 - r.v;
  return r;
}

// Plane offset alpha in [0, 1] with volume fraction C: the root of the
// increasing V(alpha) - C by Newton steps on the slope dV/dalpha, kept
// inside a bracket that every evaluation narrows (a bisection step replaces
// a Newton step that leaves it); stops when the step falls below 1e-17, the
// bracket closes, or after 100 evaluations.  The same root as a bisection
// to double precision, in a handful of evaluations.
__device__ inline double plic_alpha(const double* q, bool three_d, double C) {
  double lo = 0.0, hi = 1.0, a = C;
  for (int it = 0; it < 100; ++it) {
    const VolSlope r = plic_volume(q, three_d, a);
    const double f = r.v - C;
    if (f == 0.0) return a;
    if (f < 0.0) lo = a;
    else hi = a;
    double an = r.dv > 0.0 ? a - f / r.dv : 0.5 * (lo + hi);
    if (!(an > lo && an < hi)) an = 0.5 * (lo + hi);
    if (fabs(an - a) <= 1e-17 || !(hi - lo > 0.0)) return an;
    a = an;
  }
  return a;
}

// Interface area inside the unit cell holding fraction C with normal m.
__device__ inline double plic_unit_area(int nd, const double* mraw, double C) {
  if (!(C > 0.0 && C < 1.0)) return 0.0;
  double s = 0.0, q2 = 0.0;
  for (int d = 0; d < nd; ++d) { s += fabs(mraw[d]); q2 += mraw[d] * mraw[d]; }
  if (s == 0.0) return 0.0;
  double q[3] = {0.0, fabs(mraw[0]) / s, fabs(mraw[1]) / s};
  if (nd == 3) q[0] = fabs(mraw[2]) / s;
  // ascending order
  if (q[0] > q[1]) { double t = q[0]; q[0] = q[1]; q[1] = t; }
  if (q[1] > q[2]) { double t = q[1]; q[1] = q[2]; q[2] = t; }
  if (q[0] > q[1]) { double t = q[0]; q[0] = q[1]; q[1] = t; }
  const bool three_d = nd == 3;
  return (sqrt(q2) / s) * plic_volume(q, three_d, plic_alpha(q, three_d, C)).dv;
}


// Components |m|/sum|m| in ascending order (q[0] = 0 in 2D); false when m = 0.
__device__ inline bool plic_sorted(int nd, const double* m, double* q) {
  double s = 0.0;
  for (int d = 0; d < nd; ++d) s += fabs(m[d]);
  if (s == 0.0) return false;
  q[0] = nd == 3 ? fabs(m[2]) / s : 0.0;
  q[1] = fabs(m[0]) / s;
  q[2] = fabs(m[1]) / s;
  if (q[0] > q[1]) { double t = q[0]; q[0] = q[1]; q[1] = t; }
  if (q[1] > q[2]) { double t = q[1]; q[1] = q[2]; q[2] = t; }
  if (q[0] > q[1]) { double t = q[0]; q[0] = q[1]; q[1] = t; }
  return true;
}

// Fluid {n.z <= alpha} (n = |m|/sum|m|, z reflected where m < 0) with
// z_d <= t: t times the volume of the box scaled by t along d.
__device__ inline double plic_below(int nd, const double* n, double alpha, int d, double t) {
  if (t <= 0.0) return 0.0;
  double np[3] = {0.0, 0.0, 0.0}, s = 0.0;
  for (int e = 0; e < nd; ++e) {
    np[e] = e == d ? n[e] * t : n[e];
    s += np[e];
  }
  if (s <= 0.0) return 0.0;
  double q[3];
  if (!plic_sorted(nd, np, q)) return 0.0;
  return t * plic_volume(q, nd == 3, alpha / s).v;
}

// Volume fraction of the unit cell (fluid fraction C, normal m pointing out
// of the fluid) that lies in the slab a <= x_d <= b.
__device__ inline double plic_slab(int nd, const double* m, double C, int d, double a, double b) {
  if (C <= 0.0) return 0.0;
  if (C >= 1.0) return b - a;
  double q[3];
  if (!plic_sorted(nd, m, q)) return C * (b - a);   // no direction: uniform
  const double alpha = plic_alpha(q, nd == 3, C);
  double s = 0.0, n[3] = {0.0, 0.0, 0.0};
  for (int e = 0; e < nd; ++e) s += fabs(m[e]);
  for (int e = 0; e < nd; ++e) n[e] = fabs(m[e]) / s;
  double ra = a, rb = b;
  if (m[d] < 0.0) {
    ra = 1.0 - b;
    rb = 1.0 - a;
  }
  return plic_below(nd, n, alpha, d, rb) - plic_below(nd, n, alpha, d, ra);
}

// Youngs normal: minus the (1,2,1)-weighted gradient of C over the
// 3x3(x3) block around (i,j,k), zero-gradient walls.
__device__ inline void youngs_normal(const Level& L, const double* __restrict__ C, int i, int j,
                                     int k, double* m) {
  const int nd = L.ndim();
  m[0] = m[1] = m[2] = 0.0;
  const int kr = nd == 3 ? 1 : 0;
  for (int dk = -kr; dk <= kr; ++dk)
    for (int dj = -1; dj <= 1; ++dj)
      for (int di = -1; di <= 1; ++di) {
        const int a = min(max(i + di, 0), L.nx - 1);
        const int b = min(max(j + dj, 0), L.ny - 1);
        const int e = min(max(k + dk, 0), L.nz - 1);
        const double w = (di == 0 ? 2.0 : 1.0) * (dj == 0 ? 2.0 : 1.0) *
                         (nd == 3 ? (dk == 0 ? 2.0 : 1.0) : 1.0);
        const double v = C[cidx(L, a, b, e)];
        m[0] -= w * di * v;
        m[1] -= w * dj * v;
        m[2] -= w * dk * v;
      }
}

}  // namespace sfx
