// PLIC geometry in a unit cell: the Scardovelli-Zaleski volume below a
// plane, its slope (interface area), the plane offset for a given volume,
// the fluid volume in a slab of the cell (geometric VoF fluxes), and the
// Youngs normal of a volume-fraction field.  Templated on the arithmetic
// type T: double for SFX_F64 contexts and the FP64 force, float for the
// geometry of SFX_F32 contexts (the FP64 pipe of the GPU runs at a small
// fraction of the FP32 rate, and a plane offset costs tens of operations).
#pragma once

#include "sfx_common.cuh"

namespace sfx {

template <typename T>
struct PlicTraits;
template <>
struct PlicTraits<double> {
  static constexpr double step_tol = 1e-17;   // below the resolution of alpha in [0, 1]
};
template <>
struct PlicTraits<float> {
  static constexpr float step_tol = 1e-8f;
};

// ------------------------------------------------------------- PLIC area
// Fraction of the unit cube below the plane m.x = a (m >= 0, sum m = 1;
// Scardovelli & Zaleski 2000) and its slope dV/da.  The cubic is expanded
// per region so that near-zero components cost no precision; V(a) =
// 1 - V(1 - a) folds a into [0, 1/2].  `q` holds the components in
// ascending order (q[0] = 0 in 2D).
template <typename T>
struct VolSlope {
  T v, dv;
};

template <typename T>
__device__ inline VolSlope<T> plic_lower_half(const T* q, bool three_d, T a) {
  VolSlope<T> r{T(0), T(0)};
  if (a <= T(0)) return r;
  if (!three_d) {
    const T lo = q[1], hi = q[2];
    if (a < lo) {
      r.v = T(0.5) * a * a / (lo * hi);
      r.dv = a / (lo * hi);
    } else {
      r.v = (a - T(0.5) * lo) / hi;
      r.dv = T(1) / hi;
    }
    return r;
  }
  const T p = q[0], s = q[1], t = q[2];
  const T inv_st = T(1) / (s * t);
  if (a < p) {
    r.v = a * a * a * inv_st / (T(6) * p);
    r.dv = T(0.5) * a * a * inv_st / p;
  } else if (a < s) {
    r.v = T(0.5) * (a * (a - p) + p * p / T(3)) * inv_st;
    r.dv = (a - T(0.5) * p) * inv_st;
  } else if (t >= p + s) {
    if (a < p + s) {
      T u = a - s;
      r.v = (a * a - a * p + p * p / T(3)) * T(0.5) * inv_st - u * u * u * inv_st / (T(6) * p);
      r.dv = (a - T(0.5) * p) * inv_st - T(0.5) * u * u * inv_st / p;
    } else {
      r.v = (a - T(0.5) * (p + s)) / t;
      r.dv = T(1) / t;
    }
  } else {
    T u = a - s, w = fmax(a - t, T(0));
    r.v = (a * a - a * p + p * p / T(3)) * T(0.5) * inv_st -
          (u * u * u + w * w * w) * inv_st / (T(6) * p);
    r.dv = (a - T(0.5) * p) * inv_st - T(0.5) * (u * u + w * w) * inv_st / p;
  }
  return r;
}

template <typename T>
__device__ inline VolSlope<T> plic_volume(const T* q, bool three_d, T a) {
  if (a <= T(0)) return VolSlope<T>{T(0), T(0)};
  if (a >= T(1)) return VolSlope<T>{T(1), T(0)};
  if (a <= T(0.5)) return plic_lower_half(q, three_d, a);
  VolSlope<T> r = plic_lower_half(q, three_d, T(1) - a);
  r.v = T(1) - r.v;
  return r;
}

// Plane offset alpha in [0, 1] with volume fraction C: the root of the
// increasing V(alpha) - C by Newton steps on the slope dV/dalpha, kept
// inside a bracket that every evaluation narrows (a bisection step replaces
// a Newton step that leaves it); stops when the step falls below the
// resolution of alpha, the bracket closes, or after 100 evaluations.  The
// same root as a bisection to full precision, in a handful of evaluations.
template <typename T>
__device__ inline T plic_alpha(const T* q, bool three_d, T C) {
  T lo = T(0), hi = T(1), a = C;
  for (int it = 0; it < 100; ++it) {
    const VolSlope<T> r = plic_volume(q, three_d, a);
    const T f = r.v - C;
    if (f == T(0)) return a;
    if (f < T(0)) lo = a;
    else hi = a;
    T an = r.dv > T(0) ? a - f / r.dv : T(0.5) * (lo + hi);
    if (!(an > lo && an < hi)) an = T(0.5) * (lo + hi);
    if (fabs(an - a) <= PlicTraits<T>::step_tol || !(hi - lo > T(0))) return an;
    a = an;
  }
  return a;
}

// Components |m|/sum|m| in ascending order (q[0] = 0 in 2D); false when m = 0.
template <typename T>
__device__ inline bool plic_sorted(int nd, const T* m, T* q) {
  T s = T(0);
  for (int d = 0; d < nd; ++d) s += fabs(m[d]);
  if (s == T(0)) return false;
  q[0] = nd == 3 ? fabs(m[2]) / s : T(0);
  q[1] = fabs(m[0]) / s;
  q[2] = fabs(m[1]) / s;
  if (q[0] > q[1]) { T t = q[0]; q[0] = q[1]; q[1] = t; }
  if (q[1] > q[2]) { T t = q[1]; q[1] = q[2]; q[2] = t; }
  if (q[0] > q[1]) { T t = q[0]; q[0] = q[1]; q[1] = t; }
  return true;
}

// Interface area inside the unit cell holding fraction C with normal m.
__device__ inline double plic_unit_area(int nd, const double* mraw, double C) {
  if (!(C > 0.0 && C < 1.0)) return 0.0;
  double s = 0.0, q2 = 0.0;
  for (int d = 0; d < nd; ++d) { s += fabs(mraw[d]); q2 += mraw[d] * mraw[d]; }
  if (s == 0.0) return 0.0;
  double q[3];
  plic_sorted(nd, mraw, q);
  const bool three_d = nd == 3;
  return (sqrt(q2) / s) * plic_volume(q, three_d, plic_alpha(q, three_d, C)).dv;
}

// Fluid {n.z <= alpha} (n = |m|/sum|m|, z reflected where m < 0) with
// z_d <= t: t times the volume of the box scaled by t along d.
template <typename T>
__device__ inline T plic_below(int nd, const T* n, T alpha, int d, T t) {
  if (t <= T(0)) return T(0);
  T np[3] = {T(0), T(0), T(0)}, s = T(0);
  for (int e = 0; e < nd; ++e) {
    np[e] = e == d ? n[e] * t : n[e];
    s += np[e];
  }
  if (s <= T(0)) return T(0);
  T q[3];
  if (!plic_sorted(nd, np, q)) return T(0);
  return t * plic_volume(q, nd == 3, alpha / s).v;
}

// Volume fraction of the unit cell (fluid fraction C, normal m pointing out
// of the fluid) that lies in the slab a <= x_d <= b.
template <typename T>
__device__ inline T plic_slab(int nd, const T* m, T C, int d, T a, T b) {
  if (C <= T(0)) return T(0);
  if (C >= T(1)) return b - a;
  T q[3];
  if (!plic_sorted(nd, m, q)) return C * (b - a);   // no direction: uniform
  const T alpha = plic_alpha(q, nd == 3, C);
  T s = T(0), n[3] = {T(0), T(0), T(0)};
  for (int e = 0; e < nd; ++e) s += fabs(m[e]);
  for (int e = 0; e < nd; ++e) n[e] = fabs(m[e]) / s;
  T ra = a, rb = b;
  if (m[d] < T(0)) {
    ra = T(1) - b;
    rb = T(1) - a;
  }
  return plic_below(nd, n, alpha, d, rb) - plic_below(nd, n, alpha, d, ra);
}

// Youngs normal: minus the (1,2,1)-weighted gradient of C over the
// 3x3(x3) block around (i,j,k), zero-gradient walls.
template <typename T>
__device__ inline void youngs_normal(const Level& L, const double* __restrict__ C, int i, int j,
                                     int k, T* m) {
  const int nd = L.ndim();
  m[0] = m[1] = m[2] = T(0);
  const int kr = nd == 3 ? 1 : 0;
  for (int dk = -kr; dk <= kr; ++dk)
    for (int dj = -1; dj <= 1; ++dj)
      for (int di = -1; di <= 1; ++di) {
        const int a = min(max(i + di, 0), L.nx - 1);
        const int b = min(max(j + dj, 0), L.ny - 1);
        const int e = min(max(k + dk, 0), L.nz - 1);
        const T w = (di == 0 ? T(2) : T(1)) * (dj == 0 ? T(2) : T(1)) *
                    (nd == 3 ? (dk == 0 ? T(2) : T(1)) : T(1));
        const T v = (T)C[cidx(L, a, b, e)];
        m[0] -= w * di * v;
        m[1] -= w * dj * v;
        m[2] -= w * dk * v;
      }
}

}  // namespace sfx
