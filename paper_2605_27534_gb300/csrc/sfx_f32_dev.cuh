// Device helpers of the SFX_F32 kernels (pair arithmetic on the stencil,
// metric weights, BCG face values), shared by the single-grid and the
// batched kernels so that both evaluate identical expressions.
#pragma once

#include <cuda_fp16.h>

#include "sfx_common.cuh"
#include "sfx_df.cuh"

namespace sfx {
namespace {

__device__ __forceinline__ unsigned int fbits(float v) { return __float_as_uint(v); }

// Asynchronous copies from global into shared memory (cp.async), their
// group commit and the wait for every committed group.
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// ------------------------------------------------------------ two lanes
// Both fields at once: lane x for f, lane y for F.  The packed FP32
// instructions round each lane exactly as the scalar ones do, so every
// lane computes the bits of the scalar expression it replaces.
__device__ __forceinline__ float2 v_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b as a + b (-1): the product is exact, so the one rounding is a - b's
__device__ __forceinline__ float2 v_sub(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}
__device__ __forceinline__ float2 v_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 v_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 v_bc(float a) { return make_float2(a, a); }

// A pair per lane: (hi.x, lo.x) of f, (hi.y, lo.y) of F.
struct P2 {
  float2 hi, lo;
};
__device__ __forceinline__ P2 p2_of(float2 f, float2 F) {
  return P2{make_float2(f.x, F.x), make_float2(f.y, F.y)};
}
__device__ __forceinline__ float2 p2_f(const P2& a) { return make_float2(a.hi.x, a.lo.x); }
__device__ __forceinline__ float2 p2_F(const P2& a) { return make_float2(a.hi.y, a.lo.y); }

// acc_add and acc_sub per lane
__device__ __forceinline__ void v_acc_add(P2& s, const P2& x) {
  const float2 t = v_add(s.hi, x.hi);
  const float2 bb = v_sub(t, s.hi);
  const float2 e = v_add(v_sub(s.hi, v_sub(t, bb)), v_sub(x.hi, bb));
  s.hi = t;
  s.lo = v_add(s.lo, v_add(e, x.lo));
}
__device__ __forceinline__ void v_acc_sub(P2& s, const P2& x) {
  // the two-sum of s.hi and -x.hi: -x.hi - bb rounds to -(x.hi + bb)
  const float2 t = v_sub(s.hi, x.hi);
  const float2 bb = v_sub(t, s.hi);
  const float2 e = v_sub(v_sub(s.hi, v_sub(t, bb)), v_add(x.hi, bb));
  s.hi = t;
  s.lo = v_add(s.lo, v_sub(e, x.lo));
}
// acc_get per lane
__device__ __forceinline__ P2 v_acc_get(const P2& s) {
  const float2 t = v_add(s.hi, s.lo);
  return P2{t, v_sub(s.lo, v_sub(t, s.hi))};
}
// lp_mul per lane
__device__ __forceinline__ P2 v_lp_mul(const P2& a, float2 b) {
  const float2 p = v_mul(a.hi, b);
  return P2{p, v_fma(a.lo, b, v_fma(a.hi, b, make_float2(-p.x, -p.y)))};
}
// lp_sub per lane
__device__ __forceinline__ P2 v_lp_sub(const P2& a, const P2& b) {
  const float2 t = v_sub(a.hi, b.hi);
  const float2 bb = v_sub(t, a.hi);
  const float2 e = v_sub(v_sub(a.hi, v_sub(t, bb)), v_add(b.hi, bb));
  return P2{t, v_add(e, v_sub(a.lo, b.lo))};
}

// ------------------------------------------------------------ drifts
// Folded float copy of phi: phi where phi <= 1/2, phi - 1 elsewhere.
__device__ __forceinline__ float fold_phi(double p) {
  return p <= 0.5 ? (float)p : (float)(p - 1.0);
}

// n = grad phi/|grad phi| at cell (i,j,k) (centred differences, one-sided
// copies at walls), faded out where phi is flat: scaled by
// clamp(q/kNormalKappa - 1, 0, 1), q = |grad phi| / (phi (1 - phi)/eps),
// and 0 below |grad phi| = 1e-30.  The differences are
// taken in FP64 from the double phi: deep in the bulk they are far below
// float resolution of phi but still fix the direction.  The 1/(2h) of the
// centred difference cancels in the normalisation; the components are
// scaled by their largest magnitude so that tiny gradients neither
// underflow nor lose the guard.
__device__ __forceinline__ void normal3_f32(const Level& L, const double* __restrict__ phi, int i,
                                            int j, int k, float inv_eps, float* n) {
  const int ip = min(i + 1, L.nx - 1), im = max(i - 1, 0);
  const int jp = min(j + 1, L.ny - 1), jm = max(j - 1, 0);
  const float g0 = (float)(phi[cidx(L, ip, j, k)] - phi[cidx(L, im, j, k)]);
  const float g1 = (float)(phi[cidx(L, i, jp, k)] - phi[cidx(L, i, jm, k)]);
  float g2 = 0.0f;
  if (L.geom == SFX_CART3D) {
    const int kp = min(k + 1, L.nz - 1), km = max(k - 1, 0);
    g2 = (float)(phi[cidx(L, i, j, kp)] - phi[cidx(L, i, j, km)]);
  }
  n[0] = n[1] = n[2] = 0.0f;
  const float mx = fmaxf(fabsf(g0), fmaxf(fabsf(g1), fabsf(g2)));
  if (mx == 0.0f) return;
  const float s0 = g0 / mx, s1 = g1 / mx, s2 = g2 / mx;
  const float r = sqrtf(s0 * s0 + s1 * s1 + s2 * s2);   // in [1, sqrt 3]
  const PhiPair pc = unfold(fold_phi(phi[cidx(L, i, j, k)]));
  const float m = mx * r * (0.5f / (float)L.h);
  if (m < 1e-30f) return;
  const float w = fminf(fmaxf(m / ((float)kNormalKappa * (pc.p * pc.q * inv_eps)) - 1.0f, 0.0f),
                        1.0f);
  if (!(w > 0.0f)) return;
  n[0] = w * (s0 / r);
  n[1] = w * (s1 / r);
  n[2] = w * (s2 / r);
}

__device__ __forceinline__ float normal_f32(const Level& L, const double* __restrict__ phi, int i,
                                            int j, int k, int d, float inv_eps) {
  float n[3];
  normal3_f32(L, phi, i, j, k, inv_eps, n);
  return n[d];
}

struct Nl32 {
  Level L;
  float invh, Doh, inv_dt, ka, kd, ginf, inv_eps, eta;
  int literal;
};

#include "sfx_corr3.cuh"

// Area weight of a face relative to h^(d-1) (planar, 3D: 1) or to pi h^2
// (axisymmetric: 2 i for the radial face at r = i h, 2 i + 1 for the axial
// faces of column i); the cell volume over the same unit times h is w_c h.
__device__ __forceinline__ float wr_face(int geom, int iface) {
  return geom == SFX_AXISYM ? 2.0f * (float)iface : 1.0f;
}
__device__ __forceinline__ float wz_face(int geom, int i) {
  return geom == SFX_AXISYM ? 2.0f * (float)i + 1.0f : 1.0f;
}

// Unnormalised pair accumulator: hi by error-free two-sums, everything else
// gathered in lo; normalised once at the end.
struct Acc {
  float hi, lo;
};
__device__ __forceinline__ void acc_add(Acc& s, float2 x) {
  float2 t = ef_two_sum(s.hi, x.x);
  s.hi = t.x;
  s.lo = __fadd_rn(s.lo, __fadd_rn(t.y, x.y));
}
__device__ __forceinline__ void acc_sub(Acc& s, float2 x) { acc_add(s, make_float2(-x.x, -x.y)); }
__device__ __forceinline__ float2 acc_get(const Acc& s) { return ef_fast_two_sum(s.hi, s.lo); }

// unnormalised products and differences (exact leading part + error term)
__device__ __forceinline__ float2 lp_mul(float2 a, float b) {
  float p = __fmul_rn(a.x, b);
  return make_float2(p, fmaf(a.y, b, fmaf(a.x, b, -p)));
}
__device__ __forceinline__ float2 lp_sub(float2 a, float2 b) {
  float2 t = ef_two_sum(a.x, -b.x);
  return make_float2(t.x, __fadd_rn(t.y, __fsub_rn(a.y, b.y)));
}

// Face quantity G = D (a_R - a_L)/h + B a_up as an unnormalised pair.  Both
// cells that share the face evaluate it from the same operands in the same
// order, so their contributions cancel exactly in the totals.
__device__ __forceinline__ float2 face_G(float Doh, float B, bool upL, float2 aL, float2 aR) {
  const float2 d = lp_mul(lp_sub(aR, aL), Doh);
  const float2 u = lp_mul(upL ? aL : aR, B);
  float2 t = ef_two_sum(d.x, u.x);
  return make_float2(t.x, __fadd_rn(t.y, __fadd_rn(d.y, u.y)));
}

// Residual, diagonal and |b| of one cell from its six neighbours (nb[q]
// valid when has[q]; order x-, x+, y-, y+, z-, z+) and face drifts B[q]:
//   r = (a* - a)/dt + (1/V) sum +-A G + (FIELD ? -q : q)
// Drift velocities B_f, B_F (Sec. 2.3) on the face between cells L and R
// (sL, sR: folded phi; nL, nR: normal components along the face): the mean
// of the two cell values.  0.5 - phi from the folded value keeps its
// precision on both sides.
__device__ __forceinline__ void drift_face(float sL, float sR, float nL, float nR, float Df,
                                           float DF, float inv_eps, float& bf, float& bF) {
  const PhiPair uL = unfold(sL), uR = unfold(sR);
  const float hL = signbit(sL) ? -0.5f - sL : 0.5f - sL;
  const float hR = signbit(sR) ? -0.5f - sR : 0.5f - sR;
  bf = 0.5f * ((-Df * 2.0f * hL * inv_eps) * nL + (-Df * 2.0f * hR * inv_eps) * nR);
  bF = 0.5f * ((-DF * uL.q * inv_eps) * nL + (-DF * uR.q * inv_eps) * nR);
}

// Cell and face indices of the FP32 kernels are 32-bit: an SFX_F32 context
// refuses grids whose cells or faces reach 2^31 (sfx_ctx_create).
using ix = unsigned int;

__device__ __forceinline__ ix cidx32(const Level& L, int i, int j, int k) {
  return ((ix)k * (ix)L.ny + (ix)j) * (ix)L.nx + (ix)i;
}

// G: the grid's geometry as a compile-time constant (the Newton kernels are
// instantiated per geometry; L.geom == G), or kGeomRuntime to read it from
// the level at run time
constexpr int kGeomRuntime = -1;
template <int G>
__device__ __forceinline__ int geom_of(const Level& L) {
  return G == kGeomRuntime ? L.geom : G;
}

template <int G>
__device__ __forceinline__ void gather6(const Level& L, int i, int j, int k, ix c,
                                        bool* has, ix* nbi) {
  const ix sy = (ix)L.nx, sz = (ix)L.nx * (ix)L.ny;
  has[0] = i > 0; has[1] = i + 1 < L.nx; has[2] = j > 0; has[3] = j + 1 < L.ny;
  const bool three_d = geom_of<G>(L) == SFX_CART3D;
  has[4] = three_d && k > 0; has[5] = three_d && k + 1 < L.nz;
  nbi[0] = c - 1; nbi[1] = c + 1; nbi[2] = c - sy; nbi[3] = c + sy; nbi[4] = c - sz; nbi[5] = c + sz;
}

// Colour-packed layout of the Newton work arrays (corrections, 2x2
// coefficients, residuals): the cells of each red-black colour are stored
// contiguously, `half` = ceil(nx/2) per row, red plane first.  A colour
// launch then reads and writes whole cache lines, and the neighbours of a
// cell (all of the other colour) sit at pos - 1 + (i & 1), pos + (i & 1)
// (x), pos -+ half (y) and pos -+ ny half (z) of the other plane.
struct RBIdx {
  ix plane, pos, half;
};
__device__ __forceinline__ RBIdx rb_index(const Level& L, int i, int j, int k) {
  RBIdx r;
  r.half = (ix)((L.nx + 1) >> 1);
  r.plane = (ix)L.ny * (ix)L.nz * r.half;
  r.pos = ((ix)k * (ix)L.ny + (ix)j) * r.half + (ix)(i >> 1);
  return r;
}

// The six face drifts of cell c = (i,j,k).  With row = k ny + j the face
// indices are c + row (x), c + k nx (y) and c (z) on the minus side, plus
// 1, nx and nx ny on the plus side.
__device__ __forceinline__ float face_val(float b) { return b; }
__device__ __forceinline__ float face_val(__half b) { return __half2float(b); }

template <typename T>
__device__ __forceinline__ void faces6(const Level& L, const T* Bx, const T* By,
                                       const T* Bz, int i, int j, int k, const bool* has,
                                       float* B) {
  const ix c = cidx32(L, i, j, k);
  const ix fx = c + (ix)k * (ix)L.ny + (ix)j, fy = c + (ix)k * (ix)L.nx;
  B[0] = has[0] ? face_val(Bx[fx]) : 0.0f;
  B[1] = has[1] ? face_val(Bx[fx + 1]) : 0.0f;
  B[2] = has[2] ? face_val(By[fy]) : 0.0f;
  B[3] = has[3] ? face_val(By[fy + L.nx]) : 0.0f;
  B[4] = has[4] ? face_val(Bz[c]) : 0.0f;
  B[5] = has[5] ? face_val(Bz[c + (ix)L.nx * (ix)L.ny]) : 0.0f;
}

// faces6 for both fields at once from packed (B_f, B_F) float2 faces.
__device__ __forceinline__ void faces6f2(const Level& L, const float2* Bx, const float2* By,
                                         const float2* Bz, int i, int j, int k, const bool* has,
                                         float* Bf, float* BF) {
  const ix c = cidx32(L, i, j, k);
  const ix fx = c + (ix)k * (ix)L.ny + (ix)j, fy = c + (ix)k * (ix)L.nx;
  const float2 z = make_float2(0.0f, 0.0f);
  float2 v[6];
  v[0] = has[0] ? Bx[fx] : z;
  v[1] = has[1] ? Bx[fx + 1] : z;
  v[2] = has[2] ? By[fy] : z;
  v[3] = has[3] ? By[fy + L.nx] : z;
  v[4] = has[4] ? Bz[c] : z;
  v[5] = has[5] ? Bz[c + (ix)L.nx * (ix)L.ny] : z;
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    Bf[q] = v[q].x;
    BF[q] = v[q].y;
  }
}

// faces6f2 with each face's (B_f, B_F) kept together (one lane per field).
__device__ __forceinline__ void faces6v(const Level& L, const float2* Bx, const float2* By,
                                        const float2* Bz, int i, int j, int k, const bool* has,
                                        float2* B) {
  const ix c = cidx32(L, i, j, k);
  const ix fx = c + (ix)k * (ix)L.ny + (ix)j, fy = c + (ix)k * (ix)L.nx;
  const float2 z = make_float2(0.0f, 0.0f);
  B[0] = has[0] ? Bx[fx] : z;
  B[1] = has[1] ? Bx[fx + 1] : z;
  B[2] = has[2] ? By[fy] : z;
  B[3] = has[3] ? By[fy + L.nx] : z;
  B[4] = has[4] ? Bz[c] : z;
  B[5] = has[5] ? Bz[c + (ix)L.nx * (ix)L.ny] : z;
}

// faces6 for both fields at once from the packed (B_f, B_F) half2 faces.
__device__ __forceinline__ void faces6x2(const Level& L, const __half2* Hx, const __half2* Hy,
                                         const __half2* Hz, int i, int j, int k, const bool* has,
                                         float* Bf, float* BF) {
  const ix c = cidx32(L, i, j, k);
  const ix fx = c + (ix)k * (ix)L.ny + (ix)j, fy = c + (ix)k * (ix)L.nx;
  const __half2 z = __floats2half2_rn(0.0f, 0.0f);
  __half2 h[6];
  h[0] = has[0] ? Hx[fx] : z;
  h[1] = has[1] ? Hx[fx + 1] : z;
  h[2] = has[2] ? Hy[fy] : z;
  h[3] = has[3] ? Hy[fy + L.nx] : z;
  h[4] = has[4] ? Hz[c] : z;
  h[5] = has[5] ? Hz[c + (ix)L.nx * (ix)L.ny] : z;
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const float2 v = __half22float2(h[q]);
    Bf[q] = v.x;
    BF[q] = v.y;
  }
}

// (1/V) sum +-A G of both fields around cell i (lane x f with Doh.x and
// drifts B[q].x, lane y F) as an unnormalised pair, and
// the derivative of that sum in the cell value (negated: diagonal weight).
// The diffusive part is gathered as Doh (sum_q w_q a_q - W a_c), W = sum_q
// w_q, one pair product instead of one per face; the drift part as
// sum_q +-w_q B_q a_up(q).
template <int G>
__device__ __forceinline__ P2 flux_pair2(const Level& L, float invh, float2 Doh, int literal,
                                         int i, const P2& ac, const P2* nb, const bool* has,
                                         const float2* B, float2& dflux) {
  const bool axi = geom_of<G>(L) == SFX_AXISYM;
  P2 D{v_bc(0.0f), v_bc(0.0f)}, T{v_bc(0.0f), v_bc(0.0f)};
  float W = 0.0f;
  float2 dg = v_bc(0.0f);
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    if (!has[q]) continue;
    const bool plus = q & 1;
    const bool upf = literal ? (B[q].x > 0.0f) : (B[q].x < 0.0f);
    const bool upF = literal ? (B[q].y > 0.0f) : (B[q].y < 0.0f);
    float w = 1.0f;
    const int g = geom_of<G>(L);
    if (axi) w = q < 2 ? wr_face(g, i + (plus ? 1 : 0)) : (q < 4 ? wz_face(g, i) : 1.0f);
    v_acc_add(D, axi ? v_lp_mul(nb[q], v_bc(w)) : nb[q]);
    W = __fadd_rn(W, w);
    // upwind value per lane: the left cell when up; this cell is left on
    // plus faces
    const bool cf = plus == upf, cF = plus == upF;
    const P2 aup{make_float2(cf ? ac.hi.x : nb[q].hi.x, cF ? ac.hi.y : nb[q].hi.y),
                 make_float2(cf ? ac.lo.x : nb[q].lo.x, cF ? ac.lo.y : nb[q].lo.y)};
    P2 u = v_lp_mul(aup, B[q]);
    if (axi) u = v_lp_mul(u, v_bc(w));
    if (plus) {
      v_acc_add(T, u);
      dg = v_fma(v_bc(w), v_sub(Doh, make_float2(upf ? B[q].x : 0.0f, upF ? B[q].y : 0.0f)), dg);
    } else {
      v_acc_sub(T, u);
      dg = v_fma(v_bc(w), v_add(Doh, make_float2(upf ? 0.0f : B[q].x, upF ? 0.0f : B[q].y)), dg);
    }
  }
  v_acc_sub(D, v_lp_mul(ac, v_bc(W)));
  v_acc_add(T, v_lp_mul(v_acc_get(D), Doh));
  P2 flux = v_lp_mul(v_acc_get(T), v_bc(invh));
  dflux = v_mul(dg, v_bc(invh));
  if (axi) {
    const float wc = wz_face(geom_of<G>(L), i);
    const float2 a = df_div_f(ef_fast_two_sum(flux.hi.x, flux.lo.x), wc);
    const float2 b = df_div_f(ef_fast_two_sum(flux.hi.y, flux.lo.y), wc);
    flux = p2_of(a, b);
    dflux = make_float2(__fdividef(dflux.x, wc), __fdividef(dflux.y, wc));
  }
  return flux;
}

// linear flux of a correction field (FP32) and its diagonal weight
template <int G>
__device__ __forceinline__ float flux_lin(const Level& L, float invh, float Doh, int literal,
                                          int i, float ec, const float* en, const bool* has,
                                          const float* B, float& dflux) {
  float S = 0.0f, dg = 0.0f;
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    if (!has[q]) continue;
    const bool plus = q & 1;
    const bool upL = literal ? (B[q] > 0.0f) : (B[q] < 0.0f);
    float w = 1.0f;
    const int g = geom_of<G>(L);
    if (g == SFX_AXISYM) w = q < 2 ? wr_face(g, i + (plus ? 1 : 0)) : (q < 4 ? wz_face(g, i) : 1.0f);
    const float eL = plus ? ec : en[q], eR = plus ? en[q] : ec;
    const float fq = __fmaf_rn(Doh, __fsub_rn(eR, eL), __fmul_rn(B[q], upL ? eL : eR));
    if (plus) {
      S = __fmaf_rn(w, fq, S);
      dg = __fmaf_rn(w, __fsub_rn(Doh, upL ? B[q] : 0.0f), dg);
    } else {
      S = __fmaf_rn(-w, fq, S);
      dg = __fmaf_rn(w, __fadd_rn(Doh, upL ? 0.0f : B[q]), dg);
    }
  }
  const float s = invh / wz_face(geom_of<G>(L), i);
  dflux = __fmul_rn(dg, s);
  return __fmul_rn(S, s);
}

// flux_lin of both fields at once (lane x f with Doh.x, drifts B[q].x and
// corrections en[q].x; lane y F), the same operations per lane.
template <int G>
__device__ __forceinline__ float2 flux_lin2(const Level& L, float invh, float2 Doh, int literal,
                                            int i, float2 ec, const float2* en, const bool* has,
                                            const float2* B, float2& dflux) {
  float2 S = v_bc(0.0f), dg = v_bc(0.0f);
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    if (!has[q]) continue;
    const bool plus = q & 1;
    const bool upf = literal ? (B[q].x > 0.0f) : (B[q].x < 0.0f);
    const bool upF = literal ? (B[q].y > 0.0f) : (B[q].y < 0.0f);
    float w = 1.0f;
    const int g = geom_of<G>(L);
    if (g == SFX_AXISYM) w = q < 2 ? wr_face(g, i + (plus ? 1 : 0)) : (q < 4 ? wz_face(g, i) : 1.0f);
    const float2 eL = plus ? ec : en[q], eR = plus ? en[q] : ec;
    const float2 up = make_float2(upf ? eL.x : eR.x, upF ? eL.y : eR.y);
    const float2 fq = v_fma(Doh, v_sub(eR, eL), v_mul(B[q], up));
    if (plus) {
      S = v_fma(v_bc(w), fq, S);
      dg = v_fma(v_bc(w), v_sub(Doh, make_float2(upf ? B[q].x : 0.0f, upF ? B[q].y : 0.0f)), dg);
    } else {
      S = v_fma(v_bc(-w), fq, S);
      dg = v_fma(v_bc(w), v_add(Doh, make_float2(upf ? 0.0f : B[q].x, upF ? 0.0f : B[q].y)), dg);
    }
  }
  const float s = invh / wz_face(geom_of<G>(L), i);
  dflux = v_mul(dg, v_bc(s));
  return v_mul(S, v_bc(s));
}

__device__ __forceinline__ float mc32(float xm, float x0, float xp) {
  float dl = x0 - xm, dr = xp - x0;
  if (dl * dr <= 0.0f) return 0.0f;
  float dc = 0.5f * (xp - xm);
  float m = fminf(fabsf(dc), 2.0f * fminf(fabsf(dl), fabsf(dr)));
  return dc > 0.0f ? m : -m;
}

struct Adv32 {
  Level L;
  float dt, invh;
  const float* u[3];
};

__device__ __forceinline__ float vnb(const Level& L, const float2* __restrict__ x, const int* uc,
                                     size_t U, int d, int s) {
  int p = uc[d] + s;
  if (p < 0 || p >= L.extent(d)) return df_val(x[U]);
  size_t stride = d == 0 ? 1 : (d == 1 ? (size_t)L.nx : (size_t)L.nx * L.ny);
  return df_val(s > 0 ? x[U + stride] : x[U - stride]);
}

// BCG face value (see sfx_advect.cu) in FP32 on the pair values.
__device__ float face32v(const Adv32& A, const float2* __restrict__ x, float bc_in, int d,
                         const int* f, float u) {
  const Level& L = A.L;
  int uc[3] = {f[0], f[1], f[2]};
  if (u > 0.0f) {
    if (f[d] == 0) return bc_in;
    uc[d] -= 1;
  } else if (f[d] == L.extent(d)) {
    return bc_in;
  }
  size_t U = cidx(L, uc[0], uc[1], uc[2]);
  float x0 = df_val(x[U]);
  float slope = mc32(vnb(L, x, uc, U, d, -1), x0, vnb(L, x, uc, U, d, +1));
  float val = x0 + 0.5f * ((u > 0.0f ? 1.0f : -1.0f) - u * A.dt * A.invh) * slope;
  for (int t = 0; t < L.ndim(); ++t) {
    if (t == d) continue;
    int ap[3] = {uc[0], uc[1], uc[2]};
    ap[t] += 1;
    float vbar = 0.5f * (A.u[t][fidx(L, t, uc[0], uc[1], uc[2])] + A.u[t][fidx(L, t, ap[0], ap[1], ap[2])]);
    float dif = vbar > 0.0f ? x0 - vnb(L, x, uc, U, t, -1) : vnb(L, x, uc, U, t, +1) - x0;
    val -= 0.5f * A.dt * vbar * dif * A.invh;
  }
  return val;
}

// face32v for two fields at once: the upwind cell, its index and the
// transverse velocities are shared; each field's arithmetic is that of
// face32v.
// Neighbour value along d with a zero-gradient copy at walls, 32-bit
// indices (SFX_F32 grids stay below 2^31 faces).
__device__ __forceinline__ float vnb32(const Level& L, const float2* __restrict__ x, const int* uc,
                                       ix U, int d, int s) {
  const int p = uc[d] + s;
  if (p < 0 || p >= L.extent(d)) return df_val(x[U]);
  const ix stride = d == 0 ? 1u : (d == 1 ? (ix)L.nx : (ix)L.nx * (ix)L.ny);
  return df_val(s > 0 ? x[U + stride] : x[U - stride]);
}
__device__ __forceinline__ ix fidx32(const Level& L, int d, int i, int j, int k) {
  const ix fx = (ix)(L.nx + (d == 0)), fy = (ix)(L.ny + (d == 1));
  return ((ix)k * fy + (ix)j) * fx + (ix)i;
}

// The BCG face value of both fields (Sec. 3.1) from the upwind cell's
// values a: a + cfl x (MC-limited slope along d) minus the transverse
// upwind differences times the mean transverse velocity.  nb(t, s) gives
// both fields' values of the upwind cell's neighbour at offset s along t
// (the cell itself past a wall), vb(t) the mean velocity of its two faces
// along t.  Every rounding is spelled out, so that each kernel that
// fetches the operands its own way (global memory, shared-memory tiles)
// computes the same bits.
template <class Nb, class Vb>
__device__ __forceinline__ void bcg_face2(float2 a, float u, float dt, float invh, int d, int nd,
                                          Nb nb, Vb vb, float& v1, float& v2) {
  const float cfl = __fmul_rn(0.5f, __fmaf_rn(-__fmul_rn(u, dt), invh, u > 0.0f ? 1.0f : -1.0f));
  const float2 m = nb(d, -1), pl = nb(d, +1);
  v1 = __fmaf_rn(cfl, mc32(m.x, a.x, pl.x), a.x);
  v2 = __fmaf_rn(cfl, mc32(m.y, a.y, pl.y), a.y);
  const float hdt = __fmul_rn(0.5f, dt);
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    if (t >= nd || t == d) continue;
    const float vbar = vb(t);
    const bool up = vbar > 0.0f;
    const float2 n = nb(t, up ? -1 : +1);
    const float d1 = up ? __fsub_rn(a.x, n.x) : __fsub_rn(n.x, a.x);
    const float d2 = up ? __fsub_rn(a.y, n.y) : __fsub_rn(n.y, a.y);
    const float s = __fmul_rn(hdt, vbar);
    v1 = __fmaf_rn(-__fmul_rn(s, d1), invh, v1);
    v2 = __fmaf_rn(-__fmul_rn(s, d2), invh, v2);
  }
}

__device__ __forceinline__ void face32v2(const Adv32& A, const float2* __restrict__ x1,
                                         const float2* __restrict__ x2, float bc1, float bc2,
                                         int d, const int* f, float u, float& v1, float& v2) {
  const Level& L = A.L;
  int uc[3] = {f[0], f[1], f[2]};
  if (u > 0.0f) {
    if (f[d] == 0) { v1 = bc1; v2 = bc2; return; }
    uc[d] -= 1;
  } else if (f[d] == L.extent(d)) {
    v1 = bc1;
    v2 = bc2;
    return;
  }
  const ix U = cidx32(L, uc[0], uc[1], uc[2]);
  const float2 a = make_float2(df_val(x1[U]), df_val(x2[U]));
  const int c0 = uc[0], c1 = uc[1], c2 = uc[2];
  auto nb = [&](int t, int sgn) {
    const int pos = (t == 0 ? c0 : (t == 1 ? c1 : c2)) + sgn;
    if (pos < 0 || pos >= L.extent(t)) return a;
    const ix stride = t == 0 ? 1u : (t == 1 ? (ix)L.nx : (ix)L.nx * (ix)L.ny);
    const ix V = sgn > 0 ? U + stride : U - stride;
    return make_float2(df_val(x1[V]), df_val(x2[V]));
  };
  auto vb = [&](int t) {
    return __fmul_rn(0.5f, __fadd_rn(A.u[t][fidx32(L, t, c0, c1, c2)],
                                     A.u[t][fidx32(L, t, c0 + (t == 0), c1 + (t == 1),
                                                   c2 + (t == 2))]));
  };
  bcg_face2(a, u, A.dt, A.invh, d, L.ndim(), nb, vb, v1, v2);
}

__device__ __forceinline__ void resid2_tail(const Nw32& p, int i, int j, int k, ix c,
                                            const float* __restrict__ phi, const P2& ac,
                                            const P2& fl, float2 dfl,
                                            const float2* __restrict__ fst,
                                            const float2* __restrict__ Fst,
                                            float4* __restrict__ rc, float* m,
                                            float2* __restrict__ e2);

// `done`: the solve converged at an earlier iteration; `mode` (may be
// null): the residual kind chosen on the device for this iteration (0 the
// FP32 pass, 1 the pair pass, 2 the incremental FP32 pass); a launch whose
// kind `want` is not chosen returns at once.
__device__ __forceinline__ bool resid_skip(const int* done, const int* mode, int want) {
  return (done && *done) || (mode && *mode != want);
}

// Warp maxima of the four norms, then one atomic per block and norm.
__device__ __forceinline__ void resid_norms(const float* m, unsigned int* norms) {
  __shared__ float wm[4][8];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float v = warp_max(m[q]);
    if ((threadIdx.x & 31) == 0) wm[q][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    float v = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v = fmaxf(v, wm[threadIdx.x][w]);
    atomicMax(&norms[threadIdx.x], fbits(v));
  }
}

// Both residuals (pairs) of App. C at cell c of the current state, the
// kinetic diagonals and couplings of the linearised system, and the running
// maxima m = {|r_f|, |b_f|, |r_F|, |b_F|}.  With e2 != NULL the first red
// half-sweep of the correction is done here: it starts from zero
// corrections, so a red cell (i + j + k even) only needs its own 2x2 block,
// e = M_c^-1 r_c.
template <int G>
__device__ __forceinline__ void resid2_cell(const Nw32& p, int i, int j, int k, ix c,
                                            const float* __restrict__ phi,
                                            const float2* const* B2,
                                            const float2* __restrict__ fin,
                                            const float2* __restrict__ Fin,
                                            const float2* __restrict__ fst,
                                            const float2* __restrict__ Fst,
                                            float4* __restrict__ rc, float* m,
                                            float2* __restrict__ e2) {
  const Level& L = p.L;
  bool has[6];
  ix nbi[6];
  gather6<G>(L, i, j, k, c, has, nbi);
  // both fields' pairs, one lane per field
  P2 nb[6];
  const P2 ac = p2_of(fin[c], Fin[c]);
  float2 B[6], dfl;
  faces6v(L, B2[0], B2[1], B2[2], i, j, k, has, B);
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const float2 z = make_float2(0.0f, 0.0f);
    nb[q] = p2_of(has[q] ? fin[nbi[q]] : z, has[q] ? Fin[nbi[q]] : z);
  }
  const P2 fl = flux_pair2<G>(L, p.invh, make_float2(p.Dfh, p.DFh), p.literal, i, ac, nb, has,
                              B, dfl);
  resid2_tail(p, i, j, k, c, phi, ac, fl, dfl, fst, Fst, rc, m, e2);
}

// The rest of the pair residual of one cell from the cell's pairs ac and
// its pair fluxes fl (already over h, lane x f, lane y F) with their
// diagonal weights dfl: the exchange, both residuals, u and v, the first
// red half-sweep and the norms (the outputs of resid2_cell).
__device__ __forceinline__ void resid2_tail(const Nw32& p, int i, int j, int k, ix c,
                                            const float* __restrict__ phi, const P2& ac,
                                            const P2& fl, float2 dfl,
                                            const float2* __restrict__ fst,
                                            const float2* __restrict__ Fst,
                                            float4* __restrict__ rc, float* m,
                                            float2* __restrict__ e2) {
  const Level& L = p.L;
  const float2 fc = p2_f(ac), Fc = p2_F(ac);
  // exchange q = c1 F (f_inf - f) - r_d f, one evaluation for both equations
  const PhiPair ph = unfold(phi[c]);
  const float c1 = __fdividef(p.ka, ph.p + p.eta);
  const float finf = __fmul_rn(__fmul_rn(__fmul_rn(p.ginf, ph.p), ph.q), p.inv_eps);
  float2 fd = ef_two_sum(finf, -fc.x);
  fd.y = __fsub_rn(fd.y, fc.y);
  const float pr = __fmul_rn(Fc.x, fd.x);
  const float2 FF = make_float2(pr, fmaf(Fc.y, fd.x, fmaf(Fc.x, fd.y, fmaf(Fc.x, fd.x, -pr))));
  const float2 ads = lp_mul(FF, c1), des = lp_mul(fc, p.kd);
  Acc q{0.0f, 0.0f};
  acc_add(q, ads);
  acc_sub(q, des);
  const float2 qq = acc_get(q);
  const float2 fs = fst[c], Fs = Fst[c];
  // both residuals, one lane each: (x* - x)/dt + flux, then +q (f), -q (F)
  P2 R{v_bc(0.0f), v_bc(0.0f)};
  v_acc_add(R, v_lp_mul(v_lp_sub(p2_of(fs, Fs), ac), v_bc(p.inv_dt)));
  v_acc_add(R, fl);
  v_acc_add(R, P2{make_float2(qq.x, -qq.x), make_float2(qq.y, -qq.y)});
  const float2 rr = v_add(R.hi, R.lo);
  const float rf = rr.x, rF = rr.y;
  const float Fv = __fadd_rn(Fc.x, Fc.y), fv = __fadd_rn(fc.x, fc.y);
  // the linearised exchange: u = c1 F and v = c1 (f_inf - f) fix the 2x2
  // block (Jac2); stored with the residuals as one float4 per cell
  const float u = __fmul_rn(c1, Fv), v = __fmul_rn(c1, __fsub_rn(finf, fv));
  const RBIdx rb = rb_index(L, i, j, k);
  const ix own = (ix)((i + j + k) & 1) * rb.plane + rb.pos;
  rc[own] = make_float4(rf, rF, u, v);
  if (e2 && ((i + j + k) & 1) == 0) {
    // [a -b; -d e] [x; y] = [r_f; r_F], diagonals with the flux weights
    const Jac2 J = jac2(p, u, v);
    const float a = __fadd_rn(J.ff, dfl.x), e = __fadd_rn(J.FF, dfl.y);
    const float inv = __fdividef(1.0f, __fmaf_rn(a, e, -__fmul_rn(J.fF, J.Ff)));
    e2[own] = make_float2(__fmul_rn(__fmaf_rn(e, rf, __fmul_rn(J.fF, rF)), inv),
                          __fmul_rn(__fmaf_rn(J.Ff, rf, __fmul_rn(a, rF)), inv));
  }
  m[0] = fmaxf(m[0], fabsf(rf));
  m[1] = fmaxf(m[1], fabsf(__fmaf_rn(fs.x, p.inv_dt, __fmul_rn(__fmul_rn(c1, Fv), finf))));
  m[2] = fmaxf(m[2], fabsf(rF));
  m[3] = fmaxf(m[3], fabsf(__fmaf_rn(Fs.x, p.inv_dt, __fmul_rn(p.kd, fv))));
  if (!(fabsf(rf) <= 3.0e38f) || !(fabsf(rF) <= 3.0e38f)) m[0] = m[2] = __int_as_float(0x7f800000);
}

// resid2_cell in FP32 arithmetic on the leading floats of the pairs (the
// same outputs: residuals, u, v, the first red half-sweep and the norms;
// residuals within ~1e-7 of the scale m[1], m[3]).  The Newton iterations
// far from convergence use it: their corrections need residuals only to a
// few digits, and the iterations that decide convergence evaluate the pair
// residual.
template <int G>
__device__ __forceinline__ void resid32_cell(const Nw32& p, int i, int j, int k, ix c,
                                             const float* __restrict__ phi,
                                             const float2* const* B2,
                                             const float2* __restrict__ fin,
                                             const float2* __restrict__ Fin,
                                             const float2* __restrict__ fst,
                                             const float2* __restrict__ Fst,
                                             float4* __restrict__ rc, float* m,
                                             float2* __restrict__ e2) {
  const Level& L = p.L;
  bool has[6];
  ix nbi[6];
  gather6<G>(L, i, j, k, c, has, nbi);
  float2 B[6], nv[6], dfl;
  faces6v(L, B2[0], B2[1], B2[2], i, j, k, has, B);
#pragma unroll
  for (int q = 0; q < 6; ++q)
    nv[q] = has[q] ? make_float2(fin[nbi[q]].x, Fin[nbi[q]].x) : make_float2(0.0f, 0.0f);
  const float fc = fin[c].x, Fc = Fin[c].x;
  const float2 fl = flux_lin2<G>(L, p.invh, make_float2(p.Dfh, p.DFh), p.literal, i,
                                 make_float2(fc, Fc), nv, has, B, dfl);
  const float flf = fl.x, flF = fl.y, df_ = dfl.x, dF_ = dfl.y;
  const PhiPair ph = unfold(phi[c]);
  const float c1 = __fdividef(p.ka, ph.p + p.eta);
  const float finf = __fmul_rn(__fmul_rn(__fmul_rn(p.ginf, ph.p), ph.q), p.inv_eps);
  const float u = __fmul_rn(c1, Fc), v = __fmul_rn(c1, __fsub_rn(finf, fc));
  const float qx = __fmaf_rn(v, Fc, -__fmul_rn(p.kd, fc));   // c1 F (f_inf - f) - r_d f
  const float fs = fst[c].x, Fs = Fst[c].x;
  const float rf = __fadd_rn(__fmaf_rn(__fsub_rn(fs, fc), p.inv_dt, flf), qx);
  const float rF = __fsub_rn(__fmaf_rn(__fsub_rn(Fs, Fc), p.inv_dt, flF), qx);
  const RBIdx rb = rb_index(L, i, j, k);
  const ix own = (ix)((i + j + k) & 1) * rb.plane + rb.pos;
  rc[own] = make_float4(rf, rF, u, v);
  if (e2 && ((i + j + k) & 1) == 0) {
    const Jac2 J = jac2(p, u, v);
    const float a = __fadd_rn(J.ff, df_), e = __fadd_rn(J.FF, dF_);
    const float inv = __fdividef(1.0f, __fmaf_rn(a, e, -__fmul_rn(J.fF, J.Ff)));
    e2[own] = make_float2(__fmul_rn(__fmaf_rn(e, rf, __fmul_rn(J.fF, rF)), inv),
                          __fmul_rn(__fmaf_rn(J.Ff, rf, __fmul_rn(a, rF)), inv));
  }
  m[0] = fmaxf(m[0], fabsf(rf));
  m[1] = fmaxf(m[1], fabsf(__fmaf_rn(fs, p.inv_dt, __fmul_rn(u, finf))));
  m[2] = fmaxf(m[2], fabsf(rF));
  m[3] = fmaxf(m[3], fabsf(__fmaf_rn(Fs, p.inv_dt, __fmul_rn(p.kd, fc))));
  if (!(fabsf(rf) <= 3.0e38f) || !(fabsf(rF) <= 3.0e38f)) m[0] = m[2] = __int_as_float(0x7f800000);
}

// The residuals of the state x + e from those of x (rc) and the correction
// e just added to it (E, both colours, colour-packed), in FP32: the
// App. C residual changes by
//   r_f: -e_f/dt + flux_f(e_f) + dq,   r_F: -e_F/dt + flux_F(e_F) - dq,
//   dq = c1 (e_F (f_inf - f) - F e_f - e_F e_f) - r_d e_f
//      = e_F v - u e_f - c1 e_F e_f - r_d e_f
// with u = c1 F and v = c1 (f_inf - f) of x (rc's third and fourth
// entries), which become u + c1 e_F and v - c1 e_f for x + e: linear terms
// and a product of the correction, all of the size of the old residual,
// so FP32 rounding stays ~1e-7 of it, and after a pair residual pass this
// keeps the pair pass's accuracy.  Neither the state nor x* is read: the
// norms' scales m[1], m[3] are left at zero and the convergence test takes
// those of the pass the chain started from.  The other outputs are those
// of resid2_cell.
template <int G>
__device__ __forceinline__ void resid32_incr_cell(const Nw32& p, int i, int j, int k, ix c,
                                                  const float* __restrict__ phi,
                                                  const float2* const* B2,
                                                  const float2* __restrict__ E,
                                                  float4* __restrict__ rc, float* m,
                                                  float2* __restrict__ e2) {
  const Level& L = p.L;
  bool has[6];
  ix nbi[6];
  gather6<G>(L, i, j, k, c, has, nbi);
  // the correction of this cell and of its neighbours (the other colour)
  const RBIdx rb = rb_index(L, i, j, k);
  const int col = (i + j + k) & 1;
  const ix own = (ix)col * rb.plane + rb.pos, oth = (ix)(1 - col) * rb.plane + rb.pos;
  const ix sz = (ix)L.ny * rb.half;
  nbi[0] = oth - 1 + (i & 1);
  nbi[1] = oth + (i & 1);
  nbi[2] = oth - rb.half;
  nbi[3] = oth + rb.half;
  nbi[4] = oth - sz;
  nbi[5] = oth + sz;
  float2 B[6], ev[6], dfl;
  faces6v(L, B2[0], B2[1], B2[2], i, j, k, has, B);
#pragma unroll
  for (int q = 0; q < 6; ++q) ev[q] = has[q] ? E[nbi[q]] : make_float2(0.0f, 0.0f);
  const float2 ec = E[own];
  const float4 r0 = rc[own];
  const float2 fl = flux_lin2<G>(L, p.invh, make_float2(p.Dfh, p.DFh), p.literal, i, ec, ev, has,
                                 B, dfl);
  const float flf = fl.x, flF = fl.y, df_ = dfl.x, dF_ = dfl.y;
  const PhiPair ph = unfold(phi[c]);
  const float c1 = __fdividef(p.ka, ph.p + p.eta);
  // dq = e_F v - u e_f - c1 e_F e_f - r_d e_f with x's u, v
  const float ce = __fmul_rn(c1, ec.x);
  const float dq = __fmaf_rn(ec.y, __fsub_rn(r0.w, ce),
                             -__fmul_rn(__fadd_rn(r0.z, p.kd), ec.x));
  const float rf = __fadd_rn(__fadd_rn(__fmaf_rn(-ec.x, p.inv_dt, r0.x), flf), dq);
  const float rF = __fsub_rn(__fadd_rn(__fmaf_rn(-ec.y, p.inv_dt, r0.y), flF), dq);
  const float u = __fmaf_rn(c1, ec.y, r0.z), v = __fsub_rn(r0.w, ce);
  rc[own] = make_float4(rf, rF, u, v);
  if (col == 0) {
    const Jac2 J = jac2(p, u, v);
    const float a = __fadd_rn(J.ff, df_), e = __fadd_rn(J.FF, dF_);
    const float inv = __fdividef(1.0f, __fmaf_rn(a, e, -__fmul_rn(J.fF, J.Ff)));
    e2[own] = make_float2(__fmul_rn(__fmaf_rn(e, rf, __fmul_rn(J.fF, rF)), inv),
                          __fmul_rn(__fmaf_rn(J.Ff, rf, __fmul_rn(a, rF)), inv));
  }
  m[0] = fmaxf(m[0], fabsf(rf));
  m[2] = fmaxf(m[2], fabsf(rF));
  if (!(fabsf(rf) <= 3.0e38f) || !(fabsf(rF) <= 3.0e38f)) m[0] = m[2] = __int_as_float(0x7f800000);
}

// One cell of the coupled red-black Gauss-Seidel on the correction; with
// fst != NULL (the last black colour of an iteration) the corrections of
// this cell and of its red pair partner are added to the state.  The sweeps
// only precondition the Newton correction (the residual pass fixes the
// solution), so they read the face drifts in half precision (relative
// 5e-4), halving their face traffic.
// Everything one cell of the correction sweep reads (split from its
// arithmetic so that a thread can have two cells' loads in flight).
struct Corr2In {
  bool has[6];
  float enf[6], enF[6], Bf[6], BF[6];
  float2 ec;
  float4 q4;
  ix c, own, oth;
  int i;
  bool red;   // a red update after the first (over-relaxed)
};

template <int G>
__device__ __forceinline__ void corr2_load(const Nw32& p, int i, int j, int k,
                                           const __half2* const* H,
                                           const float4* __restrict__ rc,
                                           const float2* __restrict__ e2, int color, int first,
                                           Corr2In& in) {
  // the other colour's corrections are only read in this launch: read them
  // through the read-only path
  const Level& L = p.L;
  in.i = i;
  in.c = cidx32(L, i, j, k);
  ix nbi[6];
  gather6<G>(L, i, j, k, in.c, in.has, nbi);
  // the work arrays are colour-packed: own cell and the other colour's plane
  const RBIdx rb = rb_index(L, i, j, k);
  in.own = (ix)color * rb.plane + rb.pos;
  in.oth = (ix)(1 - color) * rb.plane + rb.pos;
  const ix sz = (ix)L.ny * rb.half;
  nbi[0] = in.oth - 1 + (i & 1);
  nbi[1] = in.oth + (i & 1);
  nbi[2] = in.oth - rb.half;
  nbi[3] = in.oth + rb.half;
  nbi[4] = in.oth - sz;
  nbi[5] = in.oth + sz;
  // every cell starts at zero in the first sweep
  const bool zero_nb = first && color == 0;
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const float2 v = (in.has[q] && !zero_nb) ? __ldg(e2 + nbi[q]) : make_float2(0.0f, 0.0f);
    in.enf[q] = v.x;
    in.enF[q] = v.y;
  }
  in.ec = first ? make_float2(0.0f, 0.0f) : e2[in.own];
  in.red = color == 0 && !first;
  faces6x2(L, H[0], H[1], H[2], i, j, k, in.has, in.Bf, in.BF);
  in.q4 = rc[in.own];
}

// The block Gauss-Seidel update of one cell's correction (e_f, e_F) from
// its flux sums (flf, flF), their diagonal weights (dgf, dgF) and its
// (r_f, r_F, u, v).  Every rounding is spelled out, so that each kernel
// that inlines it computes the same bits.
__device__ __forceinline__ float2 corr2_block(const Nw32& p, float4 q4, float2 ec, float2 fl,
                                              float2 dg) {
  const Jac2 J = jac2(p, q4.z, q4.w);
  // residuals of the correction equation at this cell, one lane per field:
  // r + flux - diag e + coupling e_other
  const float2 rho = v_fma(make_float2(J.fF, J.Ff), make_float2(ec.y, ec.x),
                           v_fma(make_float2(-J.ff, -J.FF), ec,
                                 v_add(make_float2(q4.x, q4.y), fl)));
  // 2x2 block solve: [a  -b; -d  e] [x; y] = [rhof; rhoF]
  const float2 ae = v_add(make_float2(J.ff, J.FF), dg);
  const float a = ae.x, bb = J.fF, d = J.Ff, e = ae.y;
  const float det = __fmaf_rn(a, e, -__fmul_rn(bb, d));
  const float inv = __fdividef(1.0f, det);
  return v_fma(v_fma(make_float2(e, d), v_bc(rho.x), v_mul(make_float2(bb, a), v_bc(rho.y))),
               v_bc(inv), ec);
}

template <int G>
__device__ __forceinline__ void corr2_apply(const Nw32& p, const Corr2In& in,
                                            float2* __restrict__ e2, float2* fst, float2* Fst,
                                            const float2* fsrc, const float2* Fsrc) {
  const Level& L = p.L;
  const float efc = in.ec.x, eFc = in.ec.y;
  float2 ne;
  if (G == SFX_CART3D) {
    float w[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) w[q] = in.has[q] ? 1.0f : 0.0f;
    float2 en[6], B[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      en[q] = make_float2(in.enf[q], in.enF[q]);
      B[q] = make_float2(in.Bf[q], in.BF[q]);
    }
    ne = corr3_cell(p, en, w, B, in.q4);
    // the old value is read here, not with the other loads: black launches
    // (the state update among them) never read it, and keeping it live
    // across the cell's arithmetic costs the two-plane kernel its overlap
    // of loads (at its register bound)
    if (in.red) ne = relax_red(p, ne, e2[in.own]);
  } else {
    // both fields in two lanes
    float2 en[6], B[6], dg;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      en[q] = make_float2(in.enf[q], in.enF[q]);
      B[q] = make_float2(in.Bf[q], in.BF[q]);
    }
    const float2 fl = flux_lin2<G>(L, p.invh, make_float2(p.Dfh, p.DFh), p.literal, in.i,
                                   make_float2(efc, eFc), en, in.has, B, dg);
    ne = corr2_block(p, in.q4, make_float2(efc, eFc), fl, dg);
    if (in.red) ne = relax_red(p, ne, in.ec);
  }
  const float nf = ne.x, nF = ne.y;
  e2[in.own] = make_float2(nf, nF);
  if (fst) {
    // last black colour of the iteration: the state becomes src + correction
    // (src = the state itself, or the advected x* in the first iteration,
    // which then needs no copy into the state), for this cell and for the
    // red cell that shares its pair (2t, 2t+1), which sits at the same
    // packed position of the other plane
    const ix c = in.c;
    fst[c] = df_add(fsrc[c], nf);
    Fst[c] = df_add(Fsrc[c], nF);
    const int ir = in.i ^ 1;
    if (ir < L.nx) {
      const ix cr = c - (ix)in.i + (ix)ir;
      const float2 er = __ldg(e2 + in.oth);
      fst[cr] = df_add(fsrc[cr], er.x);
      Fst[cr] = df_add(Fsrc[cr], er.y);
    }
  }
}

template <int G>
__device__ __forceinline__ void corr2_cell(const Nw32& p, int i, int j, int k,
                                           const __half2* const* H,
                                           const float4* __restrict__ rc,
                                           float2* __restrict__ e2, int color, int first,
                                           float2* fst, float2* Fst,
                                           const float2* fsrc, const float2* Fsrc) {
  Corr2In in;
  corr2_load<G>(p, i, j, k, H, rc, e2, color, first, in);
  corr2_apply<G>(p, in, e2, fst, Fst, fsrc, Fsrc);
}

// BCG update of one field at cell c: x + (-dt/V) sum of face fluxes,
// accumulated in area units so both cells of a face apply the same value.
__device__ __forceinline__ float2 advect_cell(const Adv32& A, const float2* __restrict__ x,
                                              float bc_in, size_t c) {
  const Level& L = A.L;
  int idx[3] = {(int)(c % L.nx), (int)((c / L.nx) % L.ny), (int)(c / ((size_t)L.nx * L.ny))};
  // net outflow in area units; each face term is computed bitwise alike
  // by the two cells that share the face
  float2 S = make_float2(0.0f, 0.0f);
  for (int d = 0; d < L.ndim(); ++d) {
    int pp[3] = {idx[0], idx[1], idx[2]};
    pp[d] += 1;
    float um = A.u[d][fidx(L, d, idx[0], idx[1], idx[2])];
    float up = A.u[d][fidx(L, d, pp[0], pp[1], pp[2])];
    float wm = d == 0 ? wr_face(L.geom, idx[0]) : (d == 1 ? wz_face(L.geom, idx[0]) : 1.0f);
    float wp = d == 0 ? wr_face(L.geom, idx[0] + 1) : wm;
    if (um != 0.0f) {
      float fv = face32v(A, x, bc_in, d, idx, um);
      float pr = __fmul_rn(um, fv);
      S = df_sub2(S, df_mul_f(make_float2(pr, fmaf(um, fv, -pr)), wm));
    }
    if (up != 0.0f) {
      float fv = face32v(A, x, bc_in, d, pp, up);
      float pr = __fmul_rn(up, fv);
      S = df_add2(S, df_mul_f(make_float2(pr, fmaf(up, fv, -pr)), wp));
    }
  }
  float2 inc = df_mul_f(df_mul_f(S, -A.dt), A.invh);
  if (L.geom == SFX_AXISYM) inc = df_div_f(inc, wz_face(L.geom, idx[0]));
  return df_add2(x[c], inc);
}

// A face's weighted pair fluxes (both fields) added to (plus face) or
// subtracted from (minus face) a cell's sums.
__device__ __forceinline__ void acc_face(float2& S1, float2& S2, float4 q, bool plus) {
  if (plus) {
    S1 = df_add2(S1, make_float2(q.x, q.y));
    S2 = df_add2(S2, make_float2(q.z, q.w));
  } else {
    S1 = df_sub2(S1, make_float2(q.x, q.y));
    S2 = df_sub2(S2, make_float2(q.z, q.w));
  }
}

// advect_cell for two fields sharing the face geometry (bitwise the same
// per field).
__device__ __forceinline__ void advect_cell2(const Adv32& A, const float2* __restrict__ x1,
                                             const float2* __restrict__ x2, float bc1, float bc2,
                                             int i, int j, int k, ix c, float2& o1,
                                             float2& o2) {
  const Level& L = A.L;
  int idx[3] = {i, j, k};
  float2 S1 = make_float2(0.0f, 0.0f), S2 = make_float2(0.0f, 0.0f);
  for (int d = 0; d < L.ndim(); ++d) {
    int pp[3] = {idx[0], idx[1], idx[2]};
    pp[d] += 1;
    const float um = A.u[d][fidx(L, d, idx[0], idx[1], idx[2])];
    const float up = A.u[d][fidx(L, d, pp[0], pp[1], pp[2])];
    const float wm = d == 0 ? wr_face(L.geom, idx[0]) : (d == 1 ? wz_face(L.geom, idx[0]) : 1.0f);
    const float wp = d == 0 ? wr_face(L.geom, idx[0] + 1) : wm;
    if (um != 0.0f) {
      float v1, v2;
      face32v2(A, x1, x2, bc1, bc2, d, idx, um, v1, v2);
      float pr = __fmul_rn(um, v1);
      S1 = df_sub2(S1, df_mul_f(make_float2(pr, fmaf(um, v1, -pr)), wm));
      pr = __fmul_rn(um, v2);
      S2 = df_sub2(S2, df_mul_f(make_float2(pr, fmaf(um, v2, -pr)), wm));
    }
    if (up != 0.0f) {
      float v1, v2;
      face32v2(A, x1, x2, bc1, bc2, d, pp, up, v1, v2);
      float pr = __fmul_rn(up, v1);
      S1 = df_add2(S1, df_mul_f(make_float2(pr, fmaf(up, v1, -pr)), wp));
      pr = __fmul_rn(up, v2);
      S2 = df_add2(S2, df_mul_f(make_float2(pr, fmaf(up, v2, -pr)), wp));
    }
  }
  float2 i1 = df_mul_f(df_mul_f(S1, -A.dt), A.invh);
  float2 i2 = df_mul_f(df_mul_f(S2, -A.dt), A.invh);
  if (L.geom == SFX_AXISYM) {
    i1 = df_div_f(i1, wz_face(L.geom, idx[0]));
    i2 = df_div_f(i2, wz_face(L.geom, idx[0]));
  }
  o1 = df_add2(x1[c], i1);
  o2 = df_add2(x2[c], i2);
}

}  // namespace
}  // namespace sfx
