// The cell of the FP32 Newton correction sweeps (3D) shared by the colour
// launch and the tiled sweep: the coefficients of the correction equation
// and its block Gauss-Seidel update in neighbour-coefficient form.
// Included by sfx_f32_dev.cuh (inside its namespaces).
#pragma once

struct Nw32 {
  Level L;
  float invh, Dfh, DFh, inv_dt, ka, kd, ginf, inv_eps, eta;
  int literal;
  // over-relaxation of the red updates after the first (relaxation
  // sweeps): e <- e + omega (e_GS - e) per field; 1 = Gauss-Seidel
  float om_f = 1.0f, om_F = 1.0f;
};

// Kinetic part of the pointwise 2x2 Jacobian of the App. C exchange at one
// cell, from u = c1 F and v = c1 (f_inf - f) (c1 = r_a/(phi + eta)):
//   [ff  -fF] = [1/dt + r_d + u    -v      ]
//   [-Ff  FF]   [-(u + r_d)        1/dt + v]
// (the flux operators add their diagonal weights to ff and FF).
struct Jac2 {
  float ff, fF, Ff, FF;
};
__device__ __forceinline__ Jac2 jac2(const Nw32& p, float u, float v) {
  return Jac2{__fadd_rn(__fadd_rn(p.inv_dt, p.kd), u), v, __fadd_rn(u, p.kd),
              __fadd_rn(p.inv_dt, v)};
}

// The 3D sweeps' flux of both fields' corrections in neighbour-coefficient
// form (the same linear operator as flux_lin, fewer instructions: no
// selects), one lane per field (x f, y F).  A face with drift B between
// cells L and R carries
//   G = D (e_R - e_L)/h + B e_up = (alpha e_R - beta e_L)/h,
//   alpha = D + max(B, 0), beta = D - min(B, 0)      (upwind on -B),
//   alpha = D + min(B, 0), beta = D - max(B, 0)      (literal: on +B),
// each from t = D +- |B|/2 and +-B/2 (exact halves) in FMA instructions.
// For a cell the plus faces' neighbours enter with alpha and the cell with
// beta, the minus faces' the other way round: the flux is
// (nbs - dg e_c)/h with nbs = sum of the neighbours' terms and dg the sum
// over open faces (w = 1) of the cell's terms.  A closed face's neighbour
// value is zero, so it adds nothing to nbs.  hs = +1/2 (upwind on -B) or
// -1/2 (literal).
__device__ __forceinline__ void nb3(float2 Doh, float hs, const float2* en, const float* w,
                                    const float2* B, float2& nbs, float2& dg) {
  float2 s = v_bc(0.0f), d = v_bc(0.0f);
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const float2 t = v_fma(v_bc(hs), make_float2(fabsf(B[q].x), fabsf(B[q].y)), Doh);
    const float2 al = v_fma(v_bc(0.5f), B[q], t), be = v_fma(v_bc(-0.5f), B[q], t);
    s = v_fma((q & 1) ? al : be, en[q], s);
    d = v_fma(v_bc(w[q]), (q & 1) ? be : al, d);
  }
  nbs = s;
  dg = d;
}

// The block Gauss-Seidel update of one 3D cell in the neighbour-coefficient
// form: the new correction solves the 2x2 system M e = r + (neighbour sums)
// directly (M = the exchange Jacobian plus the flux diagonals), so the
// cell's own old value does not enter.  nb, dg (f, F) already over h.
__device__ __forceinline__ float2 corr2_block_nb(const Nw32& p, float4 q4, float2 nb, float2 dg) {
  const Jac2 J = jac2(p, q4.z, q4.w);
  const float2 ae = v_add(make_float2(J.ff, J.FF), dg);   // (a, e)
  const float a = ae.x, bb = J.fF, d = J.Ff, e = ae.y;
  const float2 sv = v_add(make_float2(q4.x, q4.y), nb);   // (sf, sF)
  const float inv = __fdividef(1.0f, __fmaf_rn(a, e, -__fmul_rn(bb, d)));
  return v_mul(v_fma(make_float2(e, d), v_bc(sv.x), v_mul(make_float2(bb, a), v_bc(sv.y))),
               v_bc(inv));
}

// A red update over-relaxed from the cell's old value.  With black then
// red in each sweep, a mode whose Jacobi eigenvalue is mu is multiplied
// per sweep by 1 - omega (1 - mu^2); for mu^2 in [0, rho^2] the largest
// factor is smallest at omega = 2/(2 - rho^2): rho^2/(2 - rho^2) instead
// of Gauss-Seidel's rho^2.  omega = 1 leaves the Gauss-Seidel value.
__device__ __forceinline__ float2 relax_red(const Nw32& p, float2 gs, float2 old) {
  return make_float2(p.om_f == 1.0f ? gs.x : __fmaf_rn(p.om_f, __fsub_rn(gs.x, old.x), old.x),
                     p.om_F == 1.0f ? gs.y : __fmaf_rn(p.om_F, __fsub_rn(gs.y, old.y), old.y));
}

// One 3D correction cell from its gathered inputs (both sweeps of 3D
// grids, the colour launch and the tiled one, so they agree bit for bit).
__device__ __forceinline__ float2 corr3_cell(const Nw32& p, const float2* en, const float* w,
                                            const float2* B, float4 q4) {
  const float hs = p.literal ? -0.5f : 0.5f;
  float2 nb, dg;
  nb3(make_float2(p.Dfh, p.DFh), hs, en, w, B, nb, dg);
  return corr2_block_nb(p, q4, v_mul(nb, v_bc(p.invh)), v_mul(dg, v_bc(p.invh)));
}

