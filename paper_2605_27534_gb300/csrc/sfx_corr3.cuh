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

// The 3D sweeps' flux of one field's correction in neighbour-coefficient
// form (the same linear operator as flux_lin, fewer instructions: no
// selects).  A face with drift B between cells L and R carries
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
__device__ __forceinline__ void nb3(float Doh, float hs, const float* en, const float* w,
                                    const float* B, float& nbs, float& dg) {
  float s = 0.0f, d = 0.0f;
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const float t = __fmaf_rn(hs, fabsf(B[q]), Doh);
    const float al = __fmaf_rn(0.5f, B[q], t), be = __fmaf_rn(-0.5f, B[q], t);
    s = __fmaf_rn((q & 1) ? al : be, en[q], s);
    d = __fmaf_rn(w[q], (q & 1) ? be : al, d);
  }
  nbs = s;
  dg = d;
}

// The block Gauss-Seidel update of one 3D cell in the neighbour-coefficient
// form: the new correction solves the 2x2 system M e = r + (neighbour sums)
// directly (M = the exchange Jacobian plus the flux diagonals), so the
// cell's own old value does not enter.  nbf, nbF, dgf, dgF already over h.
__device__ __forceinline__ float2 corr2_block_nb(const Nw32& p, float4 q4, float nbf, float nbF,
                                                 float dgf, float dgF) {
  const Jac2 J = jac2(p, q4.z, q4.w);
  const float a = __fadd_rn(J.ff, dgf), bb = J.fF, d = J.Ff, e = __fadd_rn(J.FF, dgF);
  const float sf = __fadd_rn(q4.x, nbf), sF = __fadd_rn(q4.y, nbF);
  const float inv = __fdividef(1.0f, __fmaf_rn(a, e, -__fmul_rn(bb, d)));
  return make_float2(__fmul_rn(__fmaf_rn(e, sf, __fmul_rn(bb, sF)), inv),
                     __fmul_rn(__fmaf_rn(d, sf, __fmul_rn(a, sF)), inv));
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
__device__ __forceinline__ float2 corr3_cell(const Nw32& p, const float* enf, const float* enF,
                                            const float* w, const float* Bf, const float* BF,
                                            float4 q4) {
  const float hs = p.literal ? -0.5f : 0.5f;
  float nbf, nbF, dgf, dgF;
  nb3(p.Dfh, hs, enf, w, Bf, nbf, dgf);
  nb3(p.DFh, hs, enF, w, BF, nbF, dgF);
  return corr2_block_nb(p, q4, __fmul_rn(nbf, p.invh), __fmul_rn(nbF, p.invh),
                        __fmul_rn(dgf, p.invh), __fmul_rn(dgF, p.invh));
}

