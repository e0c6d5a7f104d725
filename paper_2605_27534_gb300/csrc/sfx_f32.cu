// SFX_F32 contexts: the coupled step in FP32 arithmetic with a double-float
// transported state.
//
// State.  f and F are double-float pairs (float2, value hi + lo).  Every
// residual is evaluated in pair arithmetic (FP32 instructions only) from
// FP32 coefficients, so the discrete operator is the FP64 one with its
// coefficients rounded to float (solution within ~1e-7), while residuals
// resolve ~1e-14 and the face terms cancel between the two cells of a face
// (totals conserved to pair precision).
// Phase field.  The caller passes the double phi.  The drift faces take
// the normal from FP64 differences of it (sfx_f32_dev.cuh, normal_f32); the
// per-iteration kernels read a float copy folded about 1/2 (phi if
// phi <= 1/2, phi - 1 otherwise) so that phi and 1 - phi both keep full
// relative precision.
//
// Solvers of the App. C system (SFX_TUNE_F32_SOLVER), with
//   r_f = (f* - f)/dt + div G_f + q,   r_F = (F* - F)/dt + div G_F - q,
//   q = r_a F/(phi+eta) (f_inf - f) - r_d f      (App. C),
//   G = D (a_R - a_L)/h + B a_up,  a_up upwinded on -B (Sec. 3.2 reading):
//  1 (default) coupled Newton defect correction: a pair residual pass also
//    forms the pointwise 2x2 exchange Jacobian; FP32 red-black sweeps with a
//    2x2 solve per cell relax the correction (their face drifts in half
//    precision, their work arrays colour-packed) and the last black colour
//    adds it to the state.  The convergence test runs on the device and
//    stops every later launch of the solve; the host reads it one iteration
//    late without draining the stream.
//  2 the same with the two fields linearised alternately (Picard).
//  0 nonlinear red-black Gauss-Seidel on the pair state, f and F sweeps in
//    turn, each cell taking a_c += r_c/diag_c.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "sfx_df.cuh"
#include "sfx_f32_dev.cuh"
#include "sfx_internal.h"
#include "sfx_tiled.cuh"
#include "sfx_advect3.cuh"

namespace sfx {
namespace {

// Drift faces of direction d in float (Bf, BF, B2) and half (H2) precision;
// Hm (may be null): the half pair again, at the colour-packed position of
// the cell whose minus side the face is (the layout of the tiled sweep,
// nx even; the far wall's faces have no such cell and are not kept).
__global__ void k_drift32(Level L, int d, const double* __restrict__ phi, float Df, float DF,
                          float inv_eps, float* __restrict__ Bf, float* __restrict__ BF,
                          float2* __restrict__ B2, __half2* __restrict__ H2,
                          __half2* __restrict__ Hm) {
  size_t n = L.nface(d);
  int fx = L.nx + (d == 0), fy = L.ny + (d == 1);
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n;
       q += (size_t)gridDim.x * blockDim.x) {
    int i = (int)(q % fx), j = (int)((q / fx) % fy), k = (int)(q / ((size_t)fx * fy));
    int pos = d == 0 ? i : (d == 1 ? j : k);
    float bf = 0.0f, bF = 0.0f;
    if (pos > 0 && pos < L.extent(d)) {
      int li = i - (d == 0), lj = j - (d == 1), lk = k - (d == 2);
      const float sL = fold_phi(phi[cidx(L, li, lj, lk)]), sR = fold_phi(phi[cidx(L, i, j, k)]);
      const float nL = normal_f32(L, phi, li, lj, lk, d, inv_eps);
      const float nR = normal_f32(L, phi, i, j, k, d, inv_eps);
      drift_face(sL, sR, nL, nR, Df, DF, inv_eps, bf, bF);
    }
    Bf[q] = bf;
    BF[q] = bF;
    B2[q] = make_float2(bf, bF);
    const __half2 hv = __floats2half2_rn(bf, bF);
    H2[q] = hv;
    if (Hm && pos < L.extent(d)) {
      const size_t half = (size_t)(L.nx >> 1);
      Hm[(size_t)((i + j + k) & 1) * half * L.ny * L.nz + ((size_t)k * L.ny + j) * half + (i >> 1)] =
          hv;
    }
  }
}

// ------------------------------------------------------------ sweeps
template <int FIELD>
__device__ __forceinline__ float2 cell_update32(const Nl32& p, int i, float2 ac, const float2* nb,
                                                const bool* has, const float* B, float phis,
                                                float2 as, float2 ov, float& r_out,
                                                float& b_out) {
  const int geom = p.L.geom;
  Acc S{0.0f, 0.0f};
  float dg = 0.0f;
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    if (!has[q]) continue;
    const bool plus = q & 1;                     // plus face: this cell is the left one
    const bool upL = p.literal ? (B[q] > 0.0f) : (B[q] < 0.0f);
    float w = 1.0f;
    if (geom == SFX_AXISYM) w = q < 2 ? wr_face(geom, i + (plus ? 1 : 0)) : (q < 4 ? wz_face(geom, i) : 1.0f);
    float2 G = plus ? face_G(p.Doh, B[q], upL, ac, nb[q]) : face_G(p.Doh, B[q], upL, nb[q], ac);
    if (geom == SFX_AXISYM) G = lp_mul(G, w);
    if (plus) {
      acc_add(S, G);
      dg += w * (p.Doh - (upL ? B[q] : 0.0f));
    } else {
      acc_sub(S, G);
      dg += w * (p.Doh + (upL ? 0.0f : B[q]));
    }
  }
  const float wc = wz_face(geom, i);
  float2 flux = lp_mul(acc_get(S), p.invh);
  if (geom == SFX_AXISYM) flux = df_div_f(ef_fast_two_sum(flux.x, flux.y), wc);
  float diag = dg * p.invh;
  if (geom == SFX_AXISYM) diag = __fdividef(diag, wc);
  // exchange q = r_a F/(phi+eta) (f_inf - f) - r_d f, shared by both equations
  const PhiPair ph = unfold(phis);
  const float c1 = __fdividef(p.ka, ph.p + p.eta);
  const float finf = p.ginf * ph.p * ph.q * p.inv_eps;
  const float2 fv2 = FIELD == 0 ? ac : ov;
  const float2 Fv2 = FIELD == 0 ? ov : ac;
  float2 fd = ef_two_sum(finf, -fv2.x);
  fd.y = __fsub_rn(fd.y, fv2.y);
  float pr = __fmul_rn(Fv2.x, fd.x);
  float2 FF = make_float2(pr, fmaf(Fv2.y, fd.x, fmaf(Fv2.x, fd.y, fmaf(Fv2.x, fd.x, -pr))));
  const float2 ads = lp_mul(FF, c1);
  const float2 des = lp_mul(fv2, p.kd);
  // r = (a* - a)/dt + flux +- (ads - des)
  Acc R{0.0f, 0.0f};
  acc_add(R, lp_mul(lp_sub(as, ac), p.inv_dt));
  acc_add(R, flux);
  if (FIELD == 0) { acc_add(R, ads); acc_sub(R, des); }
  else { acc_sub(R, ads); acc_add(R, des); }
  const float r = __fadd_rn(R.hi, R.lo);
  if (FIELD == 0) {
    const float Fv = __fadd_rn(ov.x, ov.y);
    diag += p.inv_dt + p.kd + c1 * Fv;
    b_out = as.x * p.inv_dt + c1 * Fv * finf;
  } else {
    const float fv = __fadd_rn(ov.x, ov.y);
    diag += p.inv_dt + c1 * (finf - fv);
    b_out = as.x * p.inv_dt + p.kd * fv;
  }
  r_out = r;
  return df_add(ac, __fdividef(r, diag));
}

// Nonlinear red-black colour sweep of field FIELD (0: f, 1: F) on the
// double-float state.  norms (optional): max |r| and max |b| of the updated
// cells, as float bit patterns, in norms[2*FIELD], norms[2*FIELD+1].
template <int FIELD>
__global__ void k_nlgs32(Nl32 p, const float* __restrict__ phi, const float* __restrict__ Bx,
                         const float* __restrict__ By, const float* __restrict__ Bz, float2* a,
                         const float2* __restrict__ astar, const float2* __restrict__ other,
                         int color, unsigned int* norms) {
  const Level& L = p.L;
  const int j = blockIdx.y, k = blockIdx.z;
  const int i = 2 * (blockIdx.x * blockDim.x + threadIdx.x) + ((j + k + color) & 1);
  float rmax = 0.0f, bmax = 0.0f;
  if (i < L.nx) {
    const size_t c = cidx(L, i, j, k);
    const size_t sy = (size_t)L.nx, sz = (size_t)L.nx * L.ny;
    bool has[6] = {i > 0, i + 1 < L.nx, j > 0, j + 1 < L.ny,
                   L.geom == SFX_CART3D && k > 0, L.geom == SFX_CART3D && k + 1 < L.nz};
    const float2 z2 = make_float2(0.0f, 0.0f);
    float2 nb[6] = {has[0] ? a[c - 1] : z2, has[1] ? a[c + 1] : z2, has[2] ? a[c - sy] : z2,
                    has[3] ? a[c + sy] : z2, has[4] ? a[c - sz] : z2, has[5] ? a[c + sz] : z2};
    float B[6] = {has[0] ? Bx[fidx(L, 0, i, j, k)] : 0.0f, has[1] ? Bx[fidx(L, 0, i + 1, j, k)] : 0.0f,
                  has[2] ? By[fidx(L, 1, i, j, k)] : 0.0f, has[3] ? By[fidx(L, 1, i, j + 1, k)] : 0.0f,
                  has[4] ? Bz[fidx(L, 2, i, j, k)] : 0.0f, has[5] ? Bz[fidx(L, 2, i, j, k + 1)] : 0.0f};
    float r, b;
    a[c] = cell_update32<FIELD>(p, i, a[c], nb, has, B, phi[c], astar[c], other[c], r, b);
    rmax = fabsf(r);
    bmax = fabsf(b);
    if (!(rmax <= 3.0e38f)) rmax = __int_as_float(0x7f800000);  // NaN -> +inf
  }
  if (norms) {
    rmax = warp_max(rmax);
    bmax = warp_max(bmax);
    if ((threadIdx.x & 31) == 0) {
      atomicMax(&norms[2 * FIELD], fbits(rmax));
      atomicMax(&norms[2 * FIELD + 1], fbits(bmax));
    }
  }
}

// ------------------------------------------------------------ defect correction
// The App. C system is solved by defect correction: a streaming pass
// applies the previous correction (a <- a + e, pair arithmetic) and
// evaluates the exact residual r of the new state in pair arithmetic, with
// lambda, the diagonal of the linearised (Picard) problem; FP32 red-black
// Gauss-Seidel sweeps then solve  A e = r,  A e = lambda e - (1/V) sum +-A G(e),
// G(e) = D (e_R - e_L)/h + B e_up.  Convergence is tested on the exact
// residual of the current state.
template <int FIELD>
__global__ void k_resid32(Nl32 p, const float* __restrict__ phi, const float* __restrict__ Bx,
                          const float* __restrict__ By, const float* __restrict__ Bz,
                          const float2* __restrict__ ain, const float* __restrict__ e,
                          float2* __restrict__ aout, const float2* __restrict__ astar,
                          const float2* __restrict__ other, float* __restrict__ rr,
                          float* __restrict__ lam, unsigned int* norms) {
  const Level& L = p.L;
  const size_t n = L.ncell();
  const size_t sy = (size_t)L.nx, sz = (size_t)L.nx * L.ny;
  float rmax = 0.0f, bmax = 0.0f;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(c % L.nx), j = (int)((c / L.nx) % L.ny), k = (int)(c / sz);
    bool has[6] = {i > 0, i + 1 < L.nx, j > 0, j + 1 < L.ny,
                   L.geom == SFX_CART3D && k > 0, L.geom == SFX_CART3D && k + 1 < L.nz};
    const size_t nbi[6] = {c - 1, c + 1, c - sy, c + sy, c - sz, c + sz};
    float2 nb[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      nb[q] = make_float2(0.0f, 0.0f);
      if (has[q]) nb[q] = e ? df_add(ain[nbi[q]], e[nbi[q]]) : ain[nbi[q]];
    }
    const float2 ac = e ? df_add(ain[c], e[c]) : ain[c];
    float B[6] = {has[0] ? Bx[fidx(L, 0, i, j, k)] : 0.0f, has[1] ? Bx[fidx(L, 0, i + 1, j, k)] : 0.0f,
                  has[2] ? By[fidx(L, 1, i, j, k)] : 0.0f, has[3] ? By[fidx(L, 1, i, j + 1, k)] : 0.0f,
                  has[4] ? Bz[fidx(L, 2, i, j, k)] : 0.0f, has[5] ? Bz[fidx(L, 2, i, j, k + 1)] : 0.0f};
    // residual and the kinetic part of the diagonal
    float r, b;
    const PhiPair ph = unfold(phi[c]);
    const float c1 = __fdividef(p.ka, ph.p + p.eta);
    const float finf = p.ginf * ph.p * ph.q * p.inv_eps;
    const float ov = __fadd_rn(other[c].x, other[c].y);
    cell_update32<FIELD>(p, i, ac, nb, has, B, phi[c], astar[c], other[c], r, b);
    aout[c] = ac;
    rr[c] = r;
    lam[c] = FIELD == 0 ? p.inv_dt + p.kd + c1 * ov : p.inv_dt + c1 * (finf - ov);
    rmax = fmaxf(rmax, fabsf(r));
    bmax = fmaxf(bmax, fabsf(b));
    if (!(fabsf(r) <= 3.0e38f)) rmax = __int_as_float(0x7f800000);
  }
  if (norms) {
    rmax = warp_max(rmax);
    bmax = warp_max(bmax);
    if ((threadIdx.x & 31) == 0) {
      atomicMax(&norms[2 * FIELD], fbits(rmax));
      atomicMax(&norms[2 * FIELD + 1], fbits(bmax));
    }
  }
}

struct Corr32 {
  Level L;
  float invh, Doh;
  int literal;
};

// One colour of FP32 red-black Gauss-Seidel on A e = r.
__global__ void k_corr32(Corr32 p, const float* __restrict__ Bx, const float* __restrict__ By,
                         const float* __restrict__ Bz, const float* __restrict__ rr,
                         const float* __restrict__ lam, float* __restrict__ e, int color,
                         int first) {
  const Level& L = p.L;
  const int j = blockIdx.y, k = blockIdx.z;
  const int i = 2 * (blockIdx.x * blockDim.x + threadIdx.x) + ((j + k + color) & 1);
  if (i >= L.nx) return;
  const size_t c = cidx(L, i, j, k);
  const size_t sy = (size_t)L.nx, sz = (size_t)L.nx * L.ny;
  // the first red colour starts from e = 0 (no neighbour has been updated)
  const bool zero_nb = first && color == 0;
  bool has[6] = {i > 0, i + 1 < L.nx, j > 0, j + 1 < L.ny,
                 L.geom == SFX_CART3D && k > 0, L.geom == SFX_CART3D && k + 1 < L.nz};
  const size_t nbi[6] = {c - 1, c + 1, c - sy, c + sy, c - sz, c + sz};
  const float B[6] = {has[0] ? Bx[fidx(L, 0, i, j, k)] : 0.0f, has[1] ? Bx[fidx(L, 0, i + 1, j, k)] : 0.0f,
                      has[2] ? By[fidx(L, 1, i, j, k)] : 0.0f, has[3] ? By[fidx(L, 1, i, j + 1, k)] : 0.0f,
                      has[4] ? Bz[fidx(L, 2, i, j, k)] : 0.0f, has[5] ? Bz[fidx(L, 2, i, j, k + 1)] : 0.0f};
  // in the first sweep every cell starts at zero (the array holds the
  // previous iteration's correction until a colour overwrites it)
  const float ec = first ? 0.0f : e[c];
  float S = 0.0f, dg = 0.0f;
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    if (!has[q]) continue;
    const bool plus = q & 1;
    const bool upL = p.literal ? (B[q] > 0.0f) : (B[q] < 0.0f);
    float w = 1.0f;
    if (L.geom == SFX_AXISYM) w = q < 2 ? wr_face(L.geom, i + (plus ? 1 : 0)) : (q < 4 ? wz_face(L.geom, i) : 1.0f);
    const float en = zero_nb ? 0.0f : e[nbi[q]];
    const float eL = plus ? ec : en, eR = plus ? en : ec;
    const float G = p.Doh * (eR - eL) + B[q] * (upL ? eL : eR);
    if (plus) {
      S += w * G;
      dg += w * (p.Doh - (upL ? B[q] : 0.0f));
    } else {
      S -= w * G;
      dg += w * (p.Doh + (upL ? 0.0f : B[q]));
    }
  }
  const float wc = wz_face(L.geom, i);
  const float flux = S * p.invh / wc, dflux = dg * p.invh / wc;
  const float l = lam[c];
  const float rho = rr[c] + flux - l * ec;
  e[c] = ec + __fdividef(rho, l + dflux);
}

// ------------------------------------------------------------ coupled Newton
// Newton form of the defect correction: the residual pass evaluates both
// residuals at a common state (one shared exchange term q) together with the
// pointwise 2x2 Jacobian of the exchange, and the correction
//   [A_f + lam_f   -j_fF ] [e_f]   [r_f]
//   [-j_Ff   A_F + lam_F ] [e_F] = [r_F]
// (A = flux operator, lam_f = 1/dt + r_d + c1 F, lam_F = 1/dt + c1 (f_inf - f),
//  j_fF = c1 (f_inf - f), j_Ff = c1 F + r_d, c1 = r_a/(phi + eta))
// is relaxed by red-black Gauss-Seidel with a 2x2 solve per cell.  The
// alternating (Picard) linearisation converges slowly where c1 dt >> 1;
// the coupled one does not.
// Evaluate both residuals (pairs), the 2x2 exchange Jacobian and the
// norms at every cell of the current state.
template <int G>
__global__ void __launch_bounds__(256, 4)
k_resid2_32(Nw32 p, const float* __restrict__ phi, const float2* __restrict__ B2x,
            const float2* __restrict__ B2y, const float2* __restrict__ B2z,
            const float2* __restrict__ fin,
            const float2* __restrict__ Fin, const float2* __restrict__ fst,
            const float2* __restrict__ Fst, float4* __restrict__ rc,
            unsigned int* norms, float2* __restrict__ e2,
            const int* __restrict__ done, const int* __restrict__ mode) {
  if (resid_skip(done, mode, 1)) return;
  const Level& L = p.L;
  float m[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  const float2* B2[3] = {B2x, B2y, B2z};
  // blocks over (x chunk, rows); each block walks rows r = k ny + j
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const ix rows = (ix)L.ny * (ix)L.nz;
  for (ix r = blockIdx.y; r < rows; r += gridDim.y) {
    const int j = (int)(r % (ix)L.ny), k = (int)(r / (ix)L.ny);
    if (i < L.nx)
      resid2_cell<G>(p, i, j, k, r * (ix)L.nx + (ix)i, phi, B2, fin, Fin, fst, Fst, rc, m, e2);
  }
  if (norms) resid_norms(m, norms);
}

// The FP32 residual pass (resid32_cell), same launch shape and outputs.
template <int G>
__global__ void __launch_bounds__(256, 5)
k_resid32_fast(Nw32 p, const float* __restrict__ phi, const float2* __restrict__ B2x,
               const float2* __restrict__ B2y, const float2* __restrict__ B2z,
               const float2* __restrict__ fin, const float2* __restrict__ Fin,
               const float2* __restrict__ fst, const float2* __restrict__ Fst,
               float4* __restrict__ rc, unsigned int* norms, float2* __restrict__ e2,
               const int* __restrict__ done, const int* __restrict__ mode) {
  if (resid_skip(done, mode, 0)) return;
  const Level& L = p.L;
  float m[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  const float2* B2[3] = {B2x, B2y, B2z};
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const ix rows = (ix)L.ny * (ix)L.nz;
  for (ix r = blockIdx.y; r < rows; r += gridDim.y) {
    const int j = (int)(r % (ix)L.ny), k = (int)(r / (ix)L.ny);
    if (i < L.nx)
      resid32_cell<G>(p, i, j, k, r * (ix)L.nx + (ix)i, phi, B2, fin, Fin, fst, Fst, rc, m, e2);
  }
  if (norms) resid_norms(m, norms);
}

// The incremental FP32 residual pass (resid32_incr_cell): the residuals of
// the current state from the previous iteration's (rc) and the correction
// it added (E); same launch shape and other outputs.
template <int G>
__global__ void __launch_bounds__(256, 4)
k_resid32_incr(Nw32 p, const float* __restrict__ phi, const float2* __restrict__ B2x,
               const float2* __restrict__ B2y, const float2* __restrict__ B2z,
               const float2* __restrict__ E, float4* __restrict__ rc, unsigned int* norms,
               float2* __restrict__ e2, const int* __restrict__ done,
               const int* __restrict__ mode) {
  if (resid_skip(done, mode, 2)) return;
  const Level& L = p.L;
  float m[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  const float2* B2[3] = {B2x, B2y, B2z};
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const ix rows = (ix)L.ny * (ix)L.nz;
  for (ix r = blockIdx.y; r < rows; r += gridDim.y) {
    const int j = (int)(r % (ix)L.ny), k = (int)(r / (ix)L.ny);
    if (i < L.nx)
      resid32_incr_cell<G>(p, i, j, k, r * (ix)L.nx + (ix)i, phi, B2, E, rc, m, e2);
  }
  if (norms) resid_norms(m, norms);
}

// One colour of the coupled red-black Gauss-Seidel on the correction.
// Block (x chunk, j, k): one colour of one row per block.  With KP = 2 a
// thread also updates the same cell of plane k + gridDim.z (3D): two
// independent cells whose loads are in flight together.
template <int G, int KP>
__device__ __forceinline__ void corr2_row(const Nw32& p, const __half2* const* H,
                                          const float4* __restrict__ rc,
                                          float2* __restrict__ e2, int color, int first,
                                          float2* fst, float2* Fst, const float2* fsrc,
                                          const float2* Fsrc, int j, int k) {
  const Level& L = p.L;
  const int i = 2 * (blockIdx.x * blockDim.x + threadIdx.x) + ((j + k + color) & 1);
  if (i >= L.nx) {
    // a row of odd length: the last red cell has no black partner
    const int ir = i ^ 1;
    if (fst && ir < L.nx) {
      const size_t cr = cidx(L, ir, j, k);
      const RBIdx rb = rb_index(L, i, j, k);
      const size_t pr = (1 - color) * rb.plane + rb.pos;   // ir's packed slot
      const float2 er = e2[pr];
      fst[cr] = df_add(fsrc[cr], er.x);
      Fst[cr] = df_add(Fsrc[cr], er.y);
    }
    return;
  }
  corr2_cell<G>(p, i, j, k, H, rc, e2, color, first, fst, Fst, fsrc, Fsrc);
}

template <int G, int KP>
__global__ void __launch_bounds__(128, KP == 1 ? 10 : 8)
k_corr2_32(Nw32 p, const __half2* __restrict__ Hx, const __half2* __restrict__ Hy,
           const __half2* __restrict__ Hz, const float4* __restrict__ rc,
           float2* __restrict__ e2, int color, int first,
           float2* fst, float2* Fst, const float2* fsrc, const float2* Fsrc,
           const int* __restrict__ done) {
  if (done && *done) return;
  const int j = blockIdx.y, k = blockIdx.z;
  const __half2* H[3] = {Hx, Hy, Hz};
  if (KP == 1) {
    corr2_row<G, 1>(p, H, rc, e2, color, first, fst, Fst, fsrc, Fsrc, j, k);
    return;
  }
  // two planes: both cells' loads are issued before either cell's
  // arithmetic (rows of even length only; the odd-row tail goes cell by cell)
  const Level& L = p.L;
  const int k2 = k + (int)gridDim.z;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int i1 = 2 * t + ((j + k + color) & 1), i2 = 2 * t + ((j + k2 + color) & 1);
  if ((L.nx & 1) || k2 >= L.nz || i1 >= L.nx || i2 >= L.nx) {
    corr2_row<G, KP>(p, H, rc, e2, color, first, fst, Fst, fsrc, Fsrc, j, k);
    if (k2 < L.nz) corr2_row<G, KP>(p, H, rc, e2, color, first, fst, Fst, fsrc, Fsrc, j, k2);
    return;
  }
  Corr2In a, b;
  corr2_load<G>(p, i1, j, k, H, rc, e2, color, first, a);
  corr2_load<G>(p, i2, j, k2, H, rc, e2, color, first, b);
  corr2_apply<G>(p, a, e2, fst, Fst, fsrc, Fsrc);
  corr2_apply<G>(p, b, e2, fst, Fst, fsrc, Fsrc);
}

// The Newton kernels of one geometry (the branches on the geometry in the
// cell functions fold at compile time).
struct NewtonKernels {
  decltype(&k_resid2_32<SFX_CART3D>) resid;
  decltype(&k_resid32_fast<SFX_CART3D>) fast;
  decltype(&k_resid32_incr<SFX_CART3D>) incr;
  decltype(&k_corr2_32<SFX_CART3D, 1>) corr;
  int kp;   // planes per thread of the correction sweep
};
template <int G>
NewtonKernels newton_kernels_of() {
  return NewtonKernels{&k_resid2_32<G>, &k_resid32_fast<G>, &k_resid32_incr<G>,
                       &k_corr2_32<G, 1>, 1};
}
NewtonKernels newton_kernels(int geom, int kp) {
  switch (geom) {
    case SFX_AXISYM: return newton_kernels_of<SFX_AXISYM>();
    case SFX_PLANAR2D: return newton_kernels_of<SFX_PLANAR2D>();
    default:
      return NewtonKernels{&k_resid2_32<SFX_CART3D>, &k_resid32_fast<SFX_CART3D>,
                           &k_resid32_incr<SFX_CART3D>,
                           kp == 2 ? &k_corr2_32<SFX_CART3D, 2> : &k_corr2_32<SFX_CART3D, 1>,
                           kp == 2 ? 2 : 1};
  }
}

// ------------------------------------------------------------ fused sweep
// One full red-black sweep in a single launch.  A block owns a TXxTYxTZ
// tile; it stages the old state of the tile and a 2-cell halo in shared
// memory, recomputes the red updates on the tile and a 1-cell halo (red
// cells depend on old black values only, so every block obtains the same
// red values), then updates its black cells from the new red values and
// writes the tile to `aout`.  Bitwise the result of two colour launches.
template <int FIELD, int TX, int TY, int TZ>
__global__ void __launch_bounds__(256) k_nlrb32(Nl32 p, const float* __restrict__ phi,
                                                const float* __restrict__ Bx,
                                                const float* __restrict__ By,
                                                const float* __restrict__ Bz,
                                                const float2* __restrict__ ain,
                                                float2* __restrict__ aout,
                                                const float2* __restrict__ astar,
                                                const float2* __restrict__ other,
                                                unsigned int* norms) {
  constexpr int HZ = TZ > 1 ? 2 : 0;           // no z halo in 2D
  constexpr int SX = TX + 4, SY = TY + 4, SZ = TZ + 2 * HZ;
  __shared__ float2 sa[SX * SY * SZ];
  const Level& L = p.L;
  const int ox = blockIdx.x * TX, oy = blockIdx.y * TY, oz = blockIdx.z * TZ;
  const int nthr = blockDim.x;
  const int tid = threadIdx.x;
  const size_t sy_g = (size_t)L.nx, sz_g = (size_t)L.nx * L.ny;
  // stage the old state (tile + 2-cell halo)
  for (int q = tid; q < SX * SY * SZ; q += nthr) {
    int li = q % SX - 2, lj = (q / SX) % SY - 2, lk = q / (SX * SY) - HZ;
    int gi = ox + li, gj = oy + lj, gk = oz + lk;
    float2 v = make_float2(0.0f, 0.0f);
    if (gi >= 0 && gi < L.nx && gj >= 0 && gj < L.ny && gk >= 0 && gk < L.nz)
      v = ain[(size_t)gk * sz_g + (size_t)gj * sy_g + gi];
    sa[q] = v;
  }
  __syncthreads();
  const int HZ1 = TZ > 1 ? 1 : 0;
  float rmax = 0.0f, bmax = 0.0f;
  for (int color = 0; color < 2; ++color) {
    // red: tile + 1-cell halo; black: tile only
    const int ex = color == 0 ? 1 : 0, ez = color == 0 ? HZ1 : 0;
    const int RX = TX + 2 * ex, RY = TY + 2 * ex, RZ = TZ + 2 * ez;
    for (int q = tid; q < RX * RY * RZ; q += nthr) {
      int li = q % RX - ex, lj = (q / RX) % RY - ex, lk = q / (RX * RY) - ez;
      int gi = ox + li, gj = oy + lj, gk = oz + lk;
      if (gi < 0 || gi >= L.nx || gj < 0 || gj >= L.ny || gk < 0 || gk >= L.nz) continue;
      if (((gi + gj + gk) & 1) != color) continue;
      const int sc = ((lk + HZ) * SY + (lj + 2)) * SX + (li + 2);
      const size_t c = (size_t)gk * sz_g + (size_t)gj * sy_g + gi;
      bool has[6] = {gi > 0, gi + 1 < L.nx, gj > 0, gj + 1 < L.ny, gk > 0, gk + 1 < L.nz};
      float2 nb[6] = {sa[sc - 1], sa[sc + 1], sa[sc - SX], sa[sc + SX], make_float2(0.f, 0.f),
                      make_float2(0.f, 0.f)};
      float B[6];
      B[0] = has[0] ? Bx[fidx(L, 0, gi, gj, gk)] : 0.0f;
      B[1] = has[1] ? Bx[fidx(L, 0, gi + 1, gj, gk)] : 0.0f;
      B[2] = has[2] ? By[fidx(L, 1, gi, gj, gk)] : 0.0f;
      B[3] = has[3] ? By[fidx(L, 1, gi, gj + 1, gk)] : 0.0f;
      if (TZ > 1) {
        nb[4] = sa[sc - SX * SY];
        nb[5] = sa[sc + SX * SY];
        B[4] = has[4] ? Bz[fidx(L, 2, gi, gj, gk)] : 0.0f;
        B[5] = has[5] ? Bz[fidx(L, 2, gi, gj, gk + 1)] : 0.0f;
      } else {
        has[4] = has[5] = false;
        B[4] = B[5] = 0.0f;
      }
      float r, b;
      const float2 nv = cell_update32<FIELD>(p, gi, sa[sc], nb, has, B, phi[c], astar[c],
                                             other[c], r, b);
      sa[sc] = nv;   // red cells read only black values, black only red
      const bool own = li >= 0 && li < TX && lj >= 0 && lj < TY && lk >= 0 && lk < TZ;
      if (own) {
        rmax = fmaxf(rmax, fabsf(r));
        bmax = fmaxf(bmax, fabsf(b));
        if (!(fabsf(r) <= 3.0e38f)) rmax = __int_as_float(0x7f800000);
      }
    }
    __syncthreads();
  }
  // write the tile
  for (int q = tid; q < TX * TY * TZ; q += nthr) {
    int li = q % TX, lj = (q / TX) % TY, lk = q / (TX * TY);
    int gi = ox + li, gj = oy + lj, gk = oz + lk;
    if (gi >= L.nx || gj >= L.ny || gk >= L.nz) continue;
    aout[(size_t)gk * sz_g + (size_t)gj * sy_g + gi] = sa[((lk + HZ) * SY + (lj + 2)) * SX + (li + 2)];
  }
  if (norms) {
    rmax = warp_max(rmax);
    bmax = warp_max(bmax);
    if ((tid & 31) == 0) {
      atomicMax(&norms[2 * FIELD], fbits(rmax));
      atomicMax(&norms[2 * FIELD + 1], fbits(bmax));
    }
  }
}

// 3D sweep marching in z with asynchronous staging.  A block owns a
// ZTX x ZTY column tile and a chunk of planes [z0, z1).  Shared memory holds
// a ring of ZNS state planes (old values, 2-cell xy halo) and a ring of ZNC
// coefficient planes (a*, the other field, phi and the six drift faces of
// every cell of the tile plus a 1-cell halo).  Step k: copies of state plane
// k+3 and coefficient plane k+2 are issued with cp.async; meanwhile the red
// cells of plane k+1 (tile + halo; they read old black values only) and
// then the black cells of plane k (they read the new red values of planes
// k-1..k+1) are updated from shared memory, and plane k of the tile is
// written out.  Bitwise the result of two colour launches.
constexpr int ZTX = 64, ZTY = 8;
constexpr int ZSX = ZTX + 4, ZSY = ZTY + 4;      // state plane with 2-cell halo
constexpr int ZCX = ZTX + 2, ZCY = ZTY + 2;      // coefficient plane, 1-cell halo
constexpr int ZNS = 5, ZNC = 3;

struct ZCoef {
  float2 as[ZCY][ZCX];
  float2 ot[ZCY][ZCX];
  float ph[ZCY][ZCX];
  float bx[ZCY][ZCX + 1];   // x-face on the minus side of cell x (x+1: plus side)
  float by[ZCY + 1][ZCX];   // y-face on the minus side of row y
  float bzl[ZCY][ZCX];      // z-faces below and above the plane
  float bzh[ZCY][ZCX];
};

struct ZSmem {
  float2 st[ZNS][ZSY][ZSX];
  ZCoef cf[ZNC];
};


template <int FIELD>
__global__ void __launch_bounds__(256) k_nlrb32_z(Nl32 p, const float* __restrict__ phi,
                                                  const float* __restrict__ Bx,
                                                  const float* __restrict__ By,
                                                  const float* __restrict__ Bz,
                                                  const float2* __restrict__ ain,
                                                  float2* __restrict__ aout,
                                                  const float2* __restrict__ astar,
                                                  const float2* __restrict__ other, int zchunk,
                                                  unsigned int* norms) {
  extern __shared__ __align__(16) unsigned char zsm_raw[];
  ZSmem& S = *reinterpret_cast<ZSmem*>(zsm_raw);
  const Level& L = p.L;
  const int ox = blockIdx.x * ZTX, oy = blockIdx.y * ZTY;
  const int z0 = blockIdx.z * zchunk, z1 = min(z0 + zchunk, L.nz);
  const int tid = threadIdx.x, nth = blockDim.x;
  const size_t pl = (size_t)L.nx * L.ny;
  float rmax = 0.0f, bmax = 0.0f;

  auto sslot = [](int gk) { return (gk + 4 * ZNS) % ZNS; };
  auto cslot = [](int gk) { return (gk + 4 * ZNC) % ZNC; };

  // issue the copies of state plane gk (zeros outside the domain)
  auto stage_state = [&](int gk) {
    if (gk < 0 || gk >= L.nz) return;
    float2(*st)[ZSX] = S.st[sslot(gk)];
    for (int q = tid; q < ZSX * ZSY; q += nth) {
      int x = q % ZSX, y = q / ZSX;
      int gi = ox + x - 2, gj = oy + y - 2;
      if (gi >= 0 && gi < L.nx && gj >= 0 && gj < L.ny)
        cp_async8(&st[y][x], &ain[gk * pl + (size_t)gj * L.nx + gi]);
      else
        st[y][x] = make_float2(0.0f, 0.0f);
    }
  };
  // issue the copies of coefficient plane gk (tile + 1-cell halo)
  auto stage_coef = [&](int gk) {
    if (gk < 0 || gk >= L.nz) return;
    ZCoef& C = S.cf[cslot(gk)];
    for (int q = tid; q < ZCX * ZCY; q += nth) {
      int x = q % ZCX, y = q / ZCX;
      int gi = ox + x - 1, gj = oy + y - 1;
      if (gi < 0 || gi >= L.nx || gj < 0 || gj >= L.ny) continue;
      size_t c = gk * pl + (size_t)gj * L.nx + gi;
      cp_async8(&C.as[y][x], &astar[c]);
      cp_async8(&C.ot[y][x], &other[c]);
      cp_async4(&C.ph[y][x], &phi[c]);
      cp_async4(&C.bx[y][x], &Bx[fidx(L, 0, gi, gj, gk)]);
      cp_async4(&C.by[y][x], &By[fidx(L, 1, gi, gj, gk)]);
      cp_async4(&C.bzl[y][x], &Bz[fidx(L, 2, gi, gj, gk)]);
      cp_async4(&C.bzh[y][x], &Bz[fidx(L, 2, gi, gj, gk + 1)]);
      if (x == ZCX - 1 || gi == L.nx - 1) cp_async4(&C.bx[y][x + 1], &Bx[fidx(L, 0, gi + 1, gj, gk)]);
      if (y == ZCY - 1 || gj == L.ny - 1) cp_async4(&C.by[y + 1][x], &By[fidx(L, 1, gi, gj + 1, gk)]);
    }
  };
  // update one cell of plane gk at tile coordinates (li, lj); sm/s0/sp are
  // the state planes gk-1, gk, gk+1 and C the coefficients of plane gk
  auto update = [&](float2 (*sm)[ZSX], float2 (*s0)[ZSX], float2 (*sp)[ZSX], const ZCoef& C,
                    int gk, int li, int lj, bool own) {
    const int gi = ox + li, gj = oy + lj;
    const int x = li + 2, y = lj + 2, cx = li + 1, cy = lj + 1;
    bool has[6] = {gi > 0, gi + 1 < L.nx, gj > 0, gj + 1 < L.ny, gk > 0, gk + 1 < L.nz};
    float2 nb[6] = {s0[y][x - 1], s0[y][x + 1], s0[y - 1][x], s0[y + 1][x], sm[y][x], sp[y][x]};
    float B[6] = {C.bx[cy][cx], C.bx[cy][cx + 1], C.by[cy][cx], C.by[cy + 1][cx], C.bzl[cy][cx],
                  C.bzh[cy][cx]};
    float r, b;
    s0[y][x] = cell_update32<FIELD>(p, gi, s0[y][x], nb, has, B, C.ph[cy][cx], C.as[cy][cx],
                                    C.ot[cy][cx], r, b);
    if (own) {
      rmax = fmaxf(rmax, fabsf(r));
      bmax = fmaxf(bmax, fabsf(b));
      if (!(fabsf(r) <= 3.0e38f)) rmax = __int_as_float(0x7f800000);
    }
  };
  // red cells of plane gk on the tile and a 1-cell halo
  auto red_plane = [&](int gk) {
    if (gk < 0 || gk >= L.nz) return;
    const bool own_plane = gk >= z0 && gk < z1;
    float2(*sm)[ZSX] = S.st[sslot(gk - 1)];
    float2(*s0)[ZSX] = S.st[sslot(gk)];
    float2(*sp)[ZSX] = S.st[sslot(gk + 1)];
    const ZCoef& C = S.cf[cslot(gk)];
    const int par = (ox - 1 + oy + gk) & 1;   // colour parity of cell (ox-1, oy) ...
    constexpr int HALF = ZCX / 2, NR = HALF * ZCY;
    for (int q = tid; q < NR; q += nth) {
      int lj = q / HALF - 1, gj = oy + lj;
      int li = -1 + 2 * (q % HALF) + ((par + lj) & 1);   // ... shifted by the row
      int gi = ox + li;
      if (li > ZTX || gi < 0 || gi >= L.nx || gj < 0 || gj >= L.ny) continue;
      update(sm, s0, sp, C, gk, li, lj, own_plane && li >= 0 && li < ZTX && lj >= 0 && lj < ZTY);
    }
  };
  // black cells of plane gk on the tile
  auto black_plane = [&](int gk) {
    float2(*sm)[ZSX] = S.st[sslot(gk - 1)];
    float2(*s0)[ZSX] = S.st[sslot(gk)];
    float2(*sp)[ZSX] = S.st[sslot(gk + 1)];
    const ZCoef& C = S.cf[cslot(gk)];
    const int par = (ox + oy + gk + 1) & 1;
    constexpr int HALF = ZTX / 2, NB = HALF * ZTY;
    for (int q = tid; q < NB; q += nth) {
      int lj = q / HALF, gj = oy + lj;
      int li = 2 * (q % HALF) + ((par + lj) & 1);
      int gi = ox + li;
      if (gi >= L.nx || gj >= L.ny) continue;
      update(sm, s0, sp, C, gk, li, lj, true);
    }
  };
  auto store_plane = [&](int gk) {
    float2(*s0)[ZSX] = S.st[sslot(gk)];
    for (int q = tid; q < ZTX * ZTY; q += nth) {
      int li = q % ZTX, lj = q / ZTX;
      int gi = ox + li, gj = oy + lj;
      if (gi < L.nx && gj < L.ny) aout[gk * pl + (size_t)gj * L.nx + gi] = s0[lj + 2][li + 2];
    }
  };

  // prologue: state z0-2..z0+2, coefficients z0-1..z0+1, red of z0-1 and z0
  for (int d = -2; d <= 2; ++d) stage_state(z0 + d);
  for (int d = -1; d <= 1; ++d) stage_coef(z0 + d);
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();
  red_plane(z0 - 1);
  __syncthreads();
  red_plane(z0);
  __syncthreads();
  for (int k = z0; k < z1; ++k) {
    // slots of planes k-2 (state) and k-1 (coefficients) are free now
    stage_state(k + 3);
    stage_coef(k + 2);
    cp_async_commit();
    red_plane(k + 1);
    __syncthreads();
    black_plane(k);
    __syncthreads();
    store_plane(k);
    cp_async_wait_all();
    __syncthreads();
  }
  if (norms) {
    rmax = warp_max(rmax);
    bmax = warp_max(bmax);
    if ((tid & 31) == 0) {
      atomicMax(&norms[2 * FIELD], fbits(rmax));
      atomicMax(&norms[2 * FIELD + 1], fbits(bmax));
    }
  }
}

// ------------------------------------------------------------ advection
__global__ void k_advect32(Adv32 A, const float2* __restrict__ x, float bc_in,
                           float2* __restrict__ out) {
  const size_t n = A.L.ncell();
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x)
    out[c] = advect_cell(A, x, bc_in, c);
}

// Both fields in one pass with every face evaluated once.  A block owns a
// tile of (kAdvX - 1) x (kAdvY - 1) cells and walks up to kAdvZ planes.
// Thread (tx, ty) evaluates the x and y faces on the minus side of cell
// (i0 + tx, j0 + ty) of the current plane (the last column and row give the
// tile's plus faces) and shares them through shared memory; the z face on
// the plus side of its cell is carried into the next plane as that plane's
// minus face.  Each face term is the weighted pair flux w u v of
// advect_cell2 and the cell sums them in its order (minus then plus face,
// x, y, z), so the result is bitwise that of advect_cell2 (the batched
// kernels).
constexpr int kAdvX = 32, kAdvY = 8, kAdvZ = 8;

// weighted pair fluxes of one face for both fields: (f.hi, f.lo, F.hi, F.lo)
__device__ __forceinline__ float4 face_flux2(const Adv32& A, const float2* __restrict__ x1,
                                             const float2* __restrict__ x2, float bc1, float bc2,
                                             int d, int* fc, float u, float w) {
  if (u == 0.0f) return make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  float v1, v2;
  face32v2(A, x1, x2, bc1, bc2, d, fc, u, v1, v2);
  float pr = __fmul_rn(u, v1);
  const float2 a = df_mul_f(make_float2(pr, fmaf(u, v1, -pr)), w);
  pr = __fmul_rn(u, v2);
  const float2 b = df_mul_f(make_float2(pr, fmaf(u, v2, -pr)), w);
  return make_float4(a.x, a.y, b.x, b.y);
}


__global__ void __launch_bounds__(kAdvX* kAdvY)
    k_advect2t_32(Adv32 A, const float2* __restrict__ f, const float2* __restrict__ F,
                  float bc_f, float bc_F, float2* __restrict__ fo, float2* __restrict__ Fo) {
  __shared__ float4 sx[kAdvY][kAdvX];
  __shared__ float4 sy[kAdvY][kAdvX];
  const Level& L = A.L;
  const int tx = threadIdx.x % kAdvX, ty = threadIdx.x / kAdvX;
  const int i = blockIdx.x * (kAdvX - 1) + tx, j = blockIdx.y * (kAdvY - 1) + ty;
  const bool is3d = L.geom == SFX_CART3D;
  const int k0 = is3d ? blockIdx.z * kAdvZ : 0;
  const int k1 = is3d ? min(k0 + kAdvZ, L.nz) : 1;
  const bool cell = tx < kAdvX - 1 && ty < kAdvY - 1 && i < L.nx && j < L.ny;
  const float wxm = wr_face(L.geom, i), wy = wz_face(L.geom, i);
  float4 zm = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  float uzm = 0.0f;
  if (is3d && cell) {
    int fcz[3] = {i, j, k0};
    uzm = A.u[2][cidx32(L, i, j, k0)];
    zm = face_flux2(A, f, F, bc_f, bc_F, 2, fcz, uzm, 1.0f);
  }
  for (int k = k0; k < k1; ++k) {
    float4 qx = make_float4(0.0f, 0.0f, 0.0f, 0.0f), qy = qx;
    if (i <= L.nx && j < L.ny) {
      int fcx[3] = {i, j, k};
      qx = face_flux2(A, f, F, bc_f, bc_F, 0, fcx, A.u[0][fidx32(L, 0, i, j, k)], wxm);
    }
    if (i < L.nx && j <= L.ny) {
      int fcy[3] = {i, j, k};
      qy = face_flux2(A, f, F, bc_f, bc_F, 1, fcy, A.u[1][fidx32(L, 1, i, j, k)], wy);
    }
    sx[ty][tx] = qx;
    sy[ty][tx] = qy;
    __syncthreads();
    if (cell) {
      float2 S1 = make_float2(0.0f, 0.0f), S2 = S1;
      const float uxm = A.u[0][fidx32(L, 0, i, j, k)], uxp = A.u[0][fidx32(L, 0, i + 1, j, k)];
      const float uym = A.u[1][fidx32(L, 1, i, j, k)], uyp = A.u[1][fidx32(L, 1, i, j + 1, k)];
      if (uxm != 0.0f) acc_face(S1, S2, sx[ty][tx], false);
      if (uxp != 0.0f) acc_face(S1, S2, sx[ty][tx + 1], true);
      if (uym != 0.0f) acc_face(S1, S2, sy[ty][tx], false);
      if (uyp != 0.0f) acc_face(S1, S2, sy[ty + 1][tx], true);
      if (is3d) {
        int fcz[3] = {i, j, k + 1};
        const float uzp = A.u[2][fidx32(L, 2, i, j, k + 1)];
        const float4 zp = face_flux2(A, f, F, bc_f, bc_F, 2, fcz, uzp, 1.0f);
        if (uzm != 0.0f) acc_face(S1, S2, zm, false);
        if (uzp != 0.0f) acc_face(S1, S2, zp, true);
        zm = zp;
        uzm = uzp;
      }
      float2 i1 = df_mul_f(df_mul_f(S1, -A.dt), A.invh);
      float2 i2 = df_mul_f(df_mul_f(S2, -A.dt), A.invh);
      if (L.geom == SFX_AXISYM) {
        i1 = df_div_f(i1, wz_face(L.geom, i));
        i2 = df_div_f(i2, wz_face(L.geom, i));
      }
      const ix c = cidx32(L, i, j, k);
      fo[c] = df_add2(f[c], i1);
      Fo[c] = df_add2(F[c], i2);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------ totals
// Per-thread double-float accumulation of w_i (hi + lo) with w_i the cell
// volume over its constant factor (1, or 2i+1 on rings); FP64 only across
// threads.
__global__ void k_total32_partials(Level L, const float2* __restrict__ x0,
                                   const float2* __restrict__ x1, int f0,
                                   double* __restrict__ partials) {
  // blockIdx.y picks the field: both fields' blocks in flight together
  const float2* __restrict__ x = blockIdx.y ? x1 : x0;
  const int fi = f0 + (int)blockIdx.y;
  const size_t n = L.ncell();
  // four independent pair accumulators: four loads in flight per thread
  float2 acc[4] = {make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f),
                   make_float2(0.0f, 0.0f)};
  const size_t step = (size_t)gridDim.x * blockDim.x;
  size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  auto weighted = [&](size_t cq) {
    float2 v = x[cq];
    if (L.geom == SFX_AXISYM) {
      float w = 2.0f * (float)(cq % L.nx) + 1.0f;
      float p = v.x * w;
      float e = fmaf(v.x, w, -p);               // exact product error
      v = make_float2(p, e + v.y * w);
    }
    return v;
  };
  // full groups of four without bounds checks (their loads issue together),
  // then the remainder
  for (; c + 3 * step < n; c += 4 * step) {
    float2 v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = weighted(c + (size_t)q * step);
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] = df_add2(acc[q], v[q]);
  }
  for (int q = 0; c < n; c += step, ++q) acc[q & 3] = df_add2(acc[q & 3], weighted(c));
  // each pair is exact in FP64 (hi + lo spans < 53 bits); the four are
  // combined by compensated FP64 sums, then reduced across threads
  double s = (double)acc[0].x + (double)acc[0].y, cc = 0.0;
#pragma unroll
  for (int q = 1; q < 4; ++q) {
    double t, e;
    two_sum(s, (double)acc[q].x + (double)acc[q].y, t, e);
    s = t;
    cc += e;
  }
  warp_sum_comp(s, cc);
  __shared__ double ss[8], sc[8];
  int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { ss[w] = s; sc[w] = cc; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = ss[0], b = sc[0];
    for (int q = 1; q < (int)(blockDim.x >> 5); ++q) {
      double t, e;
      two_sum(a, ss[q], t, e);
      a = t;
      b += sc[q] + e;
    }
    partials[2 * ((size_t)fi * gridDim.x + blockIdx.x)] = a;
    partials[2 * ((size_t)fi * gridDim.x + blockIdx.x) + 1] = b;
  }
}

__global__ void k_total32_final(const double* __restrict__ partials, int nblk, double scale,
                                double* __restrict__ out) {
  const int fi = blockIdx.x;
  double s = 0.0, cc = 0.0;
  for (int q = threadIdx.x; q < nblk; q += blockDim.x) {
    double t, e;
    two_sum(s, partials[2 * ((size_t)fi * nblk + q)], t, e);
    s = t;
    cc += partials[2 * ((size_t)fi * nblk + q) + 1] + e;
  }
  warp_sum_comp(s, cc);
  __shared__ double ss[8], sc[8];
  int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { ss[w] = s; sc[w] = cc; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = ss[0], b = sc[0];
    for (int q = 1; q < (int)(blockDim.x >> 5); ++q) {
      double t, e;
      two_sum(a, ss[q], t, e);
      a = t;
      b += sc[q] + e;
    }
    out[fi] = (a + b) * scale;
  }
}

// ------------------------------------------------------------ EOS, force
struct Eos32 {
  float ginf, eps, inv_eps, sigma0, E;
  int eos;
  double ginf_d, eps_d, sigma0_d, E_d;   // the same in FP64 (near saturation)
};

// sigma - sigma0 (kept for the gradient, where it has full relative
// precision) and sigma itself.  Near saturation (Gamma/Gamma_inf > 1/2) the
// Langmuir term is formed in FP64 throughout: delta_phi from the double
// phi, Gamma from the whole double-float pair of f, 1 - Gamma/Gamma_inf and
// its logarithm, since float spacing in Gamma/Gamma_inf (6e-8) would be a
// large relative error of 1 - Gamma/Gamma_inf there.  FP32 below.
__global__ void k_eos32(size_t n, Eos32 q, const float2* __restrict__ f,
                        const double* __restrict__ phi, float* __restrict__ dsig,
                        float* __restrict__ sigma) {
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x) {
    PhiPair ph = unfold(fold_phi(phi[c]));
    float del = ph.p * ph.q * q.inv_eps;
    float G = del >= 1e-3f * q.inv_eps ? df_val(f[c]) / del : 0.0f;
    float x = G / q.ginf;
    float ds;
    if (q.eos == SFX_EOS_LANGMUIR) {
      if (x > 0.5f) {
        const double pd = phi[c];
        const double deld = pd * (1.0 - pd) / q.eps_d;
        const float2 fc = f[c];
        const double xd = ((double)fc.x + (double)fc.y) / deld / q.ginf_d;
        ds = (float)(q.sigma0_d * q.E_d * log1p(-fmin(xd, 1.0 - 1e-12)));
      } else {
        ds = q.sigma0 * q.E * log1pf(-x);
      }
    } else if (q.eos == SFX_EOS_LINEAR) {
      ds = -q.sigma0 * q.E * x;
    } else {
      ds = -q.sigma0 * tanhf(q.E * x);
    }
    dsig[c] = ds;
    if (sigma) sigma[c] = q.sigma0 + ds;
  }
}

struct VS32 {
  float v, dv;
};

// Unit-cube volume below m.x = a (ascending m, sum 1) and its slope, FP32
// version of the region-wise Scardovelli-Zaleski evaluation.
__device__ VS32 plic32_half(const float* q, bool three_d, float a) {
  VS32 r{0.0f, 0.0f};
  if (a <= 0.0f) return r;
  if (!three_d) {
    float lo = q[1], hi = q[2];
    if (a < lo) { r.v = 0.5f * a * a / (lo * hi); r.dv = a / (lo * hi); }
    else { r.v = (a - 0.5f * lo) / hi; r.dv = 1.0f / hi; }
    return r;
  }
  float p = q[0], s = q[1], t = q[2];
  float ist = 1.0f / (s * t);
  if (a < p) {
    r.v = a * a * a * ist / (6.0f * p);
    r.dv = 0.5f * a * a * ist / p;
  } else if (a < s) {
    r.v = 0.5f * (a * (a - p) + p * p / 3.0f) * ist;
    r.dv = (a - 0.5f * p) * ist;
  } else if (t >= p + s && a >= p + s) {
    r.v = (a - 0.5f * (p + s)) / t;
    r.dv = 1.0f / t;
  } else {
    float u = a - s, w = fmaxf(a - t, 0.0f);
    r.v = 0.5f * (a * (a - p) + p * p / 3.0f) * ist - (u * u * u + w * w * w) * ist / (6.0f * p);
    r.dv = (a - 0.5f * p) * ist - 0.5f * (u * u + w * w) * ist / p;
  }
  return r;
}

__device__ float plic32_area(int nd, const float* m, float C) {
  if (!(C > 0.0f && C < 1.0f)) return 0.0f;
  float s = 0.0f, q2 = 0.0f;
  for (int d = 0; d < nd; ++d) { s += fabsf(m[d]); q2 += m[d] * m[d]; }
  if (s == 0.0f) return 0.0f;
  float q[3] = {nd == 3 ? fabsf(m[2]) / s : 0.0f, fabsf(m[0]) / s, fabsf(m[1]) / s};
  if (q[0] > q[1]) { float t = q[0]; q[0] = q[1]; q[1] = t; }
  if (q[1] > q[2]) { float t = q[1]; q[1] = q[2]; q[2] = t; }
  if (q[0] > q[1]) { float t = q[0]; q[0] = q[1]; q[1] = t; }
  const bool three_d = nd == 3;
  const bool flip = C > 0.5f;             // V(a) = 1 - V(1 - a)
  const float target = flip ? 1.0f - C : C;
  float lo = 0.0f, hi = 0.5f;
  for (int it = 0; it < 30; ++it) {
    float mid = 0.5f * (lo + hi);
    if (plic32_half(q, three_d, mid).v < target) lo = mid;
    else hi = mid;
  }
  return sqrtf(q2) / s * plic32_half(q, three_d, 0.5f * (lo + hi)).dv;
}

// One cell of the Marangoni force (F32 context).  With dm_mode 1 only
// interface cells (1e-6 < C < 1 - 1e-6) carry a PLIC area, so every other
// cell's force is zero and skips the gradient and the normal.
__device__ __forceinline__ void force32_cell(const Level& L, const double* __restrict__ phi,
                                             const float* __restrict__ C,
                                             const float* __restrict__ dsig, int dm_mode,
                                             float inv_eps, int i, int j, int k, ix c, ix n,
                                             float* __restrict__ force) {
  const int nd = L.ndim();
  const float Cc = C[c];
  if (dm_mode != 0 && !(Cc > 1e-6f && Cc < 1.0f - 1e-6f)) {
    for (int d = 0; d < nd; ++d) force[(ix)d * n + c] = 0.0f;
    return;
  }
  const int idx[3] = {i, j, k};
  const float inv2h = 0.5f / (float)L.h;
  float gs[3] = {0, 0, 0}, nn[3], ndg = 0.0f;
  float gc2 = 0;
  for (int d = 0; d < nd; ++d) {
    int pp[3] = {idx[0], idx[1], idx[2]}, pm[3] = {idx[0], idx[1], idx[2]};
    pp[d] = min(pp[d] + 1, L.extent(d) - 1);
    pm[d] = max(pm[d] - 1, 0);
    const ix cp = cidx32(L, pp[0], pp[1], pp[2]), cm = cidx32(L, pm[0], pm[1], pm[2]);
    gs[d] = (dsig[cp] - dsig[cm]) * inv2h;
    if (dm_mode == 0) {
      float gc = (C[cp] - C[cm]) * inv2h;
      gc2 += gc * gc;
    }
  }
  normal3_f32(L, phi, idx[0], idx[1], idx[2], inv_eps, nn);
  for (int d = 0; d < nd; ++d) ndg += nn[d] * gs[d];
  float dm;
  if (dm_mode == 0) {
    dm = sqrtf(gc2);
  } else {
    float m[3] = {0, 0, 0};
    const int kr = nd == 3 ? 1 : 0;
    for (int dk = -kr; dk <= kr; ++dk)
      for (int dj = -1; dj <= 1; ++dj)
        for (int di = -1; di <= 1; ++di) {
          const int a = min(max(idx[0] + di, 0), L.nx - 1);
          const int b = min(max(idx[1] + dj, 0), L.ny - 1);
          const int e = min(max(idx[2] + dk, 0), L.nz - 1);
          const float w = (di == 0 ? 2.0f : 1.0f) * (dj == 0 ? 2.0f : 1.0f) *
                          (nd == 3 ? (dk == 0 ? 2.0f : 1.0f) : 1.0f);
          const float v = C[cidx32(L, a, b, e)];
          m[0] -= w * di * v;
          m[1] -= w * dj * v;
          m[2] -= w * dk * v;
        }
    dm = plic32_area(nd, m, Cc) / (float)L.h;
  }
  for (int d = 0; d < nd; ++d) force[(ix)d * n + c] = dm * (gs[d] - nn[d] * ndg);
}

// The rows r = k ny + j that a block of a row-walking kernel visits
// (blockIdx.y, then every gridDim.y-th), their (j, k) advanced by additions
// instead of a division per row.
struct RowWalk {
  int j, k, dj, dk, ny;
  __device__ __forceinline__ RowWalk(int ny_) : ny(ny_) {
    j = (int)(blockIdx.y % (unsigned)ny_);
    k = (int)(blockIdx.y / (unsigned)ny_);
    dj = (int)(gridDim.y % (unsigned)ny_);
    dk = (int)(gridDim.y / (unsigned)ny_);
  }
  __device__ __forceinline__ void next() {
    j += dj;
    k += dk;
    if (j >= ny) {
      j -= ny;
      ++k;
    }
  }
};

// blocks over (x chunk, rows); each block walks rows r = k ny + j
__global__ void k_force32(Level L, const double* __restrict__ phi, const float* __restrict__ C,
                          const float* __restrict__ dsig, int dm_mode, float inv_eps,
                          float* __restrict__ force) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L.nx) return;
  const ix rows = (ix)L.ny * (ix)L.nz, n = rows * (ix)L.nx;
  RowWalk w(L.ny);
  for (ix r = blockIdx.y; r < rows; r += gridDim.y, w.next()) {
    const int j = w.j, k = w.k;
    force32_cell(L, phi, C, dsig, dm_mode, inv_eps, i, j, k, r * (ix)L.nx + (ix)i, n, force);
  }
}

// ------------------------------------------------------------ conversions
__global__ void k_pack_df(size_t n, const double* __restrict__ in, float2* __restrict__ out) {
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x) {
    double d = in[c];
    float hi = (float)d;
    out[c] = make_float2(hi, (float)(d - (double)hi));
  }
}

__global__ void k_fold_phi(size_t n, const double* __restrict__ phi, float* __restrict__ out) {
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x) {
    double p = phi[c];
    out[c] = p <= 0.5 ? (float)p : (float)(p - 1.0);
  }
}

__global__ void k_unpack_df(size_t n, const float2* __restrict__ in, double* __restrict__ out) {
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x)
    out[c] = (double)in[c].x + (double)in[c].y;
}

// ------------------------------------------------------------ host
sfx_status sweep32(sfx_ctx* c, int field, const Nl32& p, const float* phi, const float* const* B,
                   float2* a, const float2* astar, const float2* other, bool norms,
                   cudaStream_t s) {
  const Level& L = p.L;
  dim3 blk(128), grd((unsigned)(((L.nx + 1) / 2 + 127) / 128), (unsigned)L.ny, (unsigned)L.nz);
  unsigned int* nb = norms ? (unsigned int*)c->d_norms : nullptr;
  for (int color = 0; color < 2; ++color) {
    if (field == 0)
      SFX_KERNEL(c, K_SMOOTH_FINE, k_nlgs32<0>, grd, blk, s, p, phi, B[0], B[1], B[2], a, astar,
                 other, color, nb);
    else
      SFX_KERNEL(c, K_SMOOTH_FINE, k_nlgs32<1>, grd, blk, s, p, phi, B[0], B[1], B[2], a, astar,
                 other, color, nb);
  }
  SFX_LAUNCH_CHECK();
  return SFX_OK;
}

template <int FIELD>
sfx_status fused_sweep32(sfx_ctx* c, const Nl32& p, const float* phi, const float* const* B,
                         const float2* ain, float2* aout, const float2* astar,
                         const float2* other, bool norms, cudaStream_t s) {
  const Level& L = p.L;
  unsigned int* nb = norms ? (unsigned int*)c->d_norms : nullptr;
  if (L.geom == SFX_CART3D) {
    const int zchunk = c->f32.zchunk;
    static bool attr_set[2] = {false, false};
    if (!attr_set[FIELD]) {
      SFX_CUDA(cudaFuncSetAttribute(k_nlrb32_z<FIELD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sizeof(ZSmem)));
      attr_set[FIELD] = true;
    }
    dim3 grd((unsigned)((L.nx + ZTX - 1) / ZTX), (unsigned)((L.ny + ZTY - 1) / ZTY),
             (unsigned)((L.nz + zchunk - 1) / zchunk));
    prof_before(c, K_SMOOTH_FINE, s);
    k_nlrb32_z<FIELD><<<grd, 256, sizeof(ZSmem), s>>>(p, phi, B[0], B[1], B[2], ain, aout, astar,
                                                       other, zchunk, nb);
    prof_after(c, K_SMOOTH_FINE, s);
  } else {
    dim3 grd((unsigned)((L.nx + 31) / 32), (unsigned)((L.ny + 15) / 16), 1);
    SFX_KERNEL(c, K_SMOOTH_FINE, (k_nlrb32<FIELD, 32, 16, 1>), grd, 256, s, p, phi, B[0], B[1],
               B[2], ain, aout, astar, other, nb);
  }
  SFX_LAUNCH_CHECK();
  return SFX_OK;
}

}  // namespace

sfx_status f32_ensure_scratch(sfx_ctx* c);

namespace {

sfx_status corr_sweeps(sfx_ctx* c, const Corr32& cp, const float* const* B, const float* r,
                       const float* lam, float* e, int sweeps, cudaStream_t s) {
  const Level& L = cp.L;
  dim3 blk(128), grd((unsigned)(((L.nx + 1) / 2 + 127) / 128), (unsigned)L.ny, (unsigned)L.nz);
  for (int q = 0; q < sweeps; ++q)
    for (int color = 0; color < 2; ++color)
      SFX_KERNEL(c, K_SMOOTH_FINE, k_corr32, grd, blk, s, cp, B[0], B[1], B[2], r, lam, e, color,
                 q == 0 ? 1 : 0);
  SFX_LAUNCH_CHECK();
  return SFX_OK;
}

// Defect-correction solve of the App. C system (see k_resid32).
sfx_status solve_dc32(sfx_ctx* c, const Nl32& pf, const Nl32& pF, const float* phi,
                      float* const* Bf, float* const* BF, float2*& fc, float2*& fo,
                      float2*& Fc, float2*& Fo, const float2* fs, const float2* Fs,
                      const sfx_solve_opts* o, int* iters, bool* conv, float* nrm,
                      cudaStream_t s) {
  const Level& L = pf.L;
  const size_t n = L.ncell();
  const int nb = blocks_for(n, 256);
  Corr32 cf{L, pf.invh, pf.Doh, pf.literal}, cF{L, pF.invh, pF.Doh, pF.literal};
  float* ef = c->f32.ef;
  float* eF = c->f32.eF;
  const int sweeps = std::max(1, o->nu1 + o->nu2);
  const int first = std::min(std::max(c->f32.predicted, 1), o->max_cycles);
  int it;
  *conv = false;
  for (it = 1; it <= o->max_cycles; ++it) {
    const bool check = (it >= first && (it - first) % o->check_every == 0) || it == o->max_cycles;
    unsigned int* nbuf = check ? (unsigned int*)c->d_norms : nullptr;
    if (check) SFX_CUDA(cudaMemsetAsync(c->d_norms, 0, 8 * sizeof(unsigned long long), s));
    SFX_KERNEL(c, K_RESIDUAL, k_resid32<0>, nb, 256, s, pf, phi, Bf[0], Bf[1], Bf[2], fc,
               it == 1 ? nullptr : ef, fo, fs, Fc, c->f32.rf, c->f32.lf, nbuf);
    std::swap(fc, fo);
    sfx_status st = corr_sweeps(c, cf, Bf, c->f32.rf, c->f32.lf, ef, sweeps, s);
    if (st != SFX_OK) return st;
    SFX_KERNEL(c, K_RESIDUAL, k_resid32<1>, nb, 256, s, pF, phi, BF[0], BF[1], BF[2], Fc,
               it == 1 ? nullptr : eF, Fo, Fs, fc, c->f32.rF, c->f32.lF, nbuf);
    std::swap(Fc, Fo);
    st = corr_sweeps(c, cF, BF, c->f32.rF, c->f32.lF, eF, sweeps, s);
    if (st != SFX_OK) return st;
    SFX_LAUNCH_CHECK();
    if (check) {
      SFX_CUDA(cudaMemcpyAsync(c->h_norms, c->d_norms, 2 * sizeof(unsigned long long),
                               cudaMemcpyDeviceToHost, s));
      SFX_CUDA(cudaStreamSynchronize(s));
      memcpy(nrm, c->h_norms, 4 * sizeof(float));
      for (int q = 0; q < 4; ++q)
        if (!std::isfinite(nrm[q])) return SFX_ERR_NONFINITE;
      if (nrm[0] <= o->tol * nrm[1] && nrm[2] <= o->tol * nrm[3]) {
        *conv = true;
        break;
      }
    }
  }
  *iters = std::min(it, o->max_cycles);
  c->f32.predicted = *conv ? (it == first ? it - 1 : it) : 0;
  return SFX_OK;
}

// Convergence test of one Newton iteration on the device: once both
// relative residuals pass, `flag[0]` stops every later launch of the solve
// and flag[1] records the iteration.
// A tiled sweep of the previous iteration that gave up waiting for its
// staged planes (flag[3]) marks the norms with kTimeoutBits instead.
// Residual kinds (flag[4]): 0 while the FP32 pass evaluates the residuals,
// 1 once the pair pass does, 2 when the incremental pass follows a pair
// pass (incr_ok: the solve keeps the previous correction).  The solve
// switches from FP32 to the pair pass after `fast_max` FP32 iterations
// (counted in flag[5]) or once both relative residuals are below
// kFastSwitch; from the pair to the incremental pass once both relative
// pair residuals are below kIncrFactor x tol: an incremental chain rounds
// to about 16 float epsilons (16 x 6e-8) of the pair residual it starts
// from, which then stays below a tenth of the tolerance.  Only a pair or an
// incremental residual passes the test; nrm[4] records the kind each
// iteration's norms came from.
constexpr unsigned int kTimeoutBits = 0xffffffffu;
constexpr float kFastSwitch = kFastResidSwitch;
constexpr float kIncrFactor = 1e5f;
__global__ void k_flag32(unsigned int* __restrict__ nrm, const unsigned int* __restrict__ prev,
                         float tol, int it, int fast_max, int incr_ok, int* __restrict__ flag) {
  if (threadIdx.x != 0 || flag[0]) return;
  if (flag[3]) {
    nrm[1] = nrm[3] = kTimeoutBits;
    return;
  }
  // an incremental pass reads neither the state nor x*: its scales are
  // those of the iteration before, back to the pair pass the chain began at
  if (flag[4] == 2) {
    nrm[1] = prev[1];
    nrm[3] = prev[3];
  }
  const float rf = __uint_as_float(nrm[0]), bf = __uint_as_float(nrm[1]);
  const float rF = __uint_as_float(nrm[2]), bF = __uint_as_float(nrm[3]);
  const int kind = flag[4];
  nrm[4] = (unsigned int)kind;
  if (kind >= 1) {
    if (rf <= tol * bf && rF <= tol * bF) {
      flag[0] = 1;
      flag[1] = it;
    } else if (kind == 1 && incr_ok && rf <= kIncrFactor * tol * bf &&
               rF <= kIncrFactor * tol * bF) {
      flag[4] = 2;
    }
  } else if (++flag[5] >= fast_max || (rf <= kFastSwitch * bf && rF <= kFastSwitch * bF)) {
    flag[4] = 1;
  }
}

__global__ void k_set32(int* __restrict__ p, int v) {
  if (threadIdx.x == 0) *p = v;
}

// A predicted start whose first relative residual exceeds `rho` (or is not
// finite) is rejected: ok = 0 and the norms are cleared for the residual
// pass of the restart from x*.
__global__ void k_pred_check32(unsigned int* __restrict__ nrm, float rho, int* __restrict__ ok) {
  if (threadIdx.x != 0) return;
  const float rf = __uint_as_float(nrm[0]), bf = __uint_as_float(nrm[1]);
  const float rF = __uint_as_float(nrm[2]), bF = __uint_as_float(nrm[3]);
  const bool good = rf <= rho * bf && rF <= rho * bF;   // false for NaN
  ok[0] = good ? 1 : 0;
  if (!good)
    for (int q = 0; q < 4; ++q) nrm[q] = 0u;
}

// Restart from x* when the prediction was rejected.
__global__ void k_restore32(size_t n, const int* __restrict__ ok, const float2* __restrict__ fs,
                            const float2* __restrict__ Fs, float2* __restrict__ f,
                            float2* __restrict__ F) {
  if (*ok) return;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x) {
    f[c] = fs[c];
    F[c] = Fs[c];
  }
}

// Initial guess of the Newton iteration: x* plus the implicit increment of
// the previous step (a smooth solution changes little from step to step).
// (f, F) <- (f*, F*) when the Newton solve converged at its first check
// (flag[1] = 1): its state updates then never ran.
__global__ void k_copy_if_first32(size_t n, const int* __restrict__ flag,
                                  const float2* __restrict__ fs, const float2* __restrict__ Fs,
                                  float2* __restrict__ f, float2* __restrict__ F) {
  if (!(flag[0] && flag[1] == 1)) return;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x) {
    f[c] = fs[c];
    F[c] = Fs[c];
  }
}
__global__ void k_predict32(size_t n, const float2* __restrict__ fs, const float2* __restrict__ Fs,
                            const float* __restrict__ df, const float* __restrict__ dF,
                            float2* __restrict__ f, float2* __restrict__ F) {
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x) {
    f[c] = df_add(fs[c], df[c]);
    F[c] = df_add(Fs[c], dF[c]);
  }
}

// The implicit increment x - x* of this step, kept for the next one.
__global__ void k_increment32(size_t n, const float2* __restrict__ fs,
                              const float2* __restrict__ Fs, const float2* __restrict__ f,
                              const float2* __restrict__ F, float* __restrict__ df,
                              float* __restrict__ dF) {
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x) {
    df[c] = df_diff(f[c], fs[c]);
    dF[c] = df_diff(F[c], Fs[c]);
  }
}

// Launch shape of the row-walking kernels: x chunks of up to 256 threads
// (a multiple of 32) and enough row groups for ~8 blocks per SM.
struct RowGrid {
  dim3 grid, block;
};
// Blocks over (x chunk, row groups); each block walks its rows in turn:
// 8 row groups per SM.  (Sizing the groups to exactly one wave of resident
// blocks, 5 per SM for the residual pass, made that pass 7 % slower at
// 256^3: 22.7 vs 21.1 ms per 10 steps.)
RowGrid row_grid(const Level& L, int sms) {
  RowGrid g;
  const int tx = L.nx >= 256 ? 256 : ((L.nx + 31) / 32) * 32;
  const int xb = (L.nx + tx - 1) / tx;
  const long long rows = (long long)L.ny * L.nz;
  const long long want = std::max(1LL, ((long long)sms * 8) / xb);
  g.block = dim3(tx);
  g.grid = dim3(xb, (unsigned)std::min(rows, std::min(want, 65535LL)));
  return g;
}

// Coupled Newton defect correction (see k_resid2_32).
sfx_status solve_newton32(sfx_ctx* c, const Nw32& p, const float* phi, float* const* Bf,
                          float* const* BF, float2*& fc, float2*& fo, float2*& Fc, float2*& Fo,
                          const float2* fs, const float2* Fs, const sfx_solve_opts* o,
                          bool predicted, bool from_star, int mgl, const Mg32Coef& kc,
                          int* iters, bool* conv, float* nrm, cudaStream_t s) {
  const Level& L = p.L;
  const size_t n = L.ncell();
  const int nb = blocks_for(n, 256);
  const int sweeps = std::max(1, o->nu1 + o->nu2);
  const float tolf = (float)o->tol;
  const NewtonKernels nk = newton_kernels(L.geom, c->f32.sweep_planes);
  // with two planes per thread the grid covers the lower half of the planes
  dim3 blk(128), grd((unsigned)(((L.nx + 1) / 2 + 127) / 128), (unsigned)L.ny,
                     (unsigned)((L.nz + nk.kp - 1) / nk.kp));
  unsigned int* dn = (unsigned int*)(c->d_norms + 8);  // two 8-slot norm buffers
  unsigned int* hn = (unsigned int*)(c->h_norms + 8);
  int* flag = c->f32.flag;
  const RowGrid rg = row_grid(L, c->sm_count);
  const __half2* Hz = L.ndim() == 3 ? c->f32.H2[2] : nullptr;
  const float2* B2[3] = {c->f32.B2[0], c->f32.B2[1], L.ndim() == 3 ? c->f32.B2[2] : nullptr};
  // sweeps 1 .. S-1 (black, then red) as tiled launches where the grid
  // allows, the last black colour as a colour launch that adds the
  // corrections to the state
  bool tiled = mgl < 2 && sweeps >= 2 && c->f32.tiled && tiled_sweep_eligible(L);
  if (tiled) {
    const sfx_status ts = tiled_sweep_prepare(c);
    if (ts != SFX_OK) return ts;
  }
  // the incremental residual needs the previous correction kept: on the
  // tiled path the two correction buffers alternate, the residual pass of
  // an iteration writing the first red half-sweep into the buffer that the
  // previous iteration's correction is not in
  const int incr_ok = tiled && c->f32.incr_resid ? 1 : 0;
  auto pair_pass = [&](const float2* fa, const float2* Fa, unsigned int* nb, float2* et,
                       const int* dn) {
    SFX_KERNEL(c, K_RESIDUAL, nk.resid, rg.grid, rg.block, s, p, phi, B2[0], B2[1], B2[2], fa, Fa,
               fs, Fs, c->f32.rc, nb, et, dn, flag + 4);
  };
  float2* ebuf[2] = {c->f32.e2, tiled ? c->f32.e2b : c->f32.e2};
  int efin = 1;   // buffer of the last correction added to the state
  // flag[4] = 1: pair residuals from the first iteration (no FP32 passes)
  const int fast_max = c->f32.fast_resid;
  SFX_CUDA(cudaMemsetAsync(flag, 0, 8 * sizeof(int), s));
  if (fast_max <= 0) SFX_KERNEL(c, K_OTHER, k_set32, 1, 32, s, flag + 4, 1);
  // Each iteration: the residual pass (which also does the first red
  // half-sweep of the correction, from zero), a device-side convergence
  // test, then the rest of the red-black sweeps, the last black one adding
  // the corrections to the state.  Once an iteration passes the test every
  // later launch of the solve returns at once, so the state is the one
  // whose residuals passed.  The host waits for the norms of iteration
  // it-1 while the GPU works on iteration it: the stream never drains for
  // a test.
  *conv = false;
  int it = 0, done_it = 0;
  for (it = 1; it <= o->max_cycles; ++it) {
    unsigned int* nbuf = dn + 8 * (it & 1);
    SFX_CUDA(cudaMemsetAsync(nbuf, 0, 8 * sizeof(unsigned int), s));
    // from_star: the first iterate is x* itself, read from (f*, F*); the
    // first state update writes x* + e into (f, F), so no copy precedes it
    const bool star = from_star && it == 1;
    const float2* fsrc = star ? fs : fc;
    const float2* Fsrc = star ? Fs : Fc;
    // the FP32 or the pair residual pass, as chosen on the device
    const int etgt = tiled ? 1 - efin : 0;
    float2* e2t = ebuf[etgt];
    SFX_KERNEL(c, K_RESID_FAST, nk.fast, rg.grid, rg.block, s, p, phi, B2[0], B2[1], B2[2], fsrc,
               Fsrc, fs, Fs, c->f32.rc, nbuf, e2t, flag, flag + 4);
    pair_pass(fsrc, Fsrc, nbuf, e2t, flag);
    if (incr_ok && it > 1)
      SFX_KERNEL(c, K_RESID_INCR, nk.incr, rg.grid, rg.block, s, p, phi, B2[0], B2[1], B2[2],
                 ebuf[efin], c->f32.rc, nbuf, e2t, flag, flag + 4);
    if (it == 1 && predicted) {
      // keep the predicted start only if its residual is already small;
      // otherwise restart from x* (both launches return at once when kept)
      int* ok = flag + 2;
      const float rho = c->f32.predict_rho;
      SFX_KERNEL(c, K_OTHER, k_pred_check32, 1, 32, s, nbuf, rho, ok);
      SFX_KERNEL(c, K_SETUP, k_restore32, nb, 256, s, n, ok, fs, Fs, fc, Fc);
      SFX_KERNEL(c, K_RESID_FAST, nk.fast, rg.grid, rg.block, s, p, phi, B2[0], B2[1], B2[2],
                 fc, Fc, fs, Fs, c->f32.rc, nbuf, e2t, ok, flag + 4);
      pair_pass(fc, Fc, nbuf, e2t, ok);
    }
    SFX_KERNEL(c, K_OTHER, k_flag32, 1, 32, s, nbuf, dn + 8 * ((it - 1) & 1), tolf, it, fast_max,
               incr_ok, flag);
    SFX_CUDA(cudaMemcpyAsync(hn + 8 * (it & 1), nbuf, 8 * sizeof(unsigned int),
                             cudaMemcpyDeviceToHost, s));
    SFX_CUDA(cudaEventRecord(c->f32.ev[it & 1], s));
    if (mgl >= 2) {
      // a V-cycle on the correction: finish the first sweep, pre - 1 more
      // fine sweeps, the coarse levels, then post fine sweeps, the last
      // black one adding the corrections to the state
      const int pre = std::max(1, o->nu1), post = std::max(1, o->nu2);
      for (int q = 0; q < pre; ++q)
        for (int color = (q == 0 ? 1 : 0); color < 2; ++color)
          SFX_KERNEL(c, K_SMOOTH_FINE, nk.corr, grd, blk, s, p, c->f32.H2[0], c->f32.H2[1], Hz,
                     c->f32.rc, c->f32.e2, color, q == 0 ? 1 : 0, nullptr, nullptr, nullptr,
                     nullptr, flag);
      sfx_status st = mg32_cycle(c, kc, mgl, pre, post, o->coarse_sweeps, flag, s);
      if (st != SFX_OK) return st;
      for (int q = 0; q < post; ++q)
        for (int color = 0; color < 2; ++color) {
          const bool apply = q == post - 1 && color == 1;
          SFX_KERNEL(c, K_SMOOTH_FINE, nk.corr, grd, blk, s, p, c->f32.H2[0], c->f32.H2[1], Hz,
                     c->f32.rc, c->f32.e2, color, 0, apply ? fc : nullptr, apply ? Fc : nullptr,
                     fsrc, Fsrc, flag);
        }
    } else if (tiled) {
      int in = etgt;   // the residual pass wrote the first red half-sweep there
      for (int q = 0; q + 1 < sweeps; ++q, in ^= 1) {
        const sfx_status ts = tiled_sweep(c, p, in, flag, s);
        if (ts != SFX_OK) return ts;
      }
      // the last black colour, which adds the corrections to the state: one
      // plane per thread (0.191 vs 0.207 ms at 256^3 with two)
      const dim3 grd1(grd.x, grd.y, (unsigned)L.nz);
      SFX_KERNEL(c, K_SMOOTH_FINE, (k_corr2_32<SFX_CART3D, 1>), grd1, blk, s, p, c->f32.H2[0],
                 c->f32.H2[1], Hz, c->f32.rc, ebuf[in], 1, 0, fc, Fc, fsrc, Fsrc, flag);
      efin = in;
    } else {
      for (int q = 0; q < sweeps; ++q)
        for (int color = (q == 0 ? 1 : 0); color < 2; ++color) {
          const bool apply = q == sweeps - 1 && color == 1;
          SFX_KERNEL(c, K_SMOOTH_FINE, nk.corr, grd, blk, s, p, c->f32.H2[0], c->f32.H2[1], Hz,
                     c->f32.rc, c->f32.e2, color, q == 0 ? 1 : 0,
                     apply ? fc : nullptr, apply ? Fc : nullptr, fsrc, Fsrc, flag);
        }
    }
    SFX_LAUNCH_CHECK();
    const int prev = it - 1;
    if (prev >= 1) {
      SFX_CUDA(cudaEventSynchronize(c->f32.ev[prev & 1]));
      const unsigned int* hb = hn + 8 * (prev & 1);
      if (hb[1] == kTimeoutBits) return SFX_ERR_TIMEOUT;
      ++c->prof.work[hb[4] <= 2u ? hb[4] : 0];   // the residual kind of iteration prev
      memcpy(nrm, hb, 4 * sizeof(float));
      for (int q = 0; q < 4; ++q)
        if (!std::isfinite(nrm[q])) return SFX_ERR_NONFINITE;
      if (hb[4] >= 1u && nrm[0] <= tolf * nrm[1] && nrm[2] <= tolf * nrm[3]) {   // as k_flag32
        *conv = true;
        done_it = prev;
        break;
      }
    }
  }
  if (from_star) {
    // converged at the first check: x* was the answer and was never copied
    SFX_KERNEL(c, K_SETUP, k_copy_if_first32, nb, 256, s, n, flag, fs, Fs, fc, Fc);
    SFX_LAUNCH_CHECK();
  }
  if (!*conv) {
    // the last iteration's residuals
    SFX_CUDA(cudaStreamSynchronize(s));
    const int last = std::min(it, o->max_cycles);
    const unsigned int* hb = hn + 8 * (last & 1);
    if (hb[1] == kTimeoutBits) return SFX_ERR_TIMEOUT;
    ++c->prof.work[hb[4] <= 2u ? hb[4] : 0];   // the residual kind of the last iteration
    if (tiled) {
      int err = 0;
      SFX_CUDA(cudaMemcpy(&err, flag + 3, sizeof(int), cudaMemcpyDeviceToHost));
      if (err) return SFX_ERR_TIMEOUT;
    }
    memcpy(nrm, hb, 4 * sizeof(float));
    for (int q = 0; q < 4; ++q)
      if (!std::isfinite(nrm[q])) return SFX_ERR_NONFINITE;
    if (hb[4] >= 1u && nrm[0] <= tolf * nrm[1] && nrm[2] <= tolf * nrm[3]) *conv = true;
    done_it = last;
  }
  *iters = done_it;
  return SFX_OK;
}

}  // namespace

sfx_status step_f32(sfx_ctx* c, const sfx_params* pr, const double* phi_in, const float* ux,
                    const float* uy, const float* uz, float2* f, float2* F, double dt,
                    const sfx_solve_opts* o, sfx_step_stats* stats, cudaStream_t s) {
  sfx_status st = f32_ensure_scratch(c);
  if (st != SFX_OK) return st;
  const Level& L = c->lev[0].lv;
  const size_t n = L.ncell();
  const int nd = L.ndim();
  float* Bf[3] = {c->f32.Bf[0], c->f32.Bf[1], nd == 3 ? c->f32.Bf[2] : nullptr};
  float* BF[3] = {c->f32.BF[0], c->f32.BF[1], nd == 3 ? c->f32.BF[2] : nullptr};
  // drift faces and the folded float phi depend on phi and (Df, DF, eps)
  const bool reuse = c->f32.reuse_drift && c->f32.drift_phi == phi_in &&
                     c->f32.drift_key[0] == pr->Df && c->f32.drift_key[1] == pr->DF &&
                     c->f32.drift_key[2] == pr->eps;
  const float* phi = c->f32.phi32;
  if (!reuse) {
    SFX_KERNEL(c, K_SETUP, k_fold_phi, blocks_for(n, 256), 256, s, n, phi_in, c->f32.phi32);
    for (int d = 0; d < nd; ++d)
      SFX_KERNEL(c, K_SETUP, k_drift32, blocks_for(L.nface(d), 256), 256, s, L, d, phi_in,
                 (float)pr->Df, (float)pr->DF, (float)(1.0 / pr->eps), Bf[d], BF[d],
                 c->f32.B2[d], c->f32.H2[d], c->f32.Hm[d]);
    SFX_LAUNCH_CHECK();
    ++c->f32.drift_epoch;
    c->f32.drift_phi = phi_in;
    c->f32.drift_key[0] = pr->Df;
    c->f32.drift_key[1] = pr->DF;
    c->f32.drift_key[2] = pr->eps;
  }
  float2* fs = c->f32.fstar;
  float2* Fs = c->f32.Fstar;
  // the previous step's implicit increment predicts this one's when the
  // step continues the same problem (same state buffers, phi, dt and
  // parameters) and the Newton solver runs
  const double key[9] = {dt, pr->ka, pr->kd, pr->Df, pr->DF, pr->eps, pr->eta, pr->gamma_inf,
                         (double)pr->literal_upwind};
  const bool predict = c->f32.predict && c->f32.solver == 1 && c->f32.inc_valid &&
                       c->f32.inc_ptr[0] == f && c->f32.inc_ptr[1] == F &&
                       c->f32.inc_ptr[2] == phi_in && memcmp(c->f32.inc_key, key, sizeof key) == 0;
  c->f32.inc_valid = false;
  if (ux) {
    Adv32 A{L, (float)dt, (float)(1.0 / L.h), {ux, uy, uz}};
    const dim3 ag((unsigned)((L.nx + kAdvX - 2) / (kAdvX - 1)),
                  (unsigned)((L.ny + kAdvY - 2) / (kAdvY - 1)),
                  L.geom == SFX_CART3D ? (unsigned)((L.nz + kAdvZ - 1) / kAdvZ) : 1u);
    if (L.geom == SFX_CART3D && c->f32.adv_staged) {
      const dim3 a3((unsigned)((L.nx + kA3X - 2) / (kA3X - 1)),
                    (unsigned)((L.ny + kA3Y - 2) / (kA3Y - 1)),
                    (unsigned)((L.nz + kA3Z - 1) / kA3Z));
      SFX_KERNEL(c, K_ADVECT, k_advect3s_32, a3, kA3X * kA3Y, s, A, f, F, (float)pr->bc_f,
                 (float)pr->bc_F, fs, Fs);
    } else {
      SFX_KERNEL(c, K_ADVECT, k_advect2t_32, ag, kAdvX * kAdvY, s, A, f, F, (float)pr->bc_f,
                 (float)pr->bc_F, fs, Fs);
    }
    SFX_LAUNCH_CHECK();
  } else {
    SFX_CUDA(cudaMemcpyAsync(fs, f, n * sizeof(float2), cudaMemcpyDeviceToDevice, s));
    SFX_CUDA(cudaMemcpyAsync(Fs, F, n * sizeof(float2), cudaMemcpyDeviceToDevice, s));
  }
  // the Newton solver starts from x* in place (no copy into f, F)
  const bool from_star = ux && !predict && c->f32.solver == 1;
  if (predict) {
    SFX_KERNEL(c, K_SETUP, k_predict32, blocks_for(n, 256), 256, s, n, fs, Fs, c->f32.inc_f,
               c->f32.inc_F, f, F);
    SFX_LAUNCH_CHECK();
  } else if (ux && !from_star) {
    SFX_CUDA(cudaMemcpyAsync(f, fs, n * sizeof(float2), cudaMemcpyDeviceToDevice, s));
    SFX_CUDA(cudaMemcpyAsync(F, Fs, n * sizeof(float2), cudaMemcpyDeviceToDevice, s));
  }
  Nl32 pf{L, (float)(1.0 / L.h), (float)(pr->Df / L.h), (float)(1.0 / dt), (float)pr->ka,
          (float)pr->kd, (float)pr->gamma_inf, (float)(1.0 / pr->eps), (float)pr->eta,
          pr->literal_upwind};
  Nl32 pF = pf;
  pF.Doh = (float)(pr->DF / L.h);
  const int sweeps = o->nu1 + o->nu2;
  // current and spare buffers of each field (the fused sweep ping-pongs)
  float2 *fc = f, *fo = c->f32.falt, *Fc = F, *Fo = c->f32.Falt;
  int it = 0;
  if (c->f32.solver >= 1) {
    bool dconv = false;
    float dn[4] = {0, 0, 0, 0};
    if (c->f32.solver == 1) {
      Nw32 pw{L, pf.invh, pf.Doh, pF.Doh, pf.inv_dt, pf.ka, pf.kd, pf.ginf, pf.inv_eps, pf.eta,
              pf.literal};
      // multigrid on the correction (Sec. 3.1 solves each implicit half by
      // multigrid): mg_levels >= 2 levels, 1 = relaxation only, 0 = chosen
      // by the diffusion number D dt/h^2 (relaxation alone converges fast
      // below 1) and, for its depth, by the phase-field width: a level
      // whose h exceeds 3 eps no longer resolves the band where the drift
      // confines f, and its re-discretised correction (measured on a
      // 64^2 circle at D dt/h^2 = 20) made the V-cycle diverge; the auto
      // choice keeps the levels with h <= 3 eps (at least one coarse level)
      const int built = (int)c->lev.size();
      const double dnum = std::max(pr->Df, pr->DF) * dt / (L.h * L.h);
      int deep = 1;
      while (deep < built && c->lev[deep].lv.h <= 3.0 * pr->eps) ++deep;
      deep = std::min(std::max(deep, 2), built);
      int mgl = o->mg_levels == 0 ? (dnum > 1.0 ? deep : 1) : std::min(o->mg_levels, built);
      if (mgl >= 2) {
        st = mg32_prepare(c, mgl, s);
        if (st != SFX_OK) return st;
      } else if (c->f32.sor != 0) {
        // over-relaxed red updates (relaxation without multigrid)
        pw.om_f = sor_omega(pr->Df, dt, L.h, pr->eps, L.ndim());
        pw.om_F = c->f32.sor > 1000 ? (float)(c->f32.sor * 1e-3)
                                    : sor_omega(pr->DF, dt, L.h, pr->eps, L.ndim());
      }
      const Mg32Coef kc{(float)pr->Df, (float)pr->DF, pf.inv_dt, pf.kd, pr->literal_upwind};
      st = solve_newton32(c, pw, phi, Bf, BF, fc, fo, Fc, Fo, fs, Fs, o, predict, from_star, mgl,
                          kc, &it, &dconv, dn, s);
    } else {
      st = solve_dc32(c, pf, pF, phi, Bf, BF, fc, fo, Fc, Fo, fs, Fs, o, &it, &dconv, dn, s);
    }
    if (st != SFX_OK) return st;
    if (fc != f) SFX_CUDA(cudaMemcpyAsync(f, fc, n * sizeof(float2), cudaMemcpyDeviceToDevice, s));
    if (Fc != F) SFX_CUDA(cudaMemcpyAsync(F, Fc, n * sizeof(float2), cudaMemcpyDeviceToDevice, s));
    if (c->f32.predict && c->f32.solver == 1 && dconv) {
      SFX_KERNEL(c, K_SETUP, k_increment32, blocks_for(n, 256), 256, s, n, fs, Fs, f, F,
                 c->f32.inc_f, c->f32.inc_F);
      SFX_LAUNCH_CHECK();
      c->f32.inc_valid = true;
      c->f32.inc_ptr[0] = f;
      c->f32.inc_ptr[1] = F;
      c->f32.inc_ptr[2] = phi_in;
      memcpy(c->f32.inc_key, key, sizeof key);
    }
    if (stats) {
      stats->picard = it;
      stats->vcycles = 2 * it * std::max(1, o->nu1 + o->nu2);
      stats->res_f = dn[0] / fmax((double)dn[1], 1e-300);
      stats->res_F = dn[2] / fmax((double)dn[3], 1e-300);
      stats->converged = dconv ? 1 : 0;
      const void* fl[2] = {f, F};
      double m[2];
      st = totals32(c, fl, 2, m, s);
      if (st != SFX_OK) return st;
      stats->mass_f = m[0];
      stats->mass_F = m[1];
    }
    return dconv ? SFX_OK : SFX_ERR_NOT_CONVERGED;
  }
  bool conv = false;
  float nrm[4] = {0, 0, 0, 0};
  // Convergence is tested on the host, which stalls the stream; the step
  // first runs as many iterations as the previous step needed (minus one,
  // to keep probing downwards) without testing, then tests every
  // check_every iterations.
  const int first = std::min(std::max(c->f32.predicted, 1), o->max_cycles);
  for (it = 1; it <= o->max_cycles; ++it) {
    const bool check = (it >= first && (it - first) % o->check_every == 0) ||
                       it == o->max_cycles;
    if (check) SFX_CUDA(cudaMemsetAsync(c->d_norms, 0, 8 * sizeof(unsigned long long), s));
    for (int q = 0; q < sweeps; ++q) {
      if (c->f32.fused) {
        st = fused_sweep32<0>(c, pf, phi, Bf, fc, fo, fs, Fc, check && q == 0, s);
        std::swap(fc, fo);
      } else {
        st = sweep32(c, 0, pf, phi, Bf, fc, fs, Fc, check && q == 0, s);
      }
      if (st != SFX_OK) return st;
    }
    for (int q = 0; q < sweeps; ++q) {
      if (c->f32.fused) {
        st = fused_sweep32<1>(c, pF, phi, BF, Fc, Fo, Fs, fc, check && q == 0, s);
        std::swap(Fc, Fo);
      } else {
        st = sweep32(c, 1, pF, phi, BF, Fc, Fs, fc, check && q == 0, s);
      }
      if (st != SFX_OK) return st;
    }
    if (check) {
      SFX_CUDA(cudaMemcpyAsync(c->h_norms, c->d_norms, 2 * sizeof(unsigned long long),
                               cudaMemcpyDeviceToHost, s));
      SFX_CUDA(cudaStreamSynchronize(s));
      memcpy(nrm, c->h_norms, 4 * sizeof(float));
      for (int q = 0; q < 4; ++q)
        if (!std::isfinite(nrm[q])) return SFX_ERR_NONFINITE;
      double rf = nrm[0] / fmax((double)nrm[1], 1e-300);
      double rF = nrm[2] / fmax((double)nrm[3], 1e-300);
      if (rf <= o->tol && rF <= o->tol) {
        conv = true;
        break;
      }
    }
  }
  c->f32.predicted = conv ? (it == first ? it - 1 : it) : 0;
  if (fc != f) SFX_CUDA(cudaMemcpyAsync(f, fc, n * sizeof(float2), cudaMemcpyDeviceToDevice, s));
  if (Fc != F) SFX_CUDA(cudaMemcpyAsync(F, Fc, n * sizeof(float2), cudaMemcpyDeviceToDevice, s));
  if (stats) {
    stats->picard = it > o->max_cycles ? o->max_cycles : it;
    stats->vcycles = 2 * stats->picard * sweeps;
    stats->res_f = nrm[0] / fmax((double)nrm[1], 1e-300);
    stats->res_F = nrm[2] / fmax((double)nrm[3], 1e-300);
    stats->converged = conv ? 1 : 0;
    const void* fl[2] = {f, F};
    double m[2];
    st = totals32(c, fl, 2, m, s);
    if (st != SFX_OK) return st;
    stats->mass_f = m[0];
    stats->mass_F = m[1];
  }
  return conv ? SFX_OK : SFX_ERR_NOT_CONVERGED;
}

sfx_status advect32(sfx_ctx* c, const float* ux, const float* uy, const float* uz, double dt,
                    const float2* xi, double bc_in, float2* out, cudaStream_t s) {
  const Level& L = c->lev[0].lv;
  Adv32 A{L, (float)dt, (float)(1.0 / L.h), {ux, uy, uz}};
  SFX_KERNEL(c, K_ADVECT, k_advect32, blocks_for(L.ncell(), 256), 256, s, A, xi, (float)bc_in,
             out);
  SFX_LAUNCH_CHECK();
  return SFX_OK;
}

sfx_status totals32(sfx_ctx* c, const void* const* fields, int nf, double* out, cudaStream_t s) {
  const Level& L = c->lev[0].lv;
  const int nblk = c->n_partial_blocks;
  for (int i = 0; i < nf; i += 2) {
    const int m = std::min(2, nf - i);
    SFX_KERNEL(c, K_TOTALS, k_total32_partials, dim3((unsigned)nblk, (unsigned)m), 256, s, L,
               (const float2*)fields[i], (const float2*)fields[i + m - 1], i, c->partials);
  }
  double h = L.h;
  double scale = L.geom == SFX_PLANAR2D ? h * h : (L.geom == SFX_CART3D ? h * h * h : kPi * h * h * h);
  SFX_KERNEL(c, K_TOTALS, k_total32_final, nf, 256, s, c->partials, nblk, scale, c->d_sums);
  SFX_LAUNCH_CHECK();
  SFX_CUDA(cudaMemcpyAsync(c->h_sums, c->d_sums, nf * sizeof(double), cudaMemcpyDeviceToHost, s));
  SFX_CUDA(cudaStreamSynchronize(s));
  memcpy(out, c->h_sums, nf * sizeof(double));
  return SFX_OK;
}

sfx_status marangoni32(sfx_ctx* c, const sfx_params* p, const float2* f, const double* phi,
                       const float* C, int dm_mode, float* sigma, float* force, cudaStream_t s) {
  sfx_status st = f32_ensure_scratch(c);
  if (st != SFX_OK) return st;
  const Level& L = c->lev[0].lv;
  const size_t n = L.ncell();
  Eos32 q{(float)p->gamma_inf, (float)p->eps, (float)(1.0 / p->eps), (float)p->sigma0,
          (float)p->E, p->eos, p->gamma_inf, p->eps, p->sigma0, p->E};
  SFX_KERNEL(c, K_FORCES, k_eos32, blocks_for(n, 256), 256, s, n, q, f, phi, c->f32.dsig, sigma);
  const RowGrid fg = row_grid(L, c->sm_count);
  SFX_KERNEL(c, K_FORCES, k_force32, fg.grid, fg.block, s, L, phi, C, c->f32.dsig, dm_mode,
             q.inv_eps, force);
  SFX_LAUNCH_CHECK();
  return SFX_OK;
}

sfx_status df_pack(const double* in, void* out, size_t n, cudaStream_t s) {
  if (n == 0) return SFX_OK;
  k_pack_df<<<blocks_for(n, 256), 256, 0, s>>>(n, in, (float2*)out);
  SFX_LAUNCH_CHECK();
  return SFX_OK;
}

sfx_status df_unpack(const void* in, double* out, size_t n, cudaStream_t s) {
  if (n == 0) return SFX_OK;
  k_unpack_df<<<blocks_for(n, 256), 256, 0, s>>>(n, (const float2*)in, out);
  SFX_LAUNCH_CHECK();
  return SFX_OK;
}

sfx_status f32_ensure_scratch(sfx_ctx* c) {
  if (c->f32.ready) return SFX_OK;
  const Level& L = c->lev[0].lv;
  const size_t n = L.ncell();
  auto get = [&](size_t bytes, void** p) -> sfx_status {
    SFX_CUDA(cudaMalloc(p, bytes ? bytes : 4));
    c->allocations.push_back(*p);
    return SFX_OK;
  };
  sfx_status st;
  for (int d = 0; d < L.ndim(); ++d) {
    if ((st = get(L.nface(d) * sizeof(float), (void**)&c->f32.Bf[d])) != SFX_OK) return st;
    if ((st = get(L.nface(d) * sizeof(float), (void**)&c->f32.BF[d])) != SFX_OK) return st;
    if ((st = get(L.nface(d) * sizeof(float2), (void**)&c->f32.B2[d])) != SFX_OK) return st;
    if ((st = get(L.nface(d) * sizeof(__half2), (void**)&c->f32.H2[d])) != SFX_OK) return st;
  }
  if ((st = get(n * sizeof(float2), (void**)&c->f32.fstar)) != SFX_OK) return st;
  if ((st = get(n * sizeof(float2), (void**)&c->f32.Fstar)) != SFX_OK) return st;
  if ((st = get(n * sizeof(float), (void**)&c->f32.dsig)) != SFX_OK) return st;
  if ((st = get(n * sizeof(float), (void**)&c->f32.phi32)) != SFX_OK) return st;
  if ((st = get(n * sizeof(float), (void**)&c->f32.inc_f)) != SFX_OK) return st;
  if ((st = get(n * sizeof(float), (void**)&c->f32.inc_F)) != SFX_OK) return st;
  if ((st = get(8 * sizeof(int), (void**)&c->f32.flag)) != SFX_OK) return st;
  if ((st = get(n * sizeof(float2), (void**)&c->f32.falt)) != SFX_OK) return st;
  if ((st = get(n * sizeof(float2), (void**)&c->f32.Falt)) != SFX_OK) return st;
  // the Newton work arrays are colour-packed: 2 planes of ny nz ceil(nx/2)
  const size_t np = std::max(n, 2 * (size_t)L.ny * L.nz * ((L.nx + 1) / 2));
  float** arrs[6] = {&c->f32.ef, &c->f32.eF, &c->f32.rf, &c->f32.rF, &c->f32.lf, &c->f32.lF};
  for (float** q : arrs)
    if ((st = get(np * sizeof(float), (void**)q)) != SFX_OK) return st;
  if ((st = get(np * sizeof(float2), (void**)&c->f32.e2)) != SFX_OK) return st;
  if ((st = get(np * sizeof(float4), (void**)&c->f32.rc)) != SFX_OK) return st;
  if (tiled_sweep_eligible(L)) {
    if ((st = get(np * sizeof(float2), (void**)&c->f32.e2b)) != SFX_OK) return st;
    for (int d = 0; d < 3; ++d)
      if ((st = get(n * sizeof(__half2), (void**)&c->f32.Hm[d])) != SFX_OK) return st;
  }
  for (int q = 0; q < 2; ++q) SFX_CUDA(cudaEventCreateWithFlags(&c->f32.ev[q], cudaEventDisableTiming));
  c->f32.ready = true;
  return SFX_OK;
}

}  // namespace sfx
