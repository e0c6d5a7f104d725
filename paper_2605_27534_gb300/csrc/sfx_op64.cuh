// FP64 finite-volume operator of Sec. 3.1-3.2 (App. A in 3D, App. B in
// axisymmetric form), shared by the multigrid solver and the adjoint.
//
//   L(a) = div(alpha grad a + beta a) + lambda a,  alpha = -D, beta = -B
//
// written per cell as L(a)_c = (lambda_c - S_d/V_c) a_c - S_n/V_c with the
// face quantity G = D (a_R - a_L)/h + B a_up = cL a_L + cR a_R and
//   S_d = sum_+ A cL - sum_- A cR,   S_n = sum_+ A cR a_+ - sum_- A cL a_-.
// The drift is upwinded on its transport velocity -B (a_up = a_L when
// B < 0); `literal` selects the face value printed in Sec. 3.2 instead.
#pragma once

#include "sfx_common.cuh"

namespace sfx {

struct Op {
  double D;
  const double* B[3];   // face drifts (NULL: zero)
  int literal;
  const double* lam;
  double Bs = 1.0;      // the drift is Bs * B (B of unit diffusivity in the adjoint)
};

__device__ __forceinline__ void face_coeffs(double Doh, double B, int literal, double& cL,
                                            double& cR) {
  cL = -Doh;
  cR = Doh;
  bool left = literal ? (B > 0.0) : (B < 0.0);
  if (left) cL += B;
  else cR += B;
}

__device__ __forceinline__ double faceB(const Op& op, int d, size_t f) {
  return op.B[d] ? op.Bs * op.B[d][f] : 0.0;
}

// S_d and S_n of cell (i,j,k) (see the comment at the top).
__device__ __forceinline__ void flux_terms(const Level& L, const Op& op, const double* __restrict__ a,
                                           int i, int j, int k, double& sd, double& sn) {
  const double Doh = op.D / L.h;
  double cL, cR;
  sd = 0.0;
  sn = 0.0;
  // x (radial in the axisymmetric case)
  if (i + 1 < L.nx) {
    double A = face_area(L, 0, i + 1);
    face_coeffs(Doh, faceB(op, 0, fidx(L, 0, i + 1, j, k)), op.literal, cL, cR);
    sd += A * cL;
    sn += A * cR * a[cidx(L, i + 1, j, k)];
  }
  if (i > 0) {
    double A = face_area(L, 0, i);
    face_coeffs(Doh, faceB(op, 0, fidx(L, 0, i, j, k)), op.literal, cL, cR);
    sd -= A * cR;
    sn -= A * cL * a[cidx(L, i - 1, j, k)];
  }
  // y (axial in the axisymmetric case); both faces share the column's area
  const double Ay = face_area(L, 1, i);
  if (j + 1 < L.ny) {
    face_coeffs(Doh, faceB(op, 1, fidx(L, 1, i, j + 1, k)), op.literal, cL, cR);
    sd += Ay * cL;
    sn += Ay * cR * a[cidx(L, i, j + 1, k)];
  }
  if (j > 0) {
    face_coeffs(Doh, faceB(op, 1, fidx(L, 1, i, j, k)), op.literal, cL, cR);
    sd -= Ay * cR;
    sn -= Ay * cL * a[cidx(L, i, j - 1, k)];
  }
  if (L.geom == SFX_CART3D) {
    const double Az = L.h * L.h;
    if (k + 1 < L.nz) {
      face_coeffs(Doh, faceB(op, 2, fidx(L, 2, i, j, k + 1)), op.literal, cL, cR);
      sd += Az * cL;
      sn += Az * cR * a[cidx(L, i, j, k + 1)];
    }
    if (k > 0) {
      face_coeffs(Doh, faceB(op, 2, fidx(L, 2, i, j, k)), op.literal, cL, cR);
      sd -= Az * cR;
      sn -= Az * cL * a[cidx(L, i, j, k - 1)];
    }
  }
}

// The transposed operator: (N^T nu)_c = dT nu_c + nT for N(a)_c = (S_d a_c +
// S_n)/V_c.  A face between cells l and r with G = cL a_l + cR a_r adds
// A cL (nu_l/V_l - nu_r/V_r) to cell l and A cR (nu_l/V_l - nu_r/V_r) to
// cell r, so dT = S_d/V_c and the neighbour terms divide by the
// neighbour's volume.
__device__ __forceinline__ void flux_terms_T(const Level& L, const Op& op,
                                             const double* __restrict__ nu, int i, int j, int k,
                                             double& dT, double& nT) {
  const double Doh = op.D / L.h;
  const double Vc = cell_volume(L, i);
  double cL, cR, sd = 0.0;
  nT = 0.0;
  if (i + 1 < L.nx) {
    double A = face_area(L, 0, i + 1);
    face_coeffs(Doh, faceB(op, 0, fidx(L, 0, i + 1, j, k)), op.literal, cL, cR);
    sd += A * cL;
    nT -= A * cL * nu[cidx(L, i + 1, j, k)] / cell_volume(L, i + 1);
  }
  if (i > 0) {
    double A = face_area(L, 0, i);
    face_coeffs(Doh, faceB(op, 0, fidx(L, 0, i, j, k)), op.literal, cL, cR);
    sd -= A * cR;
    nT += A * cR * nu[cidx(L, i - 1, j, k)] / cell_volume(L, i - 1);
  }
  const double Ay = face_area(L, 1, i);
  if (j + 1 < L.ny) {
    face_coeffs(Doh, faceB(op, 1, fidx(L, 1, i, j + 1, k)), op.literal, cL, cR);
    sd += Ay * cL;
    nT -= Ay * cL * nu[cidx(L, i, j + 1, k)] / Vc;
  }
  if (j > 0) {
    face_coeffs(Doh, faceB(op, 1, fidx(L, 1, i, j, k)), op.literal, cL, cR);
    sd -= Ay * cR;
    nT += Ay * cR * nu[cidx(L, i, j - 1, k)] / Vc;
  }
  if (L.geom == SFX_CART3D) {
    const double Az = L.h * L.h;
    if (k + 1 < L.nz) {
      face_coeffs(Doh, faceB(op, 2, fidx(L, 2, i, j, k + 1)), op.literal, cL, cR);
      sd += Az * cL;
      nT -= Az * cL * nu[cidx(L, i, j, k + 1)] / Vc;
    }
    if (k > 0) {
      face_coeffs(Doh, faceB(op, 2, fidx(L, 2, i, j, k)), op.literal, cL, cR);
      sd -= Az * cR;
      nT += Az * cR * nu[cidx(L, i, j, k - 1)] / Vc;
    }
  }
  dT = sd / Vc;
}

// The same transposed operator as coefficients: (N^T nu)_c = dT nu_c +
// sum_q w[q] nu_(neighbour q), q = x-, x+, y-, y+, z-, z+ (w = 0 where the
// neighbour does not exist).
__device__ __forceinline__ void flux_weights_T(const Level& L, const Op& op, int i, int j, int k,
                                               double& dT, double* w) {
  const double Doh = op.D / L.h;
  const double Vc = cell_volume(L, i);
  double cL, cR, sd = 0.0;
  for (int q = 0; q < 6; ++q) w[q] = 0.0;
  if (i + 1 < L.nx) {
    const double A = face_area(L, 0, i + 1);
    face_coeffs(Doh, faceB(op, 0, fidx(L, 0, i + 1, j, k)), op.literal, cL, cR);
    sd += A * cL;
    w[1] = -A * cL / cell_volume(L, i + 1);
  }
  if (i > 0) {
    const double A = face_area(L, 0, i);
    face_coeffs(Doh, faceB(op, 0, fidx(L, 0, i, j, k)), op.literal, cL, cR);
    sd -= A * cR;
    w[0] = A * cR / cell_volume(L, i - 1);
  }
  const double Ay = face_area(L, 1, i);
  if (j + 1 < L.ny) {
    face_coeffs(Doh, faceB(op, 1, fidx(L, 1, i, j + 1, k)), op.literal, cL, cR);
    sd += Ay * cL;
    w[3] = -Ay * cL / Vc;
  }
  if (j > 0) {
    face_coeffs(Doh, faceB(op, 1, fidx(L, 1, i, j, k)), op.literal, cL, cR);
    sd -= Ay * cR;
    w[2] = Ay * cR / Vc;
  }
  if (L.geom == SFX_CART3D) {
    const double Az = L.h * L.h;
    if (k + 1 < L.nz) {
      face_coeffs(Doh, faceB(op, 2, fidx(L, 2, i, j, k + 1)), op.literal, cL, cR);
      sd += Az * cL;
      w[5] = -Az * cL / Vc;
    }
    if (k > 0) {
      face_coeffs(Doh, faceB(op, 2, fidx(L, 2, i, j, k)), op.literal, cL, cR);
      sd -= Az * cR;
      w[4] = Az * cR / Vc;
    }
  }
  dT = sd / Vc;
}

// Compensated block reduction of (s, c) pairs; thread 0 receives the
// block's pair in (s, c).  NT threads per block, a multiple of 32.
template <int NT>
__device__ __forceinline__ void block_sum_comp(double& s, double& c) {
  warp_sum_comp(s, c);
  __shared__ double ss[NT / 32], sc[NT / 32];
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { ss[w] = s; sc[w] = c; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = ss[0], b = sc[0];
    for (int q = 1; q < NT / 32; ++q) {
      double t, e;
      two_sum(a, ss[q], t, e);
      a = t;
      b += sc[q] + e;
    }
    s = a;
    c = b;
  }
  __syncthreads();
}

}  // namespace sfx
