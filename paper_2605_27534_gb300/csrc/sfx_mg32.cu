// FP32 multigrid of the coupled Newton correction (SFX_F32 contexts).
//
// Each Newton iteration of the App. C system solves, approximately, the
// linear correction equation
//   [A_f + J_ff   -J_fF ] [e_f]   [r_f]
//   [-J_Ff   A_F + J_FF ] [e_F] = [r_F]
// (A = the Sec. 3.1-3.2 flux operator of each field, J the pointwise 2x2
// exchange Jacobian, see jac2).  Red-black block Gauss-Seidel alone damps
// the error by a factor set by D dt/h^2: once diffusion dominates the
// kinetic diagonal (D dt/h^2 >> 1) it stalls on smooth error.  Sec. 3.1
// solves each implicit half by multigrid; here the coupled correction gets
// a V-cycle whose smoother is the same 2x2 block Gauss-Seidel on every
// level:
//   restriction  volume-weighted mean of the 2^d children of the
//                correction residual rho = r - (A + J) e and of J;
//   coarse faces area-weighted mean of the fine drift faces;
//   coarse A     re-discretised (the same D on the coarse h);
//   prolongation cell-centred bi/trilinear with mirrored walls.
// The fine level keeps its colour-packed arrays (rc, e2, half-precision
// faces) and its sweeps (k_corr2_32); the coarse levels use the plain cell
// layout and float drift faces.  Everything here is FP32: the Newton
// residual that decides convergence is the pair-arithmetic pass.
#include "sfx_internal.h"
#include "sfx_f32_dev.cuh"

namespace sfx {
namespace {

Nw32 level_coef(const Level& L, const Mg32Coef& k) {
  Nw32 p{};
  p.L = L;
  p.invh = (float)(1.0 / L.h);
  p.Dfh = (float)(k.Df / L.h);
  p.DFh = (float)(k.DF / L.h);
  p.inv_dt = k.inv_dt;
  p.kd = k.kd;
  p.literal = k.literal;
  return p;
}

// Relative volume of cell column i (axisymmetric: 2i + 1; else 1).
template <int G>
__device__ __forceinline__ float vol_w(int i) {
  return G == SFX_AXISYM ? 2.0f * (float)i + 1.0f : 1.0f;
}

// Correction residual rho = r + flux(e) - J e at a plain-layout cell, with
// the 2x2 block of the cell (a, b; d, ee as in corr2_cell) and its e.
template <int G>
__device__ __forceinline__ void plain_cell(const Nw32& p, int i, int j, int k,
                                           const float2* __restrict__ e,
                                           const float2* __restrict__ r,
                                           const float2* __restrict__ J,
                                           const float2* const* B, float2& rho, float4& blk,
                                           float2& ec) {
  const Level& L = p.L;
  const ix c = cidx32(L, i, j, k);
  bool has[6];
  ix nbi[6];
  gather6<G>(L, i, j, k, c, has, nbi);
  float enf[6], enF[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const float2 v = has[q] ? e[nbi[q]] : make_float2(0.0f, 0.0f);
    enf[q] = v.x;
    enF[q] = v.y;
  }
  ec = e[c];
  float Bf[6], BF[6], dgf, dgF;
  faces6f2(L, B[0], B[1], B[2], i, j, k, has, Bf, BF);
  const float flf = flux_lin<G>(L, p.invh, p.Dfh, p.literal, i, ec.x, enf, has, Bf, dgf);
  const float flF = flux_lin<G>(L, p.invh, p.DFh, p.literal, i, ec.y, enF, has, BF, dgF);
  const float2 jj = J[c], rr = r[c];
  const Jac2 Jc = jac2(p, jj.x, jj.y);
  rho.x = __fmaf_rn(Jc.fF, ec.y, __fmaf_rn(-Jc.ff, ec.x, __fadd_rn(rr.x, flf)));
  rho.y = __fmaf_rn(Jc.Ff, ec.x, __fmaf_rn(-Jc.FF, ec.y, __fadd_rn(rr.y, flF)));
  blk = make_float4(__fadd_rn(Jc.ff, dgf), Jc.fF, Jc.Ff, __fadd_rn(Jc.FF, dgF));
}

// The same residual at a fine cell from the colour-packed arrays of the
// Newton kernels (rc = r_f, r_F, u, v; e2; half-precision faces).
template <int G>
__device__ __forceinline__ void fine_cell(const Nw32& p, int i, int j, int k,
                                          const __half2* const* H,
                                          const float4* __restrict__ rc,
                                          const float2* __restrict__ e2, float2& rho,
                                          float2& uv) {
  const Level& L = p.L;
  const ix c = cidx32(L, i, j, k);
  bool has[6];
  ix nbi[6];
  gather6<G>(L, i, j, k, c, has, nbi);
  const RBIdx rb = rb_index(L, i, j, k);
  const int color = (i + j + k) & 1;
  const ix own = (ix)color * rb.plane + rb.pos;
  const ix oth = (ix)(1 - color) * rb.plane + rb.pos;
  const ix sz = (ix)L.ny * rb.half;
  nbi[0] = oth - 1 + (i & 1);
  nbi[1] = oth + (i & 1);
  nbi[2] = oth - rb.half;
  nbi[3] = oth + rb.half;
  nbi[4] = oth - sz;
  nbi[5] = oth + sz;
  float enf[6], enF[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const float2 v = has[q] ? e2[nbi[q]] : make_float2(0.0f, 0.0f);
    enf[q] = v.x;
    enF[q] = v.y;
  }
  const float2 ec = e2[own];
  float Bf[6], BF[6], dgf, dgF;
  faces6x2(L, H[0], H[1], H[2], i, j, k, has, Bf, BF);
  const float flf = flux_lin<G>(L, p.invh, p.Dfh, p.literal, i, ec.x, enf, has, Bf, dgf);
  const float flF = flux_lin<G>(L, p.invh, p.DFh, p.literal, i, ec.y, enF, has, BF, dgF);
  const float4 q4 = rc[own];
  const Jac2 Jc = jac2(p, q4.z, q4.w);
  rho.x = __fmaf_rn(Jc.fF, ec.y, __fmaf_rn(-Jc.ff, ec.x, __fadd_rn(q4.x, flf)));
  rho.y = __fmaf_rn(Jc.Ff, ec.x, __fmaf_rn(-Jc.FF, ec.y, __fadd_rn(q4.y, flF)));
  uv = make_float2(q4.z, q4.w);
}

__device__ __forceinline__ float2 block_solve(const float4& b, const float2& rho) {
  const float det = __fmaf_rn(b.x, b.w, -__fmul_rn(b.y, b.z));
  const float inv = __fdividef(1.0f, det);
  return make_float2(__fmul_rn(__fmaf_rn(b.w, rho.x, __fmul_rn(b.y, rho.y)), inv),
                     __fmul_rn(__fmaf_rn(b.z, rho.x, __fmul_rn(b.x, rho.y)), inv));
}

// One colour of the 2x2 block Gauss-Seidel on a coarse (plain) level.
template <int G>
__global__ void k_mg2_smooth(Nw32 p, const float2* __restrict__ r, const float2* __restrict__ J,
                             const float2* __restrict__ Bx, const float2* __restrict__ By,
                             const float2* __restrict__ Bz, float2* __restrict__ e, int color,
                             const int* __restrict__ done) {
  if (done && *done) return;
  const Level& L = p.L;
  const int j = blockIdx.y, k = blockIdx.z;
  const int i = 2 * (blockIdx.x * blockDim.x + threadIdx.x) + ((j + k + color) & 1);
  if (i >= L.nx) return;
  const float2* B[3] = {Bx, By, Bz};
  float2 rho, ec;
  float4 blk;
  plain_cell<G>(p, i, j, k, e, r, J, B, rho, blk, ec);
  const float2 d = block_solve(blk, rho);
  e[cidx32(L, i, j, k)] = make_float2(__fadd_rn(ec.x, d.x), __fadd_rn(ec.y, d.y));
}

// Coarsest level: all sweeps in one block.
template <int G>
__global__ void __launch_bounds__(1024)
k_mg2_coarse(Nw32 p, const float2* __restrict__ r, const float2* __restrict__ J,
             const float2* __restrict__ Bx, const float2* __restrict__ By,
             const float2* __restrict__ Bz, float2* e, int sweeps, const int* __restrict__ done) {
  if (done && *done) return;
  const Level& L = p.L;
  const float2* B[3] = {Bx, By, Bz};
  const int hx = (L.nx + 1) / 2;
  const int nwork = hx * L.ny * L.nz;
  for (int s = 0; s < sweeps; ++s)
    for (int color = 0; color < 2; ++color) {
      for (int w = threadIdx.x; w < nwork; w += blockDim.x) {
        const int ih = w % hx, j = (w / hx) % L.ny, k = w / (hx * L.ny);
        const int i = 2 * ih + ((j + k + color) & 1);
        if (i >= L.nx) continue;
        float2 rho, ec;
        float4 blk;
        plain_cell<G>(p, i, j, k, e, r, J, B, rho, blk, ec);
        const float2 d = block_solve(blk, rho);
        e[cidx32(L, i, j, k)] = make_float2(__fadd_rn(ec.x, d.x), __fadd_rn(ec.y, d.y));
      }
      __syncthreads();
    }
}

// Restriction of the fine correction residual and of J to level 1; the
// level-1 correction starts at zero.
template <int G>
__global__ void k_mg2_restrict_fine(Nw32 p, Level Lc, const __half2* __restrict__ Hx,
                                    const __half2* __restrict__ Hy,
                                    const __half2* __restrict__ Hz,
                                    const float4* __restrict__ rc,
                                    const float2* __restrict__ e2, float2* __restrict__ r1,
                                    float2* __restrict__ J1, float2* __restrict__ e1,
                                    const int* __restrict__ done) {
  if (done && *done) return;
  const Level& Lf = p.L;
  const __half2* H[3] = {Hx, Hy, Hz};
  const ix n = (ix)Lc.ncell();
  const int kz = G == SFX_CART3D ? 2 : 1;
  for (ix c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
    const int I = (int)(c % (ix)Lc.nx), Jj = (int)((c / (ix)Lc.nx) % (ix)Lc.ny);
    const int K = (int)(c / ((ix)Lc.nx * (ix)Lc.ny));
    float2 sr = make_float2(0.0f, 0.0f), sj = make_float2(0.0f, 0.0f);
    float sw = 0.0f;
    for (int dk = 0; dk < kz; ++dk)
      for (int dj = 0; dj < 2; ++dj)
        for (int di = 0; di < 2; ++di) {
          const int i = 2 * I + di, j = 2 * Jj + dj, k = kz == 2 ? 2 * K + dk : 0;
          if (i >= Lf.nx || j >= Lf.ny || k >= Lf.nz) continue;
          float2 rho, uv;
          fine_cell<G>(p, i, j, k, H, rc, e2, rho, uv);
          const float w = vol_w<G>(i);
          sr.x = __fmaf_rn(w, rho.x, sr.x);
          sr.y = __fmaf_rn(w, rho.y, sr.y);
          sj.x = __fmaf_rn(w, uv.x, sj.x);
          sj.y = __fmaf_rn(w, uv.y, sj.y);
          sw += w;
        }
    const float iw = 1.0f / sw;
    r1[c] = make_float2(sr.x * iw, sr.y * iw);
    J1[c] = make_float2(sj.x * iw, sj.y * iw);
    e1[c] = make_float2(0.0f, 0.0f);
  }
}

// Restriction between plain levels.
template <int G>
__global__ void k_mg2_restrict(Nw32 p, Level Lc, const float2* __restrict__ r,
                               const float2* __restrict__ J, const float2* __restrict__ Bx,
                               const float2* __restrict__ By, const float2* __restrict__ Bz,
                               const float2* __restrict__ e, float2* __restrict__ rn,
                               float2* __restrict__ Jn, float2* __restrict__ en,
                               const int* __restrict__ done) {
  if (done && *done) return;
  const Level& Lf = p.L;
  const float2* B[3] = {Bx, By, Bz};
  const ix n = (ix)Lc.ncell();
  const int kz = G == SFX_CART3D ? 2 : 1;
  for (ix c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
    const int I = (int)(c % (ix)Lc.nx), Jj = (int)((c / (ix)Lc.nx) % (ix)Lc.ny);
    const int K = (int)(c / ((ix)Lc.nx * (ix)Lc.ny));
    float2 sr = make_float2(0.0f, 0.0f), sj = make_float2(0.0f, 0.0f);
    float sw = 0.0f;
    for (int dk = 0; dk < kz; ++dk)
      for (int dj = 0; dj < 2; ++dj)
        for (int di = 0; di < 2; ++di) {
          const int i = 2 * I + di, j = 2 * Jj + dj, k = kz == 2 ? 2 * K + dk : 0;
          if (i >= Lf.nx || j >= Lf.ny || k >= Lf.nz) continue;
          float2 rho, ec;
          float4 blk;
          plain_cell<G>(p, i, j, k, e, r, J, B, rho, blk, ec);
          const float2 uv = J[cidx32(Lf, i, j, k)];
          const float w = vol_w<G>(i);
          sr.x = __fmaf_rn(w, rho.x, sr.x);
          sr.y = __fmaf_rn(w, rho.y, sr.y);
          sj.x = __fmaf_rn(w, uv.x, sj.x);
          sj.y = __fmaf_rn(w, uv.y, sj.y);
          sw += w;
        }
    const float iw = 1.0f / sw;
    rn[c] = make_float2(sr.x * iw, sr.y * iw);
    Jn[c] = make_float2(sj.x * iw, sj.y * iw);
    en[c] = make_float2(0.0f, 0.0f);
  }
}

// Bi/trilinear value of the coarse correction at fine cell (i, j, k)
// (weights 3/4 parent, 1/4 neighbour per direction; mirrored at walls).
__device__ __forceinline__ float2 prolong_at(const Level& Lc, const float2* __restrict__ ec,
                                             int i, int j, int k, bool is3) {
  const int I = i >> 1, J = j >> 1, K = k >> 1;
  const int I2 = min(max(I + ((i & 1) ? 1 : -1), 0), Lc.nx - 1);
  const int J2 = min(max(J + ((j & 1) ? 1 : -1), 0), Lc.ny - 1);
  float2 v = make_float2(0.0f, 0.0f);
  auto add = [&](float w, int a, int b, int d) {
    const float2 x = ec[cidx32(Lc, a, b, d)];
    v.x = __fmaf_rn(w, x.x, v.x);
    v.y = __fmaf_rn(w, x.y, v.y);
  };
  if (!is3) {
    add(0.5625f, I, J, 0);
    add(0.1875f, I2, J, 0);
    add(0.1875f, I, J2, 0);
    add(0.0625f, I2, J2, 0);
  } else {
    const int K2 = min(max(K + ((k & 1) ? 1 : -1), 0), Lc.nz - 1);
    add(0.421875f, I, J, K);
    add(0.140625f, I2, J, K);
    add(0.140625f, I, J2, K);
    add(0.140625f, I, J, K2);
    add(0.046875f, I2, J2, K);
    add(0.046875f, I2, J, K2);
    add(0.046875f, I, J2, K2);
    add(0.015625f, I2, J2, K2);
  }
  return v;
}

__global__ void k_mg2_prolong(Level Lc, Level Lf, const float2* __restrict__ ec,
                              float2* __restrict__ ef, const int* __restrict__ done) {
  if (done && *done) return;
  const ix n = (ix)Lf.ncell();
  const bool is3 = Lf.geom == SFX_CART3D;
  for (ix c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
    const int i = (int)(c % (ix)Lf.nx), j = (int)((c / (ix)Lf.nx) % (ix)Lf.ny);
    const int k = (int)(c / ((ix)Lf.nx * (ix)Lf.ny));
    const float2 v = prolong_at(Lc, ec, i, j, k, is3);
    const float2 x = ef[c];
    ef[c] = make_float2(__fadd_rn(x.x, v.x), __fadd_rn(x.y, v.y));
  }
}

// Level 1 -> the fine level's colour-packed correction.
__global__ void k_mg2_prolong_fine(Level Lc, Level Lf, const float2* __restrict__ ec,
                                   float2* __restrict__ e2, const int* __restrict__ done) {
  if (done && *done) return;
  const ix n = (ix)Lf.ncell();
  const bool is3 = Lf.geom == SFX_CART3D;
  for (ix c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
    const int i = (int)(c % (ix)Lf.nx), j = (int)((c / (ix)Lf.nx) % (ix)Lf.ny);
    const int k = (int)(c / ((ix)Lf.nx * (ix)Lf.ny));
    const float2 v = prolong_at(Lc, ec, i, j, k, is3);
    const RBIdx rb = rb_index(Lf, i, j, k);
    const ix own = (ix)((i + j + k) & 1) * rb.plane + rb.pos;
    const float2 x = e2[own];
    e2[own] = make_float2(__fadd_rn(x.x, v.x), __fadd_rn(x.y, v.y));
  }
}

// Area-weighted restriction of drift faces (B_f, B_F) in direction d.
template <int G>
__global__ void k_mg2_restrict_faces(Level Lf, Level Lc, int d, const float2* __restrict__ Bf,
                                     float2* __restrict__ Bc) {
  const size_t n = Lc.nface(d);
  const int fx = Lc.nx + (d == 0), fy = Lc.ny + (d == 1);
  const bool is3 = G == SFX_CART3D;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n;
       q += (size_t)gridDim.x * blockDim.x) {
    const int I = (int)(q % fx), J = (int)((q / fx) % fy), K = (int)(q / ((size_t)fx * fy));
    const int pos = d == 0 ? I : (d == 1 ? J : K);
    if (pos == 0 || pos == Lc.extent(d)) {
      Bc[q] = make_float2(0.0f, 0.0f);
      continue;
    }
    float2 num = make_float2(0.0f, 0.0f);
    float den = 0.0f;
    for (int t1 = 0; t1 < 2; ++t1)
      for (int t2 = 0; t2 < (is3 ? 2 : 1); ++t2) {
        int i = 2 * I, j = 2 * J, k = is3 ? 2 * K : 0;
        if (d == 0) { j += t1; k += t2; }
        else if (d == 1) { i += t1; k += t2; }
        else { i += t1; j += t2; }
        if (i > Lf.nx || j > Lf.ny || k > Lf.nz) continue;
        // radial faces share their radius; axial faces weigh by column area
        const float w = (G == SFX_AXISYM && d == 1) ? vol_w<G>(i) : 1.0f;
        const float2 b = Bf[fidx(Lf, d, i, j, k)];
        num.x = __fmaf_rn(w, b.x, num.x);
        num.y = __fmaf_rn(w, b.y, num.y);
        den += w;
      }
    Bc[q] = make_float2(num.x / den, num.y / den);
  }
}

dim3 colour_grid(const Level& L) {
  return dim3((unsigned)(((L.nx + 1) / 2 + 127) / 128), (unsigned)L.ny, (unsigned)L.nz);
}

template <int G>
sfx_status cycle_impl(sfx_ctx* c, const Mg32Coef& kc, int nlev, int nu1, int nu2,
                      int coarse_sweeps, const int* done, cudaStream_t s) {
  std::vector<Mg32Level>& M = c->f32.mg;
  const Level& L0 = c->lev[0].lv;
  const Level& L1 = c->lev[1].lv;
  const int nd = L0.ndim();
  const __half2* Hz = nd == 3 ? c->f32.H2[2] : nullptr;
  SFX_KERNEL(c, K_RESTRICT, k_mg2_restrict_fine<G>, blocks_for(L1.ncell(), 256), 256, s,
             level_coef(L0, kc), L1, c->f32.H2[0], c->f32.H2[1], Hz, c->f32.rc, c->f32.e2,
             M[1].r, M[1].J, M[1].e, done);
  // down to the coarsest level
  for (int l = 1; l < nlev - 1; ++l) {
    const Level& L = c->lev[l].lv;
    const Nw32 p = level_coef(L, kc);
    for (int q = 0; q < nu1; ++q)
      for (int color = 0; color < 2; ++color)
        SFX_KERNEL(c, K_SMOOTH_COARSE, k_mg2_smooth<G>, colour_grid(L), 128, s, p, M[l].r,
                   M[l].J, M[l].B[0], M[l].B[1], M[l].B[2], M[l].e, color, done);
    const Level& Ln = c->lev[l + 1].lv;
    SFX_KERNEL(c, K_RESTRICT, k_mg2_restrict<G>, blocks_for(Ln.ncell(), 256), 256, s, p, Ln,
               M[l].r, M[l].J, M[l].B[0], M[l].B[1], M[l].B[2], M[l].e, M[l + 1].r,
               M[l + 1].J, M[l + 1].e, done);
  }
  {
    const int l = nlev - 1;
    const Level& L = c->lev[l].lv;
    const Nw32 p = level_coef(L, kc);
    if (L.ncell() <= 8192) {
      SFX_KERNEL(c, K_SMOOTH_COARSE, k_mg2_coarse<G>, 1, 1024, s, p, M[l].r, M[l].J, M[l].B[0],
                 M[l].B[1], M[l].B[2], M[l].e, coarse_sweeps, done);
    } else {
      for (int q = 0; q < coarse_sweeps; ++q)
        for (int color = 0; color < 2; ++color)
          SFX_KERNEL(c, K_SMOOTH_COARSE, k_mg2_smooth<G>, colour_grid(L), 128, s, p, M[l].r,
                     M[l].J, M[l].B[0], M[l].B[1], M[l].B[2], M[l].e, color, done);
    }
  }
  // back up
  for (int l = nlev - 2; l >= 1; --l) {
    const Level& L = c->lev[l].lv;
    SFX_KERNEL(c, K_PROLONG, k_mg2_prolong, blocks_for(L.ncell(), 256), 256, s,
               c->lev[l + 1].lv, L, M[l + 1].e, M[l].e, done);
    const Nw32 p = level_coef(L, kc);
    for (int q = 0; q < nu2; ++q)
      for (int color = 0; color < 2; ++color)
        SFX_KERNEL(c, K_SMOOTH_COARSE, k_mg2_smooth<G>, colour_grid(L), 128, s, p, M[l].r,
                   M[l].J, M[l].B[0], M[l].B[1], M[l].B[2], M[l].e, color, done);
  }
  SFX_KERNEL(c, K_PROLONG, k_mg2_prolong_fine, blocks_for(L0.ncell(), 256), 256, s, L1, L0,
             M[1].e, c->f32.e2, done);
  SFX_LAUNCH_CHECK();
  return SFX_OK;
}

template <int G>
sfx_status restrict_faces_impl(sfx_ctx* c, int nlev, cudaStream_t s) {
  std::vector<Mg32Level>& M = c->f32.mg;
  const int nd = c->lev[0].lv.ndim();
  for (int l = 1; l < nlev; ++l) {
    const Level& Lf = c->lev[l - 1].lv;
    const Level& Lc = c->lev[l].lv;
    for (int d = 0; d < nd; ++d) {
      const float2* src = l == 1 ? c->f32.B2[d] : M[l - 1].B[d];
      SFX_KERNEL(c, K_SETUP, k_mg2_restrict_faces<G>, blocks_for(Lc.nface(d), 256), 256, s, Lf,
                 Lc, d, src, M[l].B[d]);
    }
  }
  SFX_LAUNCH_CHECK();
  return SFX_OK;
}

}  // namespace

sfx_status mg32_prepare(sfx_ctx* c, int nlev, cudaStream_t s) {
  std::vector<Mg32Level>& M = c->f32.mg;
  if ((int)M.size() < nlev) M.resize(nlev);
  const int nd = c->lev[0].lv.ndim();
  for (int l = 1; l < nlev; ++l) {
    const Level& L = c->lev[l].lv;
    if (M[l].e) continue;
    void* p = nullptr;
    SFX_CUDA(cudaMalloc(&p, 3 * L.ncell() * sizeof(float2)));
    c->allocations.push_back(p);
    M[l].e = (float2*)p;
    M[l].r = M[l].e + L.ncell();
    M[l].J = M[l].r + L.ncell();
    for (int d = 0; d < nd; ++d) {
      SFX_CUDA(cudaMalloc(&p, L.nface(d) * sizeof(float2)));
      c->allocations.push_back(p);
      M[l].B[d] = (float2*)p;
    }
    c->f32.mg_epoch = ~0ull;   // new levels: restrict the faces again
  }
  if (c->f32.mg_epoch == c->f32.drift_epoch) return SFX_OK;
  sfx_status st;
  switch (c->lev[0].lv.geom) {
    case SFX_AXISYM: st = restrict_faces_impl<SFX_AXISYM>(c, nlev, s); break;
    case SFX_CART3D: st = restrict_faces_impl<SFX_CART3D>(c, nlev, s); break;
    default: st = restrict_faces_impl<SFX_PLANAR2D>(c, nlev, s); break;
  }
  if (st == SFX_OK) c->f32.mg_epoch = c->f32.drift_epoch;
  return st;
}

sfx_status mg32_cycle(sfx_ctx* c, const Mg32Coef& k, int nlev, int nu1, int nu2,
                      int coarse_sweeps, const int* done, cudaStream_t s) {
  switch (c->lev[0].lv.geom) {
    case SFX_AXISYM: return cycle_impl<SFX_AXISYM>(c, k, nlev, nu1, nu2, coarse_sweeps, done, s);
    case SFX_CART3D: return cycle_impl<SFX_CART3D>(c, k, nlev, nu1, nu2, coarse_sweeps, done, s);
    default: return cycle_impl<SFX_PLANAR2D>(c, k, nlev, nu1, nu2, coarse_sweeps, done, s);
  }
}

}  // namespace sfx
