// Geometric VoF advection of the volume fraction C (the paper's interface
// tracking, Sec. 2): directionally split conservative PLIC advection.  For each direction d in turn, with face Courant numbers
// c_f = u_f dt/h,
//   C <- C - (Q_+ - Q_-) + H (c_+ - c_-),
// Q_f the volume fraction crossing face f (the fluid of the upwind cell's
// PLIC reconstruction within |c_f| h of the face, signed with u_f) and
// H = [C > 1/2] at the start of the step; the direction order alternates
// from step to step.  Walls carry no flux.  Planar 2D and 3D.  C is double
// in both precisions; SFX_F32 contexts evaluate the PLIC geometry of the
// fluxes in FP32.
#include <algorithm>

#include "sfx_internal.h"
#include "sfx_plic.cuh"

namespace sfx {
namespace {

__global__ void k_vof_indicator(size_t n, const double* __restrict__ C, double* __restrict__ H) {
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x)
    H[c] = C[c] > 0.5 ? 1.0 : 0.0;
}

// Volume fractions crossing the faces of direction d; blocks cover
// (x chunk, rows of faces) and walk the rows.  G is the arithmetic of the
// PLIC geometry (double in SFX_F64 contexts, float in SFX_F32 contexts: the
// fluxes then carry float rounding, while C and its update stay double and
// the update stays exactly conservative).
template <typename U, typename G>
__global__ void k_vof_flux(Level L, int d, const double* __restrict__ C,
                           const U* __restrict__ u, double dt_h, double* __restrict__ Q) {
  const int fx = L.nx + (d == 0), fy = L.ny + (d == 1), fz = L.nz + (d == 2);
  const int nd = L.ndim();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= fx) return;
  const unsigned rows = (unsigned)fy * (unsigned)fz;
  for (unsigned r = blockIdx.y; r < rows; r += gridDim.y) {
    const int j = (int)(r % (unsigned)fy), k = (int)(r / (unsigned)fy);
    const unsigned f = r * (unsigned)fx + (unsigned)i;
    const int pos = d == 0 ? i : (d == 1 ? j : k);
    if (pos == 0 || pos == L.extent(d)) {
      Q[f] = 0.0;
      continue;
    }
    // upwind cell: the one behind the face along the flow; both candidates
    // are loaded with u (independent of its sign), so the face costs one
    // round of loads rather than u and then C
    const double cf = (double)u[f] * dt_h;
    const double cm = C[cidx(L, i - (d == 0), j - (d == 1), k - (d == 2))];
    const double cq = C[cidx(L, i, j, k)];
    if (cf == 0.0) {
      Q[f] = 0.0;
      continue;
    }
    const int ui = (cf > 0.0 && d == 0) ? i - 1 : i;
    const int uj = (cf > 0.0 && d == 1) ? j - 1 : j;
    const int uk = (cf > 0.0 && d == 2) ? k - 1 : k;
    const double cu = cf > 0.0 ? cm : cq;
    G m[3] = {G(0), G(0), G(0)};
    if (cu > 0.0 && cu < 1.0) youngs_normal(L, C, ui, uj, uk, m);   // empty/full: no plane
    const G cg = (G)cu;
    Q[f] = cf > 0.0 ? (double)plic_slab<G>(nd, m, cg, d, G(1) - (G)cf, G(1))
                    : -(double)plic_slab<G>(nd, m, cg, d, G(0), (G)(-cf));
  }
}

template <typename U>
__global__ void k_vof_update(Level L, int d, const U* __restrict__ u, double dt_h,
                             const double* __restrict__ Q, const double* __restrict__ H,
                             double* __restrict__ C) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L.nx) return;
  const unsigned rows = (unsigned)L.ny * (unsigned)L.nz;
  for (unsigned r = blockIdx.y; r < rows; r += gridDim.y) {
    const int j = (int)(r % (unsigned)L.ny), k = (int)(r / (unsigned)L.ny);
    const unsigned c = r * (unsigned)L.nx + (unsigned)i;
    const size_t fm = fidx(L, d, i, j, k);
    const size_t fp = fidx(L, d, i + (d == 0), j + (d == 1), k + (d == 2));
    const double cm = (double)u[fm] * dt_h, cp = (double)u[fp] * dt_h;
    C[c] = C[c] - (Q[fp] - Q[fm]) + H[c] * (cp - cm);
  }
}

// (x chunks of up to 256 threads, row groups) for an x extent and a row count.
// One row per block where the grid allows it (up to 65535 row groups): a
// face or cell costs a few dependent loads, so the kernels are bound by
// latency, and a thread that walked ~50 rows in turn (8 blocks per SM)
// left the 256^3 flux pass at 11 % of DRAM bandwidth.
void rows_launch(int nxl, long long rows, dim3& grid, dim3& block) {
  const int tx = nxl >= 256 ? 256 : ((nxl + 31) / 32) * 32;
  const unsigned xb = (unsigned)((nxl + tx - 1) / tx);
  block = dim3(tx);
  grid = dim3(xb, (unsigned)std::min(std::max(rows, 1LL), 65535LL));
}

template <typename U, typename G>
sfx_status vof_impl(sfx_ctx* c, const U* const* u, double dt, int order, double* C,
                    cudaStream_t s) {
  const Level& L = c->lev[0].lv;
  const size_t n = L.ncell();
  const int nd = L.ndim();
  const double dt_h = dt / L.h;
  SFX_KERNEL(c, K_OTHER, k_vof_indicator, blocks_for(n, 256), 256, s, n, C, c->vofH);
  dim3 gc, bc;
  rows_launch(L.nx, (long long)L.ny * L.nz, gc, bc);
  for (int q = 0; q < nd; ++q) {
    const int d = order ? nd - 1 - q : q;
    dim3 gf, bf;
    rows_launch(L.nx + (d == 0), (long long)(L.ny + (d == 1)) * (L.nz + (d == 2)), gf, bf);
    SFX_KERNEL(c, K_OTHER, (k_vof_flux<U, G>), gf, bf, s, L, d, C, u[d], dt_h, c->vofQ);
    SFX_KERNEL(c, K_OTHER, (k_vof_update<U>), gc, bc, s, L, d, u[d], dt_h, c->vofQ, c->vofH, C);
  }
  SFX_LAUNCH_CHECK();
  return SFX_OK;
}

}  // namespace

sfx_status vof_advect(sfx_ctx* c, const void* ux, const void* uy, const void* uz, double dt,
                      int order, double* C, cudaStream_t s) {
  const Level& L = c->lev[0].lv;
  if (!c->vofH) {
    const size_t nf = std::max(std::max(L.nface(0), L.nface(1)), L.nface(2));
    SFX_CUDA(cudaMalloc((void**)&c->vofH, L.ncell() * sizeof(double)));
    c->allocations.push_back(c->vofH);
    SFX_CUDA(cudaMalloc((void**)&c->vofQ, nf * sizeof(double)));
    c->allocations.push_back(c->vofQ);
  }
  if (c->prec == SFX_F32) {
    const float* u[3] = {(const float*)ux, (const float*)uy, (const float*)uz};
    return vof_impl<float, float>(c, u, dt, order, C, s);
  }
  const double* u[3] = {(const double*)ux, (const double*)uy, (const double*)uz};
  return vof_impl<double, double>(c, u, dt, order, C, s);
}

}  // namespace sfx
