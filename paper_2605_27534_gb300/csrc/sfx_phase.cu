// Phase-field carrier from the VoF fraction (Sec. 2.5): signed distance by
// Hamilton-Jacobi redistancing, then the tanh profile and its regularised
// delta (Sec. 2.6).
//
// chi0 = 2h(C - 1/2) (positive inside fluid 1).  Each Jacobi step:
//   away from the interface  chi <- chi - dtau s (|grad chi|_G - 1)
//     with s = sign(chi0) and |grad chi|_G the first-order Godunov upwind
//     gradient;
//   in cells whose chi0 changes sign against a face neighbour (the
//   Russo-Smereka sub-cell fix)  chi <- chi - (dtau/h)(s |chi| - d)
//     with d = h chi0 / |Delta chi0| the distance estimated from chi0 alone.
#include <algorithm>
#include <cmath>

#include "sfx_internal.h"

namespace sfx {
namespace {

__global__ void k_chi0(size_t n, double h, const double* __restrict__ C, double* __restrict__ chi0,
                       double* __restrict__ chi) {
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x) {
    double v = 2.0 * h * (C[c] - 0.5);
    chi0[c] = v;
    chi[c] = v;
  }
}

template <typename T> __device__ __forceinline__ T tiny_pos();
template <> __device__ __forceinline__ double tiny_pos<double>() { return 1e-300; }
template <> __device__ __forceinline__ float tiny_pos<float>() { return 1e-30f; }

// One Jacobi update of chi at a cell from its own chi0 (s0) and iterate
// (x0) and those of its neighbours along each direction (the cell itself at
// a wall): Godunov upwind |grad chi| away from the interface, the
// Russo-Smereka sub-cell fix in cells where chi0 changes sign.
template <typename T>
__device__ __forceinline__ T redist_update(int nd, T s0, T x0, const T* z0m, const T* z0p,
                                           const T* xm, const T* xp, const bool* hasm,
                                           const bool* hasp, T h, T invh, T dtau, T dtau_h) {
  const T sg = s0 > (T)0 ? (T)1 : (s0 < (T)0 ? (T)-1 : (T)0);
  bool cut = false;
  T gsum = 0, dsum = 0;
  for (int d = 0; d < nd; ++d) {
    if ((hasm[d] && s0 * z0m[d] < (T)0) || (hasp[d] && s0 * z0p[d] < (T)0)) cut = true;
    // sub-cell estimate of |grad chi0| h along d
    T q = fabs(z0p[d] - z0m[d]) * (T)0.5;
    q = fmax(q, fabs(z0p[d] - s0));
    q = fmax(q, fabs(s0 - z0m[d]));
    dsum += q * q;
    // Godunov upwind gradient of the current iterate
    const T bwd = (x0 - xm[d]) * invh, fwd = (xp[d] - x0) * invh;
    T t;
    if (sg > (T)0) {
      const T ap = fmax(bwd, (T)0), bm = fmin(fwd, (T)0);
      t = fmax(ap * ap, bm * bm);
    } else {
      const T am = fmin(bwd, (T)0), bp = fmax(fwd, (T)0);
      t = fmax(am * am, bp * bp);
    }
    gsum += t;
  }
  if (cut) {
    const T dchi = fmax(sqrt(dsum), (T)tiny_pos<T>());
    return x0 - dtau_h * (sg * fabs(x0) - h * s0 / dchi);
  }
  return x0 - dtau * sg * (sqrt(gsum) - (T)1);
}

// One Jacobi step; blocks cover (x chunk, rows) and walk rows r = k ny + j.
template <typename T>
__global__ void k_redistance_step(Level L, T dtau, const T* __restrict__ chi0,
                                  const T* __restrict__ cin, T* __restrict__ cout) {
  const int nd = L.ndim();
  const T h = (T)L.h, invh = (T)(1.0 / L.h), dtau_h = dtau / h;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L.nx) return;
  const unsigned rows = (unsigned)L.ny * (unsigned)L.nz;
  const unsigned stride[3] = {1u, (unsigned)L.nx, (unsigned)L.nx * (unsigned)L.ny};
  for (unsigned r = blockIdx.y; r < rows; r += gridDim.y) {
    const int idx[3] = {i, (int)(r % (unsigned)L.ny), (int)(r / (unsigned)L.ny)};
    const unsigned c = r * (unsigned)L.nx + (unsigned)i;
    T z0m[3], z0p[3], xm[3], xp[3];
    bool hasm[3], hasp[3];
    for (int d = 0; d < nd; ++d) {
      hasm[d] = idx[d] > 0;
      hasp[d] = idx[d] + 1 < L.extent(d);
      const unsigned cm = hasm[d] ? c - stride[d] : c, cp = hasp[d] ? c + stride[d] : c;
      z0m[d] = chi0[cm];
      z0p[d] = chi0[cp];
      xm[d] = cin[cm];
      xp[d] = cin[cp];
    }
    cout[c] = redist_update<T>(nd, chi0[c], cin[c], z0m, z0p, xm, xp, hasm, hasp, h, invh, dtau,
                               dtau_h);
  }
}

// Up to kRdK Jacobi steps of a 2D grid in one launch: a block loads a
// (kRdX + 2 kRdK) x (kRdY + 2 kRdK) window of chi0 and the iterate into
// shared memory and updates a window that shrinks by one cell per step, so
// that after `steps` steps its kRdX x kRdY core holds exactly the values of
// `steps` single-step launches (the same update of the same operands).
constexpr int kRdX = 64, kRdY = 32, kRdK = 8;
constexpr int kRdWX = kRdX + 2 * kRdK, kRdWY = kRdY + 2 * kRdK;

__global__ void __launch_bounds__(256)
    k_redistance_fused2d(Level L, float dtau, const float* __restrict__ chi0,
                         const float* __restrict__ cin, float* __restrict__ cout, int steps) {
  __shared__ float sz[kRdWY][kRdWX];
  __shared__ float sx[2][kRdWY][kRdWX];
  const float h = (float)L.h, invh = (float)(1.0 / L.h), dtau_h = dtau / h;
  const int gx0 = blockIdx.x * kRdX - kRdK, gy0 = blockIdx.y * kRdY - kRdK;
  for (int q = threadIdx.x; q < kRdWX * kRdWY; q += blockDim.x) {
    const int lx = q % kRdWX, ly = q / kRdWX;
    const int gx = gx0 + lx, gy = gy0 + ly;
    float z = 0.0f, x = 0.0f;
    if (gx >= 0 && gx < L.nx && gy >= 0 && gy < L.ny) {
      const unsigned c = (unsigned)gy * (unsigned)L.nx + (unsigned)gx;
      z = chi0[c];
      x = cin[c];
    }
    sz[ly][lx] = z;
    sx[0][ly][lx] = x;
  }
  __syncthreads();
  int cur = 0;
  for (int st = 0; st < steps; ++st) {
    // cells at least st + 1 away from the window edge can be updated
    const int lo = st + 1, nxw = kRdWX - 2 * lo, nyw = kRdWY - 2 * lo;
    for (int q = threadIdx.x; q < nxw * nyw; q += blockDim.x) {
      const int lx = lo + q % nxw, ly = lo + q / nxw;
      const int gx = gx0 + lx, gy = gy0 + ly;
      if (gx < 0 || gx >= L.nx || gy < 0 || gy >= L.ny) continue;
      bool hasm[2] = {gx > 0, gy > 0}, hasp[2] = {gx + 1 < L.nx, gy + 1 < L.ny};
      const float s0 = sz[ly][lx], x0 = sx[cur][ly][lx];
      float z0m[2], z0p[2], xm[2], xp[2];
      z0m[0] = hasm[0] ? sz[ly][lx - 1] : s0;
      z0p[0] = hasp[0] ? sz[ly][lx + 1] : s0;
      z0m[1] = hasm[1] ? sz[ly - 1][lx] : s0;
      z0p[1] = hasp[1] ? sz[ly + 1][lx] : s0;
      xm[0] = hasm[0] ? sx[cur][ly][lx - 1] : x0;
      xp[0] = hasp[0] ? sx[cur][ly][lx + 1] : x0;
      xm[1] = hasm[1] ? sx[cur][ly - 1][lx] : x0;
      xp[1] = hasp[1] ? sx[cur][ly + 1][lx] : x0;
      sx[cur ^ 1][ly][lx] = redist_update<float>(2, s0, x0, z0m, z0p, xm, xp, hasm, hasp, h, invh,
                                                 dtau, dtau_h);
    }
    __syncthreads();
    cur ^= 1;
  }
  for (int q = threadIdx.x; q < kRdX * kRdY; q += blockDim.x) {
    const int lx = kRdK + q % kRdX, ly = kRdK + q / kRdX;
    const int gx = gx0 + lx, gy = gy0 + ly;
    if (gx < L.nx && gy < L.ny) cout[(unsigned)gy * (unsigned)L.nx + (unsigned)gx] = sx[cur][ly][lx];
  }
}

// SFX_F32 contexts iterate the redistancing in FP32 (their solution depends
// on phi only to ~1e-8 through it): chi0 and the float iterate.
__global__ void k_chi0_32(size_t n, double h, const double* __restrict__ C,
                          float* __restrict__ chi0, float* __restrict__ chi) {
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x) {
    const float v = (float)(2.0 * h * (C[c] - 0.5));
    chi0[c] = v;
    chi[c] = v;
  }
}

__global__ void k_widen(size_t n, const float* __restrict__ x, double* __restrict__ y) {
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x)
    y[c] = (double)x[c];
}

__global__ void k_phi_delta64(size_t n, double eps, const double* __restrict__ chi,
                              double* __restrict__ phi, double* __restrict__ delta) {
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x) {
    double p = 0.5 * (1.0 - tanh(chi[c] / (2.0 * eps)));
    phi[c] = p;
    if (delta) delta[c] = p * (1.0 - p) / eps;
  }
}

}  // namespace

sfx_status phase_field_build(sfx_ctx* c, const double* C, double* chi, void* phi, void* delta,
                             int iters, double dtau, double eps, cudaStream_t s) {
  const Level& L = c->lev[0].lv;
  const size_t n = L.ncell();
  const int nb = blocks_for(n, 256);
  const int tx = L.nx >= 256 ? 256 : ((L.nx + 31) / 32) * 32;
  const unsigned xb = (unsigned)((L.nx + tx - 1) / tx);
  const long long rows = (long long)L.ny * L.nz;
  // one row per block where the grid allows it: a redistancing step is a
  // short chain of dependent loads per cell, bound by latency (at 256^3 an
  // FP64 step took 2.7 ms with ~50 rows walked in turn per thread)
  const unsigned yb = (unsigned)std::min(std::max(rows, 1LL), 65535LL);
  if (c->prec == SFX_F32 && c->f32.redist32) {
    if (!c->chi32) {
      SFX_CUDA(cudaMalloc((void**)&c->chi32, 3 * n * sizeof(float)));
      c->allocations.push_back(c->chi32);
    }
    float* z0 = c->chi32;
    float* a = c->chi32 + n;
    float* b = c->chi32 + 2 * n;
    SFX_KERNEL(c, K_PHASE, k_chi0_32, nb, 256, s, n, L.h, C, z0, a);
    if (L.ndim() == 2) {
      // kRdK steps per launch
      const dim3 fg((unsigned)((L.nx + kRdX - 1) / kRdX), (unsigned)((L.ny + kRdY - 1) / kRdY));
      for (int it = 0; it < iters; it += kRdK) {
        const int steps = std::min(kRdK, iters - it);
        SFX_KERNEL(c, K_PHASE, k_redistance_fused2d, fg, 256, s, L, (float)dtau, z0, a, b, steps);
        float* t = a;
        a = b;
        b = t;
      }
    } else {
      for (int it = 0; it < iters; ++it) {
        SFX_KERNEL(c, K_PHASE, k_redistance_step<float>, dim3(xb, yb), dim3(tx), s, L,
                   (float)dtau, z0, a, b);
        float* t = a;
        a = b;
        b = t;
      }
    }
    SFX_KERNEL(c, K_PHASE, k_widen, nb, 256, s, n, a, chi);
    SFX_LAUNCH_CHECK();
  } else {
    SFX_KERNEL(c, K_PHASE, k_chi0, nb, 256, s, n, L.h, C, c->chi0, chi);
    SFX_LAUNCH_CHECK();
    double* a = chi;
    double* b = c->chi_tmp;
    for (int it = 0; it < iters; ++it) {
      SFX_KERNEL(c, K_PHASE, k_redistance_step<double>, dim3(xb, yb), dim3(tx), s, L, dtau,
                 c->chi0, a, b);
      double* t = a;
      a = b;
      b = t;
    }
    SFX_LAUNCH_CHECK();
    if (a != chi)
      SFX_CUDA(cudaMemcpyAsync(chi, a, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  SFX_KERNEL(c, K_PHASE, k_phi_delta64, nb, 256, s, n, eps, chi, (double*)phi, (double*)delta);
  SFX_LAUNCH_CHECK();
  return SFX_OK;
}

sfx_status phase_field_from_chi(sfx_ctx* c, const double* chi, double* phi, double* delta,
                                double eps, cudaStream_t s) {
  const size_t n = c->lev[0].lv.ncell();
  SFX_KERNEL(c, K_PHASE, k_phi_delta64, blocks_for(n, 256), 256, s, n, eps, chi, phi, delta);
  SFX_LAUNCH_CHECK();
  return SFX_OK;
}

}  // namespace sfx
