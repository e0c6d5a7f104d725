// BCG advection of both fields of an SFX_F32 context on 3D grids (Sec.
// 3.1), every face evaluated once, from shared-memory planes (included by
// sfx_f32.cu).
//
// A block of kA3X x kA3Y threads owns (kA3X - 1) x (kA3Y - 1) cells of the
// (x, y) plane and a chunk of z-planes.  Each plane of the chunk and its
// neighbours are staged once into a ring of kA3Ring slots: both fields'
// values (the pairs rounded to float, as the face values use them) on the
// tile with a 2-cell ring, their index clamped to the grid (so a neighbour
// past a wall reads the wall cell, which is the upwind cell itself there),
// and the three face velocity arrays on the tile with a 1-cell ring.
// Thread (tx, ty) evaluates the x face on the minus side of cell
// (ox + tx, oy + ty) (rows ty < kA3Y - 1) and the y face on its minus side
// (columns tx < kA3X - 1), shares them through shared memory, and carries
// the z face on the plus side of its cell to the next plane.  Each face
// value comes from bcg_face2 and each cell sums its fluxes in the order of
// advect_cell2, so the result is bitwise that of k_advect2t_32 and of the
// batched kernels.
#pragma once

#include "sfx_df.cuh"
#include "sfx_f32_dev.cuh"

namespace sfx {
namespace {

constexpr int kA3X = 32, kA3Y = 8;        // threads; cells (kA3X - 1) x (kA3Y - 1)
constexpr int kA3Z = 16;                  // planes per block
constexpr int kVX = kA3X + 3, kVY = kA3Y + 3;   // values: x [ox - 2, + kVX), y [oy - 2, + kVY)
constexpr int kUX = kA3X + 1, kUY = kA3Y + 1;   // velocities: x [ox - 1, + kUX), y [oy - 1, + kUY)
constexpr int kA3Ring = 4;                // planes k - 1 .. k + 2 (and k0 - 2 first)

struct Adv3Plane {
  float2 v[kVY][kVX];                     // (f, F) rounded to float
  float ux[kUY][kUX], uy[kUY][kUX], uz[kUY][kUX];   // faces on the minus sides of the cells
};

// What one thread stages of every plane: up to two value entries and up to
// two velocity entries of the boxes, with their plane-independent offsets
// and bounds, fixed for the block (so staging a plane costs an add and a
// predicated load per entry).
struct Adv3Stage {
  int vpos[2];          // flat position in the value box, -1: none
  unsigned vbase[2];    // clamped (i, j) of the cell
  int upos[2];          // flat position in the velocity boxes, -1: none
  unsigned ubase[3][2]; // face index of (i, j) in plane 0 for ux, uy, uz
  bool uin[3][2];       // (i, j) in the range of that face array
};

__device__ __forceinline__ Adv3Stage adv3_stage_init(const Level& L, int ox, int oy) {
  Adv3Stage S;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int q = threadIdx.x + r * blockDim.x;
    S.vpos[r] = q < kVX * kVY ? q : -1;
    const int x = q % kVX, y = q / kVX;
    const int i = min(max(ox - 2 + x, 0), L.nx - 1), j = min(max(oy - 2 + y, 0), L.ny - 1);
    S.vbase[r] = (unsigned)j * (unsigned)L.nx + (unsigned)i;
    S.upos[r] = q < kUX * kUY ? q : -1;
    const int xu = q % kUX, yu = q / kUX;
    const int iu = ox - 1 + xu, ju = oy - 1 + yu;
    S.uin[0][r] = iu >= 0 && iu <= L.nx && ju >= 0 && ju < L.ny;
    S.uin[1][r] = iu >= 0 && iu < L.nx && ju >= 0 && ju <= L.ny;
    S.uin[2][r] = iu >= 0 && iu < L.nx && ju >= 0 && ju < L.ny;
    S.ubase[0][r] = (unsigned)ju * (unsigned)(L.nx + 1) + (unsigned)iu;
    S.ubase[1][r] = (unsigned)ju * (unsigned)L.nx + (unsigned)iu;
    S.ubase[2][r] = (unsigned)ju * (unsigned)L.nx + (unsigned)iu;
  }
  return S;
}

// Stage plane m (values clamped to the grid, velocities zero outside it).
__device__ __forceinline__ void adv3_stage(const Adv32& A, const Adv3Stage& S,
                                           const float2* __restrict__ f,
                                           const float2* __restrict__ F, Adv3Plane& P, int m) {
  const Level& L = A.L;
  const unsigned plane = (unsigned)L.nx * (unsigned)L.ny;
  const unsigned vz = (unsigned)min(max(m, 0), L.nz - 1) * plane;
  float2* pv = &P.v[0][0];
#pragma unroll
  for (int r = 0; r < 2; ++r)
    if (S.vpos[r] >= 0) {
      const unsigned c = vz + S.vbase[r];
      pv[S.vpos[r]] = make_float2(df_val(f[c]), df_val(F[c]));
    }
  const bool m_in = m >= 0 && m < L.nz, mz_in = m >= 0 && m <= L.nz;
  const unsigned zx = (unsigned)m * (unsigned)L.ny * (unsigned)(L.nx + 1);
  const unsigned zy = (unsigned)m * (unsigned)(L.ny + 1) * (unsigned)L.nx;
  const unsigned zz = (unsigned)m * plane;
  float* px = &P.ux[0][0];
  float* py = &P.uy[0][0];
  float* pz = &P.uz[0][0];
#pragma unroll
  for (int r = 0; r < 2; ++r)
    if (S.upos[r] >= 0) {
      px[S.upos[r]] = (m_in && S.uin[0][r]) ? A.u[0][zx + S.ubase[0][r]] : 0.0f;
      py[S.upos[r]] = (m_in && S.uin[1][r]) ? A.u[1][zy + S.ubase[1][r]] : 0.0f;
      pz[S.upos[r]] = (mz_in && S.uin[2][r]) ? A.u[2][zz + S.ubase[2][r]] : 0.0f;
    }
}

// The weighted pair fluxes u v of one face for both fields, (f.hi, f.lo,
// F.hi, F.lo), the face on the minus side of cell (i, j, k) along d, from
// the staged planes; R(m) is the slot of plane m.
template <class Slot>
__device__ __forceinline__ float4 adv3_face(const Adv32& A, Slot R, float bc1, float bc2, int d,
                                            int i, int j, int k, float u, int ox, int oy) {
  if (u == 0.0f) return make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  const Level& L = A.L;
  const int pos = d == 0 ? i : (d == 1 ? j : k);
  float v1, v2;
  if ((u > 0.0f && pos == 0) || (u <= 0.0f && pos == L.extent(d))) {
    v1 = bc1;
    v2 = bc2;
  } else {
    // the upwind cell and its place in the staged boxes
    const int ui = i - (u > 0.0f && d == 0), uj = j - (u > 0.0f && d == 1),
              uk = k - (u > 0.0f && d == 2);
    const int x = ui - ox + 2, y = uj - oy + 2;
    const Adv3Plane& P0 = R(uk);
    const float2 a = P0.v[y][x];
    auto nb = [&](int t, int s) {
      return t == 0 ? P0.v[y][x + s] : (t == 1 ? P0.v[y + s][x] : R(uk + s).v[y][x]);
    };
    const int xu = ui - ox + 1, yu = uj - oy + 1;
    auto vb = [&](int t) {
      const float ua = t == 0 ? P0.ux[yu][xu] : (t == 1 ? P0.uy[yu][xu] : P0.uz[yu][xu]);
      const float ub = t == 0 ? P0.ux[yu][xu + 1]
                              : (t == 1 ? P0.uy[yu + 1][xu] : R(uk + 1).uz[yu][xu]);
      return __fmul_rn(0.5f, __fadd_rn(ua, ub));
    };
    bcg_face2(a, u, A.dt, A.invh, d, 3, nb, vb, v1, v2);
  }
  // u v as an exact pair (the unit area weight of 3D faces, which the
  // other kernels multiply in, leaves such a pair unchanged)
  const float p1 = __fmul_rn(u, v1), p2 = __fmul_rn(u, v2);
  return make_float4(p1, fmaf(u, v1, -p1), p2, fmaf(u, v2, -p2));
}

__global__ void __launch_bounds__(kA3X* kA3Y)
k_advect3s_32(Adv32 A, const float2* __restrict__ f, const float2* __restrict__ F, float bc_f,
              float bc_F, float2* __restrict__ fo, float2* __restrict__ Fo) {
  __shared__ Adv3Plane ring[kA3Ring];
  __shared__ float4 sx[kA3Y][kA3X];
  __shared__ float4 sy[kA3Y][kA3X];
  const Level& L = A.L;
  const int tx = threadIdx.x % kA3X, ty = threadIdx.x / kA3X;
  const int ox = blockIdx.x * (kA3X - 1), oy = blockIdx.y * (kA3Y - 1);
  const int i = ox + tx, j = oy + ty;
  const int k0 = blockIdx.z * kA3Z, k1 = min(k0 + kA3Z, L.nz);
  const bool cell = tx < kA3X - 1 && ty < kA3Y - 1 && i < L.nx && j < L.ny;
  auto R = [&](int m) -> Adv3Plane& { return ring[(m - k0 + 2 * kA3Ring) & (kA3Ring - 1)]; };
  const Adv3Stage St = adv3_stage_init(L, ox, oy);
  // planes k0 - 2 .. k0 + 1 for the first z face and the first plane
  for (int m = k0 - 2; m <= k0 + 1; ++m) adv3_stage(A, St, f, F, R(m), m);
  __syncthreads();
  float4 zm = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  float uzm = 0.0f;
  if (cell) {
    uzm = R(k0).uz[ty + 1][tx + 1];
    zm = adv3_face(A, R, bc_f, bc_F, 2, i, j, k0, uzm, ox, oy);
  }
  __syncthreads();   // the first z faces read plane k0 - 2, whose slot is refilled next
  for (int k = k0; k < k1; ++k) {
    // plane k + 2 into the slot plane k - 2 left (last read in step k - 1:
    // step k reads planes k - 1 .. k + 2)
    adv3_stage(A, St, f, F, R(k + 2), k + 2);
    __syncthreads();
    const Adv3Plane& P = R(k);
    float4 qx = make_float4(0.0f, 0.0f, 0.0f, 0.0f), qy = qx;
    if (ty < kA3Y - 1 && i <= L.nx && j < L.ny)
      qx = adv3_face(A, R, bc_f, bc_F, 0, i, j, k, P.ux[ty + 1][tx + 1], ox, oy);
    if (tx < kA3X - 1 && i < L.nx && j <= L.ny)
      qy = adv3_face(A, R, bc_f, bc_F, 1, i, j, k, P.uy[ty + 1][tx + 1], ox, oy);
    sx[ty][tx] = qx;
    sy[ty][tx] = qy;
    __syncthreads();
    if (cell) {
      float2 S1 = make_float2(0.0f, 0.0f), S2 = S1;
      const float uxm = P.ux[ty + 1][tx + 1], uxp = P.ux[ty + 1][tx + 2];
      const float uym = P.uy[ty + 1][tx + 1], uyp = P.uy[ty + 2][tx + 1];
      const float uzp = R(k + 1).uz[ty + 1][tx + 1];
      if (uxm != 0.0f) acc_face(S1, S2, sx[ty][tx], false);
      if (uxp != 0.0f) acc_face(S1, S2, sx[ty][tx + 1], true);
      if (uym != 0.0f) acc_face(S1, S2, sy[ty][tx], false);
      if (uyp != 0.0f) acc_face(S1, S2, sy[ty + 1][tx], true);
      const float4 zp = adv3_face(A, R, bc_f, bc_F, 2, i, j, k + 1, uzp, ox, oy);
      if (uzm != 0.0f) acc_face(S1, S2, zm, false);
      if (uzp != 0.0f) acc_face(S1, S2, zp, true);
      zm = zp;
      uzm = uzp;
      const float2 i1 = df_mul_f(df_mul_f(S1, -A.dt), A.invh);
      const float2 i2 = df_mul_f(df_mul_f(S2, -A.dt), A.invh);
      const ix c = cidx32(L, i, j, k);
      fo[c] = df_add2(f[c], i1);
      Fo[c] = df_add2(F[c], i2);
    }
    __syncthreads();
  }
}

}  // namespace
}  // namespace sfx
