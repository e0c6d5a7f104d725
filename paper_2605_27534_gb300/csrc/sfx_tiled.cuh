// Tiled sweep of the coupled Newton correction (SFX_F32, 3D grids whose nx
// is a multiple of 8; included by sfx_f32.cu): one launch performs a whole
// red-black sweep, both colours, from shared memory.
//
// A block owns a tile of kTX x kTY cells of the (x, y) plane and a chunk of
// z-planes [z0, z1), and marches through the planes.  The tensor memory
// accelerator stages, per plane, the old corrections of colour B (tile + a
// 2-cell ring), the (r_f, r_F, u, v) float4 of both colours (tile + 1-cell
// ring) and the half-precision minus-side drifts (B_f, B_F) of the three
// face directions (colour-packed like the corrections) into a ring of plane
// slots, kInFlight planes ahead of the one being used.  (Each thread
// streaming its cells' float4 into registers instead, two steps ahead,
// made the sweep 26 % slower at 256^3.)  Step t updates the
// first colour A on plane t + 2 (the tile and its 1-cell ring: A cells read
// old B values only, so every block computes the same ring values as the
// block that owns them) and the second colour B on plane t (the tile, from
// the new A values of planes t - 1 .. t + 1).  The two updates of a step
// read and write disjoint data, so one block barrier per step orders
// everything.  Each cell's arithmetic is the 3D colour launch's
// (corr3_cell), so the sweep equals one B colour launch followed by one A
// colour launch bit for bit.  The corrections are read from one buffer and
// written to another: a block's ring reads must see the old values, which
// a neighbouring block may already have overwritten in place.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <type_traits>

#include "sfx_df.cuh"
#include "sfx_f32_dev.cuh"
#include "sfx_internal.h"

namespace sfx {
namespace {

constexpr int kTX = 64, kTY = 8;          // tile: cells along x, rows along y
constexpr int kPX = kTX / 2;              // packed positions of one colour per tile row
// staged boxes, per colour (packed positions x rows):
//   corrections: [ox/2 - 2, + kEX) x [oy - 2, + kEY)
//   float4:      [ox/2 - 1, + kRX) x [oy - 1, + kRY)
//   faces:       [ox/2 - 4, + kGX) x [oy - 1, + kFY)   (x start 16 B aligned)
constexpr int kEX = kPX + 4, kEY = kTY + 4;
constexpr int kRX = kPX + 2, kRY = kTY + 2;
constexpr int kGX = kPX + 8, kFY = kTY + 3;
constexpr int kFPad = 2 * kFY * kGX + 16;  // half2 entries per face array, to 128 B
#ifndef SFX_TILED_INFLIGHT
#define SFX_TILED_INFLIGHT 3
#endif
constexpr int kInFlight = SFX_TILED_INFLIGHT;   // planes staged ahead of the newest one in use
constexpr int kRing = 5 + kInFlight;      // a step uses planes t - 1 .. t + 3
// warps: B rows, A rows with the ring rows, the ring columns, the producer
constexpr int kBWarps = kTY, kAWarps = kTY + 3, kThreads = 32 * (kBWarps + kAWarps + 1);

struct TileSlot {
  float2 e[2][kEY][kEX];     // corrections (e_f, e_F): old B values (staged), new A values
  float4 r[2][kRY][kRX];     // (r_f, r_F, u, v) of both colours
  __half2 f[3][kFPad];       // minus-side drifts (B_f, B_F) of the x, y, z faces, [2][kFY][kGX]
};
static_assert(sizeof(TileSlot) % 128 == 0, "slots keep the bulk-copy destinations 128 B aligned");
static_assert(sizeof(float2) * 2 * kEY * kEX % 128 == 0 && sizeof(float4) * 2 * kRY * kRX % 128 == 0,
              "each staged array starts 128 B aligned");
static_assert(kFPad * sizeof(__half2) % 128 == 0, "face array padding");
constexpr unsigned kSlotBytes = (unsigned)(sizeof(float2) * kEY * kEX +
                                           sizeof(float4) * 2 * kRY * kRX +
                                           3 * sizeof(__half2) * 2 * kFY * kGX);
// the slots, then three barrier rings (planes staged, A planes done, slots
// free) and the abort flag
constexpr size_t kSmemBytes = kRing * sizeof(TileSlot) + 3 * kRing * sizeof(unsigned long long) + 16;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* b, unsigned bytes) {
  asm volatile(
      "{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}" ::"r"(
          smem_u32(b)),
      "r"(bytes)
      : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* b) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(smem_u32(b))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for a phase of a slot's barrier; gives up after one second (false).
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, unsigned parity) {
  if (mbar_try_wait(b, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(b, parity))
    if (global_ns() - t0 > 1000000000ull) return false;
  return true;
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* m, int x, int y, int z,
                                            int w, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(m)), "r"(x), "r"(y), "r"(z), "r"(w),
      "r"(smem_u32(bar))
      : "memory");
}
// A (black) is updated on the tile and its ring, B (red) on the tile
constexpr int cA = 1, cB = 0;

struct TiledArgs {
  Nw32 p;
  float2* eout;       // corrections written (colour-packed, the layout of the input)
  int zchunk;         // planes per block
  int* err;           // set to 1 when a staging wait gave up
  const int* done;    // the solve converged at an earlier iteration
};

// One cell of colour col from the slots of its plane (S0) and of the
// planes below (Sm) and above (Sp): pe, ye its packed position and row in
// the correction box (pe - 1 and ye - 1 in the float4 box, pe + 2 and
// ye - 1 in the face boxes), par = i & 1, w its open faces (1 or 0).
// Returns the new correction; keep: also leave it in the correction box.
__device__ __forceinline__ float2 tiled_cell(const Nw32& p, TileSlot& S0, const TileSlot& Sm,
                                             const TileSlot& Sp, int col, int pe, int ye,
                                             int par, const float* w, bool keep) {
  const int oc = 1 - col;
  // the other colour's neighbours: x at packed pe - 1 + par and pe + par,
  // y in the rows above and below, z in the planes below and above
  float2 nb[6];
  nb[0] = S0.e[oc][ye][pe - 1 + par];
  nb[1] = S0.e[oc][ye][pe + par];
  nb[2] = S0.e[oc][ye - 1][pe];
  nb[3] = S0.e[oc][ye + 1][pe];
  nb[4] = Sm.e[oc][ye][pe];
  nb[5] = Sp.e[oc][ye][pe];
  // minus faces are the cell's own; a plus face is the minus face of the
  // neighbour across it (the other colour): x at packed + par, y one row
  // up, z in the plane above
  const int pg = pe + 2, fy = ye - 1;
  const int own = (col * kFY + fy) * kGX + pg, oth = (oc * kFY + fy) * kGX + pg;
  __half2 hf[6];
  hf[0] = S0.f[0][own];
  hf[1] = S0.f[0][oth + par];
  hf[2] = S0.f[1][own];
  hf[3] = S0.f[1][oth + kGX];
  hf[4] = S0.f[2][own];
  hf[5] = Sp.f[2][oth];
  const float4 q4 = S0.r[col][ye - 1][pe - 1];
  float2 B[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) B[q] = __half22float2(hf[q]);
  const float2 ne = corr3_cell(p, nb, w, B, q4);
  if (keep) S0.e[col][ye][pe] = ne;
  // colour B (red) is staged: its old value is at hand for over-relaxation
  return col == cB ? relax_red(p, ne, S0.e[col][ye][pe]) : ne;
}

// The five copies of one plane into its slot, completing on the slot's
// barrier (issued by one thread).  Of the corrections only colour B is
// staged: the A cells' old values are never read (each update solves for
// the cell's new value from its neighbours), and their new values are
// written by the A updates of this launch.
struct TiledMaps {
  const CUtensorMap *e, *r, *fx, *fy, *fz;
};
__device__ __forceinline__ void stage_plane(const TiledMaps& tm, TileSlot& S,
                                            unsigned long long* bar, int ox, int oy, int m,
                                            int cB) {
  mbar_expect_tx(bar, kSlotBytes);
  tma_load_4d(&S.e[cB][0][0], tm.e, ox - 4, oy - 2, m, cB, bar);
  tma_load_4d(&S.r[0][0][0], tm.r, 2 * ox - 4, oy - 1, m, 0, bar);
  tma_load_4d(&S.f[0][0], tm.fx, ox / 2 - 4, oy - 1, m, 0, bar);
  tma_load_4d(&S.f[1][0], tm.fy, ox / 2 - 4, oy - 1, m, 0, bar);
  tma_load_4d(&S.f[2][0], tm.fz, ox / 2 - 4, oy - 1, m, 0, bar);
}

// Warp-specialised pipeline, no block barrier in the loop.  Plane m is
// staged plane q = m - z0 + 2 (planes z0 - 2 .. z1 + 1), in slot q % kRing,
// the u-th use of that slot (u = q / kRing; phase parity u & 1) for each of
// its three barriers:
//   full:  the slot's copies landed (the producer's expect_tx);
//   adone: the A warps finished plane m (one arrival per A warp);
//   empty: the B warps finished with the slot (one arrival per B warp).
// Producer (last warp, one lane): stage plane q once the slot's previous
// plane is released.  A warps: A on planes z0 - 1 .. z1 in order, each
// after its planes m - 1 .. m + 1 landed.  B warps: B on planes z0 .. z1 - 1
// in order, each after A finished plane t + 1 (so A finished t - 1 .. t
// too); B(t) is the last reader of plane t - 1 (A read it for A(t) and
// A(t - 1), both finished before A(t + 1)), so it then releases that slot.
// The A warps run ahead by up to kRing - 3 planes.  Every wait gives up
// after one second: that warp stops and records the error, the waits of
// the others then give up in turn, and the producer lets the copies it
// issued land before it exits.
__global__ void __launch_bounds__(kThreads, 1)
k_corr2_tiled(const __grid_constant__ CUtensorMap tm_e, const __grid_constant__ CUtensorMap tm_r,
              const __grid_constant__ CUtensorMap tm_fx, const __grid_constant__ CUtensorMap tm_fy,
              const __grid_constant__ CUtensorMap tm_fz, TiledArgs a) {
  if (a.done && *a.done) return;   // converged at an earlier iteration
  extern __shared__ __align__(128) unsigned char smem[];
  TileSlot* ring = reinterpret_cast<TileSlot*>(smem);
  unsigned long long* full = reinterpret_cast<unsigned long long*>(smem + kRing * sizeof(TileSlot));
  unsigned long long* adone = full + kRing;
  unsigned long long* empty = adone + kRing;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + kRing);
  const TiledMaps tm{&tm_e, &tm_r, &tm_fx, &tm_fy, &tm_fz};
  const Level& L = a.p.L;
  const int ox = blockIdx.x * kTX, oy = blockIdx.y * kTY;
  const int z0 = blockIdx.z * a.zchunk, z1 = min(z0 + a.zchunk, L.nz);
  const int nq = (z1 - z0) + 4;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int sl = 0; sl < kRing; ++sl) {
      mbar_init(&full[sl], 1);
      mbar_init(&adone[sl], kAWarps);
      mbar_init(&empty[sl], kBWarps);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto give_up = [&]() {
    *abort_flag = 1;
    atomicExch(a.err, 1);
  };
  const unsigned half = (unsigned)(L.nx >> 1);
  const size_t cplane = (size_t)L.ny * L.nz * half;

  if (warp == kBWarps + kAWarps) {
    // ---- producer
    if (lane != 0) return;
    int q = 0;
    for (; q < nq; ++q) {
      if (*abort_flag) break;
      const int sl = q % kRing;
      if (q >= kRing && !mbar_wait(&empty[sl], ((q - kRing) / kRing) & 1)) {
        give_up();
        break;
      }
      stage_plane(tm, ring[sl], &full[sl], ox, oy, z0 - 2 + q, cB);
    }
    if (*abort_flag) {
      // let the issued copies land before the block's shared memory goes
      for (int r = max(0, q - kRing); r < q; ++r) mbar_wait(&full[r % kRing], (r / kRing) & 1);
    }
    return;
  }

  const size_t pstride = (size_t)L.ny * half;   // one plane of one colour
  if (warp >= kBWarps) {
    // ---- A warps: rows -1 .. kTY (warps kBWarps .. kBWarps + kTY + 1) and
    // the ring columns (last A warp, lanes 0 .. kTY - 1: the A cell of the
    // row at x = ox - 1 or ox + kTX, whichever has colour A); one loop body
    // per kind (COLS a compile-time constant)
    auto a_loop = [&](auto cols_tag) {
      constexpr bool COLS = decltype(cols_tag)::value;
      const int jr = COLS ? lane : warp - kBWarps - 1;
      const int j = oy + jr;
      const bool active = !COLS || lane < kTY;
      const bool row_in = active && j >= 0 && j < L.ny;
      const float wym = j > 0 ? 1.0f : 0.0f, wyp = j + 1 < L.ny ? 1.0f : 0.0f;
      // x of the cell for par = 0 and 1 (rows: ox + 2 lane + par; columns:
      // ox + kTX (even) or ox - 1 (odd)), its walls and packed position
      const int i0 = COLS ? ox + kTX : ox + 2 * lane, i1 = COLS ? ox - 1 : ox + 2 * lane + 1;
      const bool in0 = row_in && i0 < L.nx, in1 = row_in && i1 >= 0 && i1 < L.nx;
      const float wxm0 = i0 > 0 ? 1.0f : 0.0f, wxp0 = i0 + 1 < L.nx ? 1.0f : 0.0f;
      const float wxm1 = i1 > 0 ? 1.0f : 0.0f, wxp1 = i1 + 1 < L.nx ? 1.0f : 0.0f;
      // rows store their tile cells: packed position ox/2 + lane of plane m
      const bool stores = !COLS && jr >= 0 && jr < kTY && j < L.ny;
      float2* out = stores ? a.eout + (size_t)cA * cplane + (size_t)j * half + (ox >> 1) + lane
                           : a.eout;
      for (int q = 0; q < 2; ++q)
        if (!mbar_wait(&full[q], 0)) give_up();
      // plane z0 - 2 has no A cells but takes the first phase of its slot's
      // barrier, like every staged plane
      if (lane == 0) mbar_arrive(&adone[0]);
      for (int m = z0 - 1; m <= z1; ++m) {
        const int qm = m - z0 + 2, qp = qm + 1;
        if (!mbar_wait(&full[qp % kRing], (qp / kRing) & 1)) {
          give_up();
          break;
        }
        if (active) {
          // colour A at (x, j, m): rows par = (j + m + cA) & 1; columns
          // par = 1 when x = ox - 1 has colour A
          const int par = COLS ? ((ox - 1 + j + m + cA) & 1) ^ 1 : (j + m + cA) & 1;
          const int pe = COLS ? (par ? 1 : kPX + 2) : lane + 2;
          TileSlot& S0 = ring[qm % kRing];
          if ((par ? in1 : in0) && m >= 0 && m < L.nz) {
            const float w[6] = {par ? wxm1 : wxm0, par ? wxp1 : wxp0, wym, wyp,
                                m > 0 ? 1.0f : 0.0f, m + 1 < L.nz ? 1.0f : 0.0f};
            const float2 ne = tiled_cell(a.p, S0, ring[(qm + kRing - 1) % kRing],
                                         ring[qp % kRing], cA, pe, jr + 2, par, w, true);
            if (stores && m >= z0 && m < z1) out[(size_t)m * pstride] = ne;
          } else {
            S0.e[cA][jr + 2][pe] = make_float2(0.0f, 0.0f);   // the neighbour of a wall
          }
        }
        // the slot is refilled by tensor copies later: order these shared
        // writes before them, then signal the plane done
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&adone[qm % kRing]);
      }
    };
    if (warp == kBWarps + kAWarps - 1)
      a_loop(std::true_type{});
    else
      a_loop(std::false_type{});
    return;
  }

  // ---- B warps: tile row jr = warp, cell x = ox + 2 lane + par (nx is a
  // multiple of 8: both parities are in or out together)
  const int jr = warp, j = oy + jr;
  const bool in = j < L.ny && ox + 2 * lane < L.nx;
  const float wym = j > 0 ? 1.0f : 0.0f, wyp = j + 1 < L.ny ? 1.0f : 0.0f;
  const int i0 = ox + 2 * lane, i1 = i0 + 1;
  const float wxm0 = i0 > 0 ? 1.0f : 0.0f, wxp0 = i0 + 1 < L.nx ? 1.0f : 0.0f;
  const float wxm1 = i1 > 0 ? 1.0f : 0.0f, wxp1 = i1 + 1 < L.nx ? 1.0f : 0.0f;
  float2* out = in ? a.eout + (size_t)cB * cplane + (size_t)j * half + (ox >> 1) + lane : a.eout;
  for (int t = z0; t < z1; ++t) {
    const int qt = t - z0 + 2, qp = qt + 1;
    // A finished plane t + 1 (and so t - 1 .. t); the planes' copies landed
    if (!mbar_wait(&adone[qp % kRing], (qp / kRing) & 1) ||
        !mbar_wait(&full[qp % kRing], (qp / kRing) & 1)) {
      give_up();
      break;
    }
    if (in) {
      const int par = (j + t + cB) & 1;
      const float w[6] = {par ? wxm1 : wxm0, par ? wxp1 : wxp0, wym, wyp, t > 0 ? 1.0f : 0.0f,
                          t + 1 < L.nz ? 1.0f : 0.0f};
      out[(size_t)t * pstride] = tiled_cell(a.p, ring[qt % kRing], ring[(qt - 1) % kRing],
                                            ring[qp % kRing], cB, lane + 2, jr + 2, par, w,
                                            false);
    }
    // the last reads of plane t - 1 (and, at the first plane, of z0 - 2,
    // which only the A warps read)
    __syncwarp();
    if (lane == 0) {
      mbar_arrive(&empty[(qt - 1) % kRing]);
      if (t == z0) mbar_arrive(&empty[0]);
    }
  }
}

// ---------------------------------------------------------------- host
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// A tensor map of 4-byte words: rank dims (innermost first), byte strides
// of dims 1 .. rank-1, the box; out-of-range words read as zeros.
sfx_status encode(CUtensorMap* m, void* base, int rank, const cuuint64_t* dims,
                  const cuuint64_t* strides, const cuuint32_t* box) {
  auto fn = encode_fn();
  if (!fn) return SFX_ERR_CUDA;
  const cuuint32_t es[4] = {1, 1, 1, 1};
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, base, dims, strides,
                        box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? SFX_OK : SFX_ERR_CUDA;
}

// 3D grids whose packed rows (nx/2 words of 4 bytes) are whole 16-byte units
bool tiled_sweep_eligible(const Level& L) {
  return L.geom == SFX_CART3D && L.nx % 8 == 0;
}

sfx_status tiled_sweep_prepare(sfx_ctx* c) {
  F32Scratch& S = c->f32;
  if (S.tiled_ready) return SFX_OK;
  const Level& L = c->lev[0].lv;
  if (!tiled_sweep_eligible(L) || !S.e2b || !S.Hm[0]) return SFX_ERR_ARG;
  static_assert(sizeof(CUtensorMap) == sizeof(S.tmaps[0]), "tensor map storage");
  const cuuint64_t half = (cuuint64_t)(L.nx / 2), ny = (cuuint64_t)L.ny, nz = (cuuint64_t)L.nz;
  sfx_status st;
  // corrections: float2 words [colour][nz][ny][half] as 4-byte words
  {
    const cuuint64_t dims[4] = {2 * half, ny, nz, 2};
    const cuuint64_t str[3] = {8 * half, 8 * half * ny, 8 * half * ny * nz};
    const cuuint32_t box[4] = {2 * kEX, kEY, 1, 1};   // one colour
    float2* bufs[2] = {S.e2, S.e2b};
    for (int b = 0; b < 2; ++b)
      if ((st = encode(reinterpret_cast<CUtensorMap*>(S.tmaps[b]), bufs[b], 4, dims, str, box)) !=
          SFX_OK)
        return st;
  }
  {
    // (r_f, r_F, u, v): float4 words [colour][nz][ny][half] as 4-byte words
    const cuuint64_t dims[4] = {4 * half, ny, nz, 2};
    const cuuint64_t str[3] = {16 * half, 16 * half * ny, 16 * half * ny * nz};
    const cuuint32_t box[4] = {4 * kRX, kRY, 1, 2};
    if ((st = encode(reinterpret_cast<CUtensorMap*>(S.tmaps[2]), S.rc, 4, dims, str, box)) != SFX_OK)
      return st;
  }
  {
    // minus-side face drifts, half2 words colour-packed like the corrections
    const cuuint64_t dims[4] = {half, ny, nz, 2};
    const cuuint64_t str[3] = {4 * half, 4 * half * ny, 4 * half * ny * nz};
    const cuuint32_t box[4] = {kGX, kFY, 1, 2};
    for (int d = 0; d < 3; ++d)
      if ((st = encode(reinterpret_cast<CUtensorMap*>(S.tmaps[3 + d]), S.Hm[d], 4, dims, str,
                       box)) != SFX_OK)
        return st;
  }
  SFX_CUDA(cudaFuncSetAttribute(k_corr2_tiled, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kSmemBytes));
  S.tiled_ready = true;
  return SFX_OK;
}

// Planes per block: one block per SM at a time, so the launch takes
// ceil(blocks / SMs) waves of blocks whose time grows with their planes
// plus the chunk's overhead (two extra A planes and the pipeline fill,
// about three planes); the chunk length in [4, 64] that minimises
// waves x (planes + 3).
int tiled_zchunk_auto(const Level& L, int sms) {
  const long long tiles = (long long)((L.nx + kTX - 1) / kTX) * ((L.ny + kTY - 1) / kTY);
  int best = 32;
  long long best_cost = -1;
  for (int zc = 4; zc <= 64; ++zc) {
    const long long chunks = (L.nz + zc - 1) / zc;
    const long long waves = (tiles * chunks + sms - 1) / sms;
    const long long cost = waves * (zc + 3);
    if (best_cost < 0 || cost < best_cost) {
      best = zc;
      best_cost = cost;
    }
  }
  return std::min(best, std::max(L.nz, 1));
}

sfx_status tiled_sweep(sfx_ctx* c, const Nw32& p, int in_buf, const int* done,
                       cudaStream_t s) {
  F32Scratch& S = c->f32;
  const Level& L = p.L;
  const int zc = S.tiled_zchunk > 0 ? S.tiled_zchunk : tiled_zchunk_auto(L, c->sm_count);
  TiledArgs a{p, in_buf == 0 ? S.e2b : S.e2, zc, S.flag + 3, done};
  const dim3 grd((unsigned)((L.nx + kTX - 1) / kTX), (unsigned)((L.ny + kTY - 1) / kTY),
                 (unsigned)((L.nz + zc - 1) / zc));
  const CUtensorMap* tm = reinterpret_cast<const CUtensorMap*>(S.tmaps);
  prof_before(c, K_SMOOTH_TILED, s);
  k_corr2_tiled<<<grd, kThreads, kSmemBytes, s>>>(tm[in_buf], tm[2], tm[3], tm[4], tm[5], a);
  prof_after(c, K_SMOOTH_TILED, s);
  SFX_LAUNCH_CHECK();
  return SFX_OK;
}

}  // namespace
}  // namespace sfx
