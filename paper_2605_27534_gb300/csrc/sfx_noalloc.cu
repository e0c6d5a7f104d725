// sfx_totals_noalloc: the compensated totals of sfx_totals for callers that
// cannot allocate device memory.  Some callers may not call cudaMalloc:
// host programs whose device memory is owned by another allocator (a
// framework's caching pool or a fixed reservation), and code that must not
// pay the implicit device synchronisation of cudaMalloc/cudaFree.  Such a
// caller cannot create an sfx_ctx either, so this entry point takes the grid
// directly and keeps its scratch in a file-scope device array instead.
//
// The scratch (block partial sums and the per-field results) lives in
// `g_noalloc_scratch`, a static __device__ array of fixed size that every GPU
// loading the library holds until the process exits.  All calls share it and
// it keeps the last call's contents; every slot a call reads is written
// earlier in the same call, so nothing needs clearing.  Calls whose work
// overlaps on the GPU (different streams, no ordering between them) race on
// the array.
#include <cstring>
#include <mutex>

#include "sfx_internal.h"

namespace sfx {
namespace {

constexpr int kNaThreads = kTotalsThreads;
constexpr int kNaBlocks = kTotalsBlocks;
constexpr int kNaSlots = 2 * SFX_NOALLOC_MAX_FIELDS * kNaBlocks + SFX_NOALLOC_MAX_FIELDS;

// Device scratch: partial sums (s, c) per field and block, then one result
// per field.  In host code this name is only a stand-in for the symbol; its
// device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) double g_noalloc_scratch[kNaSlots];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_addr[kMaxDevices] = {};

// Once per device, with that device current: the device address of the
// scratch array.
sfx_status scratch_address(double** out) {
  int dev = 0;
  SFX_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return SFX_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    SFX_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_scratch_addr[dev] = (double*)p;
  }
  *out = g_scratch_addr[dev];
  return SFX_OK;
}

__global__ void k_na_partials(Level L, const double* __restrict__ x, int fi,
                              double* __restrict__ scratch) {
  const size_t n = L.ncell();
  double s = 0.0, cc = 0.0;
  for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n;
       c += (size_t)gridDim.x * blockDim.x) {
    double t, e;
    two_sum(s, cell_volume(L, (int)(c % L.nx)) * x[c], t, e);
    s = t;
    cc += e;
  }
  warp_sum_comp(s, cc);
  __shared__ double ws[kNaThreads / 32], wc[kNaThreads / 32];
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { ws[w] = s; wc[w] = cc; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = ws[0], b = wc[0];
    for (int q = 1; q < kNaThreads / 32; ++q) {
      double t, e;
      two_sum(a, ws[q], t, e);
      a = t;
      b += wc[q] + e;
    }
    scratch[2 * ((size_t)fi * kNaBlocks + blockIdx.x)] = a;
    scratch[2 * ((size_t)fi * kNaBlocks + blockIdx.x) + 1] = b;
  }
}

__global__ void k_na_final(double* __restrict__ scratch) {
  const int fi = blockIdx.x;
  double s = 0.0, cc = 0.0;
  for (int q = threadIdx.x; q < kNaBlocks; q += blockDim.x) {
    double t, e;
    two_sum(s, scratch[2 * (fi * kNaBlocks + q)], t, e);
    s = t;
    cc += scratch[2 * (fi * kNaBlocks + q) + 1] + e;
  }
  warp_sum_comp(s, cc);
  __shared__ double ws[kNaThreads / 32], wc[kNaThreads / 32];
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { ws[w] = s; wc[w] = cc; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = ws[0], b = wc[0];
    for (int q = 1; q < kNaThreads / 32; ++q) {
      double t, e;
      two_sum(a, ws[q], t, e);
      a = t;
      b += wc[q] + e;
    }
    scratch[2 * SFX_NOALLOC_MAX_FIELDS * kNaBlocks + fi] = a + b;
  }
}

bool noalloc_grid_ok(const sfx_grid* g) {
  return g && g->geom >= SFX_PLANAR2D && g->geom <= SFX_CART3D && g->nx >= 1 && g->ny >= 1 &&
         g->nz >= 1 && (g->geom == SFX_CART3D || g->nz == 1) && g->h > 0.0;
}

}  // namespace
}  // namespace sfx

extern "C" sfx_status sfx_totals_noalloc(const sfx_grid* grid, const double* const* fields,
                                         int n_fields, double* out, void* stream) {
  using namespace sfx;
  if (!noalloc_grid_ok(grid) || !fields || !out || n_fields < 1) return SFX_ERR_ARG;
  if (n_fields > SFX_NOALLOC_MAX_FIELDS) return SFX_ERR_WORKSPACE;
  for (int i = 0; i < n_fields; ++i)
    if (!fields[i]) return SFX_ERR_ARG;
  double* scratch = nullptr;
  sfx_status st = scratch_address(&scratch);
  if (st != SFX_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  Level L{grid->geom, grid->nx, grid->ny, grid->nz, grid->h};
  for (int i = 0; i < n_fields; ++i) k_na_partials<<<kNaBlocks, kNaThreads, 0, s>>>(L, fields[i], i, scratch);
  k_na_final<<<n_fields, kNaThreads, 0, s>>>(scratch);
  SFX_LAUNCH_CHECK();
  SFX_CUDA(cudaMemcpyAsync(out, scratch + 2 * SFX_NOALLOC_MAX_FIELDS * kNaBlocks,
                           n_fields * sizeof(double), cudaMemcpyDeviceToHost, s));
  SFX_CUDA(cudaStreamSynchronize(s));
  return SFX_OK;
}
