// Batched SFX_F32 step over many independent axisymmetric instances of
// uneven sizes and parameters.
//
// Every phase of the coupled step (drift faces, BCG advection, the coupled
// Newton residual, the coupled correction sweeps, per-instance convergence
// flags, per-instance totals) is one kernel over all instances: blocks are
// dealt to instances through prefix tables, so a block never straddles two
// instances.  An instance whose residuals pass the tolerance is switched off
// and its blocks return at once.  The whole step is captured into a CUDA
// graph on first use (and again when a pointer or the schedule changes) and
// replayed, one graph launch per step with no host synchronisation.  The
// per-cell arithmetic is the single-grid SFX_F32 code (sfx_f32_dev.cuh).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "sfx_df.cuh"
#include "sfx_f32_dev.cuh"
#include "sfx_internal.h"

namespace sfx {
namespace {

struct BInst {
  Nw32 p;                 // grid (axisymmetric, nx = nr, ny = nz) and coefficients
  float dt, bc_f, bc_F, Df, DF;
  size_t coff, rfoff, zfoff;    // offsets of cells, radial faces, axial faces
  size_t poff;                  // offset of the colour-packed Newton work arrays
};

// block -> instance through a prefix table of block counts
__device__ __forceinline__ int find_inst(const int* __restrict__ pre, int n, int b) {
  int lo = 0, hi = n;   // pre[lo] <= b < pre[hi]
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (pre[mid] <= b) lo = mid;
    else hi = mid;
  }
  return lo;
}

struct BPtr {
  const double* phi;      // phase field (caller's)
  float* phi32;           // its folded float copy
  const float* ur;
  const float* uz;
  float2* f;
  float2* F;
  float2* fs;
  float2* Fs;
  float2* B2[2];          // radial, axial drift faces (B_f, B_F)
  __half2* H2[2];         // (B_f, B_F) in half precision (correction sweeps)
  float4* rc;             // r_f, r_F, u = c1 F, v = c1 (f_inf - f) per cell (colour-packed)
  float2* e2;             // Newton corrections (e_f, e_F), colour-packed
  unsigned int* norms;    // 4 per instance
  int* rkind;             // 2 per instance: residual kind (0 FP32, 1 pair), FP32 passes so far
  int* active;
  int* iters;
  float* rres;            // 2 per instance: last relative residuals
  double* mass;           // 2 per instance
  unsigned long long* work;   // 2 per instance: residual passes, sweep groups
  int* loop;              // Newton iterations done in the current step
  float* part;            // per cell block: the 4 residual maxima
  double* tpart;          // per cell block: (s, c) compensated sums of f and F
};

// drift faces: blocks over radial faces then axial faces of every instance
__global__ void k_b_drift(const BInst* __restrict__ I, int n, const int* __restrict__ pre, int dir,
                          BPtr P) {
  const int inst = find_inst(pre, n, blockIdx.x);
  const BInst& B = I[inst];
  const Level& L = B.p.L;
  const size_t nf = L.nface(dir);
  const size_t q = (size_t)(blockIdx.x - pre[inst]) * blockDim.x + threadIdx.x;
  if (q >= nf) return;
  const size_t fo = dir == 0 ? B.rfoff : B.zfoff;
  float2* B2 = P.B2[dir] + fo;
  const double* phi = P.phi + B.coff;
  const int fx = L.nx + (dir == 0);
  const int i = (int)(q % fx), j = (int)(q / fx);
  const int pos = dir == 0 ? i : j;
  float bf = 0.0f, bF = 0.0f;
  if (pos > 0 && pos < L.extent(dir)) {
    const int li = i - (dir == 0), lj = j - (dir == 1);
    const float sL = fold_phi(phi[cidx(L, li, lj, 0)]), sR = fold_phi(phi[cidx(L, i, j, 0)]);
    const float nL = normal_f32(L, phi, li, lj, 0, dir, B.p.inv_eps);
    const float nR = normal_f32(L, phi, i, j, 0, dir, B.p.inv_eps);
    drift_face(sL, sR, nL, nR, B.Df, B.DF, B.p.inv_eps, bf, bF);
  }
  B2[q] = make_float2(bf, bF);
  P.H2[dir][fo + q] = __floats2half2_rn(bf, bF);
}

__global__ void k_b_advect(const BInst* __restrict__ I, int n, const int* __restrict__ pre, BPtr P) {
  const int inst = find_inst(pre, n, blockIdx.x);
  const BInst& B = I[inst];
  const Level& L = B.p.L;
  const size_t c = (size_t)(blockIdx.x - pre[inst]) * blockDim.x + threadIdx.x;
  if (c >= L.ncell()) return;
  Adv32 A{L, B.dt, B.p.invh, {P.ur + B.rfoff, P.uz + B.zfoff, nullptr}};
  const int i = (int)((ix)c % (ix)L.nx), j = (int)((ix)c / (ix)L.nx);
  advect_cell2(A, P.f + B.coff, P.F + B.coff, B.bc_f, B.bc_F, i, j, 0, (ix)c, P.fs[B.coff + c],
               P.Fs[B.coff + c]);
}

// folded float copy of phi, and the start of the step
__global__ void k_b_fold(const BInst* __restrict__ I, int n, const int* __restrict__ pre, BPtr P) {
  const int inst = find_inst(pre, n, blockIdx.x);
  const BInst& B = I[inst];
  const size_t c = (size_t)(blockIdx.x - pre[inst]) * blockDim.x + threadIdx.x;
  if (c >= B.p.L.ncell()) return;
  P.phi32[B.coff + c] = fold_phi(P.phi[B.coff + c]);
}

// state <- post-advection fields (the Newton iteration starts there)
__global__ void k_b_copy(const BInst* __restrict__ I, int n, const int* __restrict__ pre, BPtr P,
                         int from_star) {
  const int inst = find_inst(pre, n, blockIdx.x);
  const BInst& B = I[inst];
  const size_t c = (size_t)(blockIdx.x - pre[inst]) * blockDim.x + threadIdx.x;
  if (c >= B.p.L.ncell()) return;
  const size_t g = B.coff + c;
  if (from_star) { P.f[g] = P.fs[g]; P.F[g] = P.Fs[g]; }
  else { P.fs[g] = P.f[g]; P.Fs[g] = P.F[g]; }
}

__global__ void k_b_init(int n, BPtr P, int fast) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) *P.loop = 0;
  if (i >= n) return;
  P.active[i] = 1;
  P.iters[i] = 0;
  P.rkind[2 * i] = fast > 0 ? 0 : 1;
  P.rkind[2 * i + 1] = 0;
  for (int q = 0; q < 4; ++q) P.norms[4 * i + q] = 0u;
}

// G: the geometry of every instance of the batch (compile time, as in the
// single-grid Newton kernels, so that both run the same cell arithmetic)
template <int G>
__global__ void k_b_resid(const BInst* __restrict__ I, int n, const int* __restrict__ pre, BPtr P) {
  const int inst = find_inst(pre, n, blockIdx.x);
  if (!P.active[inst]) return;
  const BInst& B = I[inst];
  const Level& L = B.p.L;
  const size_t c = (size_t)(blockIdx.x - pre[inst]) * blockDim.x + threadIdx.x;
  float m[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  if (c < L.ncell()) {
    const int i = (int)((ix)c % (ix)L.nx), j = (int)((ix)c / (ix)L.nx);
    const float2* B2[3] = {P.B2[0] + B.rfoff, P.B2[1] + B.zfoff, nullptr};
    const size_t o = B.coff, w = B.poff;
    // the FP32 residual for the instance's first iterations (the kind is
    // the same for every block of an instance)
    if (P.rkind[2 * inst] == 0)
      resid32_cell<G>(B.p, i, j, 0, c, P.phi32 + o, B2, P.f + o, P.F + o, P.fs + o, P.Fs + o,
                      P.rc + w, m, P.e2 + w);
    else
      resid2_cell<G>(B.p, i, j, 0, c, P.phi32 + o, B2, P.f + o, P.F + o, P.fs + o, P.Fs + o,
                     P.rc + w, m, P.e2 + w);
  }
  // block maxima; the flags kernel combines the blocks of each instance
  __shared__ float wm[4][16];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float v = warp_max(m[q]);
    if ((threadIdx.x & 31) == 0) wm[q][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    float v = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v = fmaxf(v, wm[threadIdx.x][w]);
    P.part[4 * (size_t)blockIdx.x + threadIdx.x] = v;
  }
}

// convergence test of the current iteration: one block per instance still
// active combines the residual maxima of the instance's blocks
__global__ void k_b_flags(int n, const int* __restrict__ pre, BPtr P, float tol, int fast) {
  const int i = blockIdx.x;
  if (i >= n || !P.active[i]) return;
  const int it = *P.loop + 1;
  float mx[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  for (int b = pre[i] + threadIdx.x; b < pre[i + 1]; b += blockDim.x)
#pragma unroll
    for (int q = 0; q < 4; ++q) mx[q] = fmaxf(mx[q], P.part[4 * (size_t)b + q]);
  __shared__ float wm[4][8];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    mx[q] = warp_max(mx[q]);
    if ((threadIdx.x & 31) == 0) wm[q][threadIdx.x >> 5] = mx[q];
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
#pragma unroll
    for (int q = 0; q < 4; ++q) mx[q] = fmaxf(mx[q], wm[q][w]);
  const float rf = mx[0], bf = mx[1], rF = mx[2], bF = mx[3];
  P.rres[2 * i] = rf / fmaxf(bf, 1e-30f);
  P.rres[2 * i + 1] = rF / fmaxf(bF, 1e-30f);
  P.iters[i] = it;
  P.work[2 * i] += 1;
  if (P.rkind[2 * i] != 0 && rf <= tol * bf && rF <= tol * bF) {
    P.active[i] = 0;   // converged on a pair residual: stop here
    return;
  }
  P.work[2 * i + 1] += 1;   // the sweeps run
  // after `fast` FP32 passes, or once the residuals are small, the pair
  // residual (as the single-grid solve switches)
  if (P.rkind[2 * i] == 0 && (++P.rkind[2 * i + 1] >= fast ||
                              (rf <= kFastResidSwitch * bf && rF <= kFastResidSwitch * bF)))
    P.rkind[2 * i] = 1;
}

// end of an iteration: count it, and let the step's loop run again while
// an instance is active and the iteration budget lasts
__global__ void k_b_next(int n, BPtr P, int max_it, cudaGraphConditionalHandle loop) {
  int any = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) any |= P.active[i];
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) {
    const int done = *P.loop + 1;
    *P.loop = done;
    cudaGraphSetConditional(loop, (any && done < max_it) ? 1u : 0u);
  }
}

// one colour of the coupled correction sweep; blocks over half-rows
template <int G>
__global__ void k_b_corr(const BInst* __restrict__ I, int n, const int* __restrict__ pre, BPtr P,
                         int color, int first, int apply) {
  const int inst = find_inst(pre, n, blockIdx.x);
  if (!P.active[inst]) return;
  const BInst& B = I[inst];
  const Level& L = B.p.L;
  const int half = (L.nx + 1) / 2;
  const size_t t = (size_t)(blockIdx.x - pre[inst]) * blockDim.x + threadIdx.x;
  if (t >= (size_t)half * L.ny) return;
  const int j = (int)(t / half);
  const int i = 2 * (int)(t % half) + ((j + color) & 1);
  const size_t o = B.coff, w = B.poff;
  float2* fst = apply ? P.f + o : nullptr;
  float2* Fst = apply ? P.F + o : nullptr;
  if (i >= L.nx) {
    const int ir = i ^ 1;
    if (apply && ir < L.nx) {
      const size_t cr = cidx(L, ir, j, 0);
      const RBIdx rb = rb_index(L, i, j, 0);
      const size_t pr = w + (1 - color) * rb.plane + rb.pos;   // ir's packed slot
      const float2 er = P.e2[pr];
      fst[cr] = df_add(fst[cr], er.x);
      Fst[cr] = df_add(Fst[cr], er.y);
    }
    return;
  }
  const __half2* H[3] = {P.H2[0] + B.rfoff, P.H2[1] + B.zfoff, nullptr};
  corr2_cell<G>(B.p, i, j, 0, H, P.rc + w, P.e2 + w, color, first, fst, Fst, fst, Fst);
}

// per-instance compensated totals: kTotBlocks blocks per instance each walk
// a share of its cells, accumulate both fields in double-float pairs and
// combine their threads in compensated doubles ...
constexpr int kTotBlocks = 8;
__global__ void k_b_totals(const BInst* __restrict__ I, BPtr P) {
  const int inst = blockIdx.x / kTotBlocks, part = blockIdx.x % kTotBlocks;
  const BInst& B = I[inst];
  const Level& L = B.p.L;
  const ix n = (ix)L.ncell(), nx = (ix)L.nx;
  float2 acc[2] = {make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f)};
  for (ix c = part * blockDim.x + threadIdx.x; c < n; c += kTotBlocks * blockDim.x) {
    // ring volume / (pi h^3), or 1 for planar cells (volume h^2)
    const float w = L.geom == SFX_AXISYM ? 2.0f * (float)(c % nx) + 1.0f : 1.0f;
#pragma unroll
    for (int fld = 0; fld < 2; ++fld) {
      float2 v = (fld ? P.F : P.f)[B.coff + c];
      const float pr = v.x * w;
      v = make_float2(pr, fmaf(v.x, w, -pr) + v.y * w);
      acc[fld] = df_add2(acc[fld], v);
    }
  }
  __shared__ double ss[2][16], sc[2][16];
#pragma unroll
  for (int fld = 0; fld < 2; ++fld) {
    double s = (double)acc[fld].x, cc = (double)acc[fld].y;
    warp_sum_comp(s, cc);
    if ((threadIdx.x & 31) == 0) {
      ss[fld][threadIdx.x >> 5] = s;
      sc[fld][threadIdx.x >> 5] = cc;
    }
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    const int fld = threadIdx.x;
    double a = ss[fld][0], b = sc[fld][0];
    for (int q = 1; q < (int)(blockDim.x >> 5); ++q) {
      double t, e;
      two_sum(a, ss[fld][q], t, e);
      a = t;
      b += sc[fld][q] + e;
    }
    P.tpart[4 * (size_t)blockIdx.x + 2 * fld] = a;
    P.tpart[4 * (size_t)blockIdx.x + 2 * fld + 1] = b;
  }
}

// ... and one warp per instance combines its blocks in a fixed order
__global__ void k_b_totals_final(const BInst* __restrict__ I, int n, BPtr P) {
  const int inst = blockIdx.x;
  if (inst >= n) return;
  for (int fld = 0; fld < 2; ++fld) {
    double s = 0.0, cc = 0.0;
    for (int b = inst * kTotBlocks + threadIdx.x; b < (inst + 1) * kTotBlocks; b += blockDim.x) {
      double t, e;
      two_sum(s, P.tpart[4 * (size_t)b + 2 * fld], t, e);
      s = t;
      cc += P.tpart[4 * (size_t)b + 2 * fld + 1] + e;
    }
    warp_sum_comp(s, cc);
    if (threadIdx.x == 0) {
      const Level& L = I[inst].p.L;
      const double h = L.h;
      P.mass[2 * inst + fld] = (s + cc) * (L.geom == SFX_AXISYM ? kPi * h * h * h : h * h);
    }
  }
}

}  // namespace
}  // namespace sfx

using namespace sfx;

struct sfx_batch {
  int n = 0;
  std::vector<sfx_batch_instance> hinst;
  std::vector<BInst> hI;
  size_t ncell = 0, nrf = 0, nzf = 0, npack = 0;
  std::vector<size_t> coff, rfoff, zfoff;
  BInst* dI = nullptr;
  int* pre_cell = nullptr;   // blocks of `block` threads over cells
  int* pre_rf = nullptr;
  int* pre_zf = nullptr;
  int* pre_pair = nullptr;
  int nb_cell = 0, nb_rf = 0, nb_zf = 0, nb_pair = 0;
  int block = 256;
  int geom = SFX_AXISYM;   // of every instance
  BPtr P{};
  std::vector<void*> allocs;
  // graph cache
  cudaGraphExec_t exec = nullptr;
  const void* key[5] = {};
  int key_sched[6] = {};
  bool reuse_phi = false;         // phi static: fold and drifts outside the graph
  const void* drift_phi = nullptr;
  double key_tol = 0;
  cudaStream_t cap = nullptr;
  cudaStream_t cap_body = nullptr;   // captures the body of the iteration loop
  // last schedule
  int sweeps = 3, max_it = 8;
  int fast = 2;                   // FP32 residual passes at most per instance and step
  int sor = 1;                    // over-relaxed red updates (as SFX_TUNE_F32_SOR)
  std::vector<int> h_iters;
};

namespace {

template <typename T>
sfx_status balloc(sfx_batch* b, T** p, size_t n) {
  void* q = nullptr;
  SFX_CUDA(cudaMalloc(&q, (n ? n : 1) * sizeof(T)));
  b->allocs.push_back(q);
  *p = (T*)q;
  return SFX_OK;
}

// prefix tables of blocks per instance for the current block size
sfx_status build_prefix(sfx_batch* b) {
  const int bs = b->block;
  std::vector<int> pc(b->n + 1), pr(b->n + 1), pz(b->n + 1), pp(b->n + 1);
  pc[0] = pr[0] = pz[0] = pp[0] = 0;
  for (int i = 0; i < b->n; ++i) {
    const Level& L = b->hI[i].p.L;
    pc[i + 1] = pc[i] + (int)((L.ncell() + bs - 1) / bs);
    pr[i + 1] = pr[i] + (int)((L.nface(0) + bs - 1) / bs);
    pz[i + 1] = pz[i] + (int)((L.nface(1) + bs - 1) / bs);
    pp[i + 1] = pp[i] + (int)(((size_t)((L.nx + 1) / 2) * L.ny + bs - 1) / bs);
  }
  b->nb_cell = pc[b->n];
  b->nb_rf = pr[b->n];
  b->nb_zf = pz[b->n];
  b->nb_pair = pp[b->n];
  SFX_CUDA(cudaMemcpy(b->pre_cell, pc.data(), pc.size() * sizeof(int), cudaMemcpyHostToDevice));
  SFX_CUDA(cudaMemcpy(b->pre_rf, pr.data(), pr.size() * sizeof(int), cudaMemcpyHostToDevice));
  SFX_CUDA(cudaMemcpy(b->pre_zf, pz.data(), pz.size() * sizeof(int), cudaMemcpyHostToDevice));
  SFX_CUDA(cudaMemcpy(b->pre_pair, pp.data(), pp.size() * sizeof(int), cudaMemcpyHostToDevice));
  return SFX_OK;
}

// Enqueue one batched step on s under stream capture: the set-up kernels,
// the Newton iterations as the body of a conditional while node (run again
// while an instance is active and the budget lasts, so a step whose
// instances converge early launches no further kernels), then the totals.
sfx_status enqueue_step(sfx_batch* b, bool advect, float tol, cudaStream_t s) {
  const int n = b->n, bs = b->block;
  BPtr& P = b->P;
  k_b_init<<<(n + 127) / 128, 128, 0, s>>>(n, P, b->fast);
  if (!b->reuse_phi) {
    k_b_fold<<<b->nb_cell, bs, 0, s>>>(b->dI, n, b->pre_cell, P);
    k_b_drift<<<b->nb_rf, bs, 0, s>>>(b->dI, n, b->pre_rf, 0, P);
    k_b_drift<<<b->nb_zf, bs, 0, s>>>(b->dI, n, b->pre_zf, 1, P);
  }
  if (advect) {
    k_b_advect<<<b->nb_cell, bs, 0, s>>>(b->dI, n, b->pre_cell, P);
    k_b_copy<<<b->nb_cell, bs, 0, s>>>(b->dI, n, b->pre_cell, P, 1);
  } else {
    k_b_copy<<<b->nb_cell, bs, 0, s>>>(b->dI, n, b->pre_cell, P, 0);
  }
  SFX_LAUNCH_CHECK();
  // the while node, after everything captured so far
  cudaStreamCaptureStatus cs;
  cudaGraph_t cg = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  SFX_CUDA(cudaStreamGetCaptureInfo(s, &cs, nullptr, &cg, &deps, nullptr, &ndeps));
  cudaGraphConditionalHandle loop;
  SFX_CUDA(cudaGraphConditionalHandleCreate(&loop, cg, 1u, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = loop;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cnode;
  SFX_CUDA(cudaGraphAddNode(&cnode, cg, deps, nullptr, ndeps, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  if (!b->cap_body) SFX_CUDA(cudaStreamCreateWithFlags(&b->cap_body, cudaStreamNonBlocking));
  cudaStream_t sb = b->cap_body;
  SFX_CUDA(cudaStreamBeginCaptureToGraph(sb, body, nullptr, nullptr, 0,
                                         cudaStreamCaptureModeThreadLocal));
  const bool axi = b->geom == SFX_AXISYM;
  auto resid = axi ? &k_b_resid<SFX_AXISYM> : &k_b_resid<SFX_PLANAR2D>;
  auto corr = axi ? &k_b_corr<SFX_AXISYM> : &k_b_corr<SFX_PLANAR2D>;
  resid<<<b->nb_cell, bs, 0, sb>>>(b->dI, n, b->pre_cell, P);
  k_b_flags<<<n, 256, 0, sb>>>(n, b->pre_cell, P, tol, b->fast);
  // the residual pass did the first red half-sweep
  for (int q = 0; q < b->sweeps; ++q)
    for (int color = (q == 0 ? 1 : 0); color < 2; ++color)
      corr<<<b->nb_pair, bs, 0, sb>>>(b->dI, n, b->pre_pair, P, color, q == 0 ? 1 : 0,
                                      q == b->sweeps - 1 && color == 1 ? 1 : 0);
  k_b_next<<<1, 256, 0, sb>>>(n, P, b->max_it, loop);
  const cudaError_t le = cudaGetLastError();
  cudaGraph_t body_out = nullptr;
  const cudaError_t be = cudaStreamEndCapture(sb, &body_out);
  SFX_CUDA(le);
  SFX_CUDA(be);
  SFX_CUDA(cudaStreamUpdateCaptureDependencies(s, &cnode, nullptr, 1,
                                               cudaStreamSetCaptureDependencies));
  k_b_totals<<<n * kTotBlocks, 256, 0, s>>>(b->dI, P);
  k_b_totals_final<<<n, 32, 0, s>>>(b->dI, n, P);
  SFX_LAUNCH_CHECK();
  return SFX_OK;
}

sfx_status ensure_graph(sfx_batch* b, const void* phi, const void* ur, const void* uz, void* f,
                        void* F, float tol) {
  const void* k[5] = {phi, ur, uz, f, F};
  const int sched[6] = {b->block, b->sweeps, b->max_it, ur != nullptr, b->reuse_phi ? 1 : 0,
                        b->fast};
  bool same = b->exec != nullptr && tol == b->key_tol;
  for (int i = 0; i < 5 && same; ++i) same = k[i] == b->key[i];
  for (int i = 0; i < 6 && same; ++i) same = sched[i] == b->key_sched[i];
  if (same) return SFX_OK;
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  b->P.phi = (const double*)phi;
  b->P.ur = (const float*)ur;
  b->P.uz = (const float*)uz;
  b->P.f = (float2*)f;
  b->P.F = (float2*)F;
  if (!b->cap) SFX_CUDA(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  SFX_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
  sfx_status st = enqueue_step(b, ur != nullptr, tol, b->cap);
  cudaError_t e = cudaStreamEndCapture(b->cap, &g);
  if (st != SFX_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  SFX_CUDA(e);
  e = cudaGraphInstantiate(&b->exec, g, 0);
  cudaGraphDestroy(g);
  SFX_CUDA(e);
  for (int i = 0; i < 5; ++i) b->key[i] = k[i];
  for (int i = 0; i < 6; ++i) b->key_sched[i] = sched[i];
  b->key_tol = tol;
  return SFX_OK;
}

// The over-relaxation of an instance's red updates, as the single-grid
// solve sets it for the same parameters (sor: SFX_TUNE_F32_SOR).
void set_omega(BInst& B, const sfx_batch_instance& q, int sor) {
  B.p.om_f = B.p.om_F = 1.0f;
  if (sor == 0) return;
  B.p.om_f = sor_omega(q.params.Df, q.dt, q.h, q.params.eps, 2);
  B.p.om_F = sor > 1000 ? (float)(sor * 1e-3) : sor_omega(q.params.DF, q.dt, q.h, q.params.eps, 2);
}

bool inst_ok(const sfx_batch_instance& q) {
  return q.nr >= 1 && q.nz >= 1 && q.h > 0.0 && q.dt > 0.0 && q.params.eps > 0.0 &&
         q.params.gamma_inf > 0.0 && q.params.ka >= 0.0 && q.params.kd >= 0.0 &&
         q.params.Df >= 0.0 && q.params.DF >= 0.0;
}

}  // namespace

extern "C" {

sfx_status sfx_batch_create(const sfx_batch_instance* inst, int n, sfx_batch** out) {
  return sfx_batch_create_geom(inst, n, SFX_AXISYM, out);
}

sfx_status sfx_batch_create_geom(const sfx_batch_instance* inst, int n, int geom,
                                 sfx_batch** out) {
  if (!out || !inst || n < 1) return SFX_ERR_ARG;
  if (geom != SFX_AXISYM && geom != SFX_PLANAR2D) return SFX_ERR_ARG;
  *out = nullptr;
  for (int i = 0; i < n; ++i)
    if (!inst_ok(inst[i])) return SFX_ERR_ARG;
  sfx_batch* b = new sfx_batch();
  b->n = n;
  b->geom = geom;
  b->hinst.assign(inst, inst + n);
  for (int i = 0; i < n; ++i) {
    const sfx_batch_instance& q = inst[i];
    BInst B{};
    Level L{geom, q.nr, q.nz, 1, q.h};
    B.p = Nw32{L, (float)(1.0 / q.h), (float)(q.params.Df / q.h), (float)(q.params.DF / q.h),
               (float)(1.0 / q.dt), (float)q.params.ka, (float)q.params.kd,
               (float)q.params.gamma_inf, (float)(1.0 / q.params.eps), (float)q.params.eta,
               q.params.literal_upwind};
    set_omega(B, q, 1);
    B.dt = (float)q.dt;
    B.bc_f = (float)q.params.bc_f;
    B.bc_F = (float)q.params.bc_F;
    B.Df = (float)q.params.Df;
    B.DF = (float)q.params.DF;
    B.coff = b->ncell;
    B.rfoff = b->nrf;
    B.zfoff = b->nzf;
    B.poff = b->npack;
    b->npack += 2 * (size_t)L.ny * ((L.nx + 1) / 2);
    b->coff.push_back(b->ncell);
    b->rfoff.push_back(b->nrf);
    b->zfoff.push_back(b->nzf);
    b->ncell += L.ncell();
    b->nrf += L.nface(0);
    b->nzf += L.nface(1);
    b->hI.push_back(B);
  }
  sfx_status st = SFX_OK;
  const size_t nc = b->ncell;
  // the FP32 kernels index cells and faces with 32-bit integers
  if (std::max(std::max(nc, b->npack), std::max(b->nrf, b->nzf)) >= ((size_t)1 << 31)) {
    delete b;
    return SFX_ERR_ARG;
  }
  BPtr& P = b->P;
  if (st == SFX_OK) st = balloc(b, &b->dI, (size_t)n);
  if (st == SFX_OK) st = balloc(b, &b->pre_cell, (size_t)n + 1);
  if (st == SFX_OK) st = balloc(b, &b->pre_rf, (size_t)n + 1);
  if (st == SFX_OK) st = balloc(b, &b->pre_zf, (size_t)n + 1);
  if (st == SFX_OK) st = balloc(b, &b->pre_pair, (size_t)n + 1);
  if (st == SFX_OK) st = balloc(b, &P.phi32, nc);
  if (st == SFX_OK) st = balloc(b, &P.fs, nc);
  if (st == SFX_OK) st = balloc(b, &P.Fs, nc);
  if (st == SFX_OK) st = balloc(b, &P.B2[0], b->nrf);
  if (st == SFX_OK) st = balloc(b, &P.B2[1], b->nzf);
  if (st == SFX_OK) st = balloc(b, &P.H2[0], b->nrf);
  if (st == SFX_OK) st = balloc(b, &P.H2[1], b->nzf);
  if (st == SFX_OK) st = balloc(b, &P.rc, b->npack);
  if (st == SFX_OK) st = balloc(b, &P.e2, b->npack);
  if (st == SFX_OK) st = balloc(b, &P.norms, 4 * (size_t)n);
  if (st == SFX_OK) st = balloc(b, &P.rkind, 2 * (size_t)n);
  if (st == SFX_OK) st = balloc(b, &P.active, (size_t)n);
  if (st == SFX_OK) st = balloc(b, &P.iters, (size_t)n);
  if (st == SFX_OK) st = balloc(b, &P.loop, (size_t)1);
  if (st == SFX_OK) st = balloc(b, &P.rres, 2 * (size_t)n);
  if (st == SFX_OK) st = balloc(b, &P.mass, 2 * (size_t)n);
  if (st == SFX_OK) st = balloc(b, &P.work, 2 * (size_t)n);
  // block partials: at most one block per 128 cells of each instance
  const size_t maxblk = nc / 128 + (size_t)n + 1;
  if (st == SFX_OK) st = balloc(b, &P.part, 4 * maxblk);
  if (st == SFX_OK) st = balloc(b, &P.tpart, 4 * (size_t)n * kTotBlocks);
  if (st == SFX_OK) {
    cudaError_t e = cudaMemset(P.work, 0, 2 * (size_t)n * sizeof(unsigned long long));
    if (e != cudaSuccess) st = cuda_fail(e);
  }
  if (st == SFX_OK) {
    cudaError_t e = cudaMemcpy(b->dI, b->hI.data(), n * sizeof(BInst), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) st = cuda_fail(e);
  }
  if (st == SFX_OK) st = build_prefix(b);
  if (st != SFX_OK) {
    sfx_batch_destroy(b);
    return st;
  }
  *out = b;
  return SFX_OK;
}

void sfx_batch_destroy(sfx_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->cap_body) cudaStreamDestroy(b->cap_body);
  for (void* p : b->allocs) cudaFree(p);
  delete b;
}

sfx_status sfx_batch_layout(const sfx_batch* b, size_t* n_cells, size_t* n_rfaces,
                            size_t* n_zfaces, size_t* cell_off, size_t* rface_off,
                            size_t* zface_off) {
  if (!b) return SFX_ERR_ARG;
  if (n_cells) *n_cells = b->ncell;
  if (n_rfaces) *n_rfaces = b->nrf;
  if (n_zfaces) *n_zfaces = b->nzf;
  for (int i = 0; i < b->n; ++i) {
    if (cell_off) cell_off[i] = b->coff[i];
    if (rface_off) rface_off[i] = b->rfoff[i];
    if (zface_off) zface_off[i] = b->zfoff[i];
  }
  return SFX_OK;
}

sfx_status sfx_batch_set_tuning(sfx_batch* b, int key, int value) {
  if (!b) return SFX_ERR_ARG;
  if (key == SFX_TUNE_F32_FAST_RESID && value >= 0 && value <= 16) {
    b->fast = value;
    return SFX_OK;
  }
  if (key == SFX_TUNE_F32_SOR && (value == 0 || value == 1 || (value > 1000 && value < 2000))) {
    b->sor = value;
    for (int i = 0; i < b->n; ++i) set_omega(b->hI[i], b->hinst[i], value);
    SFX_CUDA(cudaMemcpy(b->dI, b->hI.data(), b->n * sizeof(BInst), cudaMemcpyHostToDevice));
    return SFX_OK;
  }
  return SFX_ERR_ARG;
}

sfx_status sfx_batch_set_schedule(sfx_batch* b, int block, int sweeps, int max_iters) {
  if (!b || (block != 128 && block != 256 && block != 512) || sweeps < 1 || sweeps > 16 ||
      max_iters < 1 || max_iters > 200)
    return SFX_ERR_ARG;
  if (block != b->block) {
    b->block = block;
    sfx_status st = build_prefix(b);
    if (st != SFX_OK) return st;
  }
  b->sweeps = sweeps;
  b->max_it = max_iters;
  return SFX_OK;
}

sfx_status sfx_batch_step(sfx_batch* b, const void* phi, const void* ur, const void* uz, void* f,
                          void* F, double tol, void* stream) {
  if (!b || !phi || !f || !F || f == F || !(tol > 0.0)) return SFX_ERR_ARG;
  if ((ur == nullptr) != (uz == nullptr)) return SFX_ERR_ARG;
  sfx_status st = ensure_graph(b, phi, ur, uz, f, F, (float)tol);
  if (st != SFX_OK) return st;
  if (b->reuse_phi && b->drift_phi != phi) {
    // phi declared static: its folded copy and the drifts once, outside the graph
    cudaStream_t s = (cudaStream_t)stream;
    const int n = b->n, bs = b->block;
    k_b_fold<<<b->nb_cell, bs, 0, s>>>(b->dI, n, b->pre_cell, b->P);
    k_b_drift<<<b->nb_rf, bs, 0, s>>>(b->dI, n, b->pre_rf, 0, b->P);
    k_b_drift<<<b->nb_zf, bs, 0, s>>>(b->dI, n, b->pre_zf, 1, b->P);
    SFX_LAUNCH_CHECK();
    b->drift_phi = phi;
  }
  SFX_CUDA(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
  return SFX_OK;
}

sfx_status sfx_batch_reuse_phi(sfx_batch* b, int on) {
  if (!b) return SFX_ERR_ARG;
  b->reuse_phi = on != 0;
  b->drift_phi = nullptr;   // rebuild on the next step
  return SFX_OK;
}

sfx_status sfx_batch_stats(sfx_batch* b, int* iters, float* res_f, float* res_F, double* mass_f,
                           double* mass_F, int* converged, void* stream) {
  if (!b) return SFX_ERR_ARG;
  const int n = b->n;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<int> it(n), act(n);
  std::vector<float> rr(2 * n);
  std::vector<double> m(2 * n);
  SFX_CUDA(cudaMemcpyAsync(it.data(), b->P.iters, n * sizeof(int), cudaMemcpyDeviceToHost, s));
  SFX_CUDA(cudaMemcpyAsync(act.data(), b->P.active, n * sizeof(int), cudaMemcpyDeviceToHost, s));
  SFX_CUDA(cudaMemcpyAsync(rr.data(), b->P.rres, 2 * n * sizeof(float), cudaMemcpyDeviceToHost, s));
  SFX_CUDA(cudaMemcpyAsync(m.data(), b->P.mass, 2 * n * sizeof(double), cudaMemcpyDeviceToHost, s));
  SFX_CUDA(cudaStreamSynchronize(s));
  for (int i = 0; i < n; ++i) {
    if (iters) iters[i] = it[i];
    if (res_f) res_f[i] = rr[2 * i];
    if (res_F) res_F[i] = rr[2 * i + 1];
    if (mass_f) mass_f[i] = m[2 * i];
    if (mass_F) mass_F[i] = m[2 * i + 1];
    if (converged) converged[i] = act[i] ? 0 : 1;
  }
  return SFX_OK;
}

sfx_status sfx_batch_work(sfx_batch* b, long long* resid_passes, long long* sweep_groups,
                          int reset, void* stream) {
  if (!b) return SFX_ERR_ARG;
  const int n = b->n;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<unsigned long long> w(2 * (size_t)n);
  SFX_CUDA(cudaMemcpyAsync(w.data(), b->P.work, w.size() * sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, s));
  SFX_CUDA(cudaStreamSynchronize(s));
  for (int i = 0; i < n; ++i) {
    if (resid_passes) resid_passes[i] = (long long)w[2 * i];
    if (sweep_groups) sweep_groups[i] = (long long)w[2 * i + 1];
  }
  if (reset) SFX_CUDA(cudaMemsetAsync(b->P.work, 0, w.size() * sizeof(unsigned long long), s));
  return SFX_OK;
}

// Autotuner: candidate schedules (threads per block, i.e. the tile of
// packed cells one block updates, x sweeps per iteration) are run on scratch
// copies of the state; each gets the smallest iteration budget that
// converges every instance (read from a probe step with a generous budget),
// then the fastest candidate is kept.
namespace {

struct TuneBest {
  float ms = 1e30f;
  int block = 0, sweeps = 0, iters = 0;
};

// Probes and times every candidate; returns on the first error (the caller
// releases the scratch and events on every path).
sfx_status autotune_candidates(sfx_batch* b, const void* phi, const void* ur, const void* uz,
                               const void* f, const void* F, float2* fw, float2* Fw,
                               size_t bytes, double tol, cudaStream_t s, void* stream,
                               cudaEvent_t e0, cudaEvent_t e1, TuneBest* best) {
  const int blocks[3] = {128, 256, 512};
  const int sweeps[3] = {2, 3, 4};
  std::vector<int> it(b->n), conv(b->n);
  for (int bi = 0; bi < 3; ++bi)
    for (int si = 0; si < 3; ++si) {
      // probe: generous budget, read the iterations each instance needs
      sfx_status st = sfx_batch_set_schedule(b, blocks[bi], sweeps[si], 40);
      if (st != SFX_OK) return st;
      SFX_CUDA(cudaMemcpyAsync(fw, f, bytes, cudaMemcpyDeviceToDevice, s));
      SFX_CUDA(cudaMemcpyAsync(Fw, F, bytes, cudaMemcpyDeviceToDevice, s));
      if ((st = sfx_batch_step(b, phi, ur, uz, fw, Fw, tol, stream)) != SFX_OK) return st;
      if ((st = sfx_batch_stats(b, it.data(), nullptr, nullptr, nullptr, nullptr, conv.data(),
                                stream)) != SFX_OK)
        return st;
      int need = 1;
      bool all = true;
      for (int i = 0; i < b->n; ++i) {
        need = std::max(need, it[i]);
        all = all && conv[i];
      }
      if (!all) continue;
      if ((st = sfx_batch_set_schedule(b, blocks[bi], sweeps[si], need + 1)) != SFX_OK) return st;
      float ms_best = 1e30f;
      for (int rep = 0; rep < 3; ++rep) {
        SFX_CUDA(cudaMemcpyAsync(fw, f, bytes, cudaMemcpyDeviceToDevice, s));
        SFX_CUDA(cudaMemcpyAsync(Fw, F, bytes, cudaMemcpyDeviceToDevice, s));
        if ((st = ensure_graph(b, phi, ur, uz, fw, Fw, (float)tol)) != SFX_OK) return st;
        SFX_CUDA(cudaEventRecord(e0, s));
        SFX_CUDA(cudaGraphLaunch(b->exec, s));
        SFX_CUDA(cudaEventRecord(e1, s));
        SFX_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        SFX_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        ms_best = std::min(ms_best, ms);
      }
      if (ms_best < best->ms) *best = TuneBest{ms_best, blocks[bi], sweeps[si], need + 1};
    }
  return SFX_OK;
}

}  // namespace

sfx_status sfx_batch_autotune(sfx_batch* b, const void* phi, const void* ur, const void* uz,
                              const void* f, const void* F, double tol, void* stream,
                              int* chosen) {
  if (!b || !phi || !f || !F) return SFX_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = b->ncell * sizeof(float2);
  const int block0 = b->block, sweeps0 = b->sweeps, iters0 = b->max_it;
  float2 *fw = nullptr, *Fw = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  TuneBest best;
  sfx_status st = SFX_OK;
  cudaError_t ce = cudaMalloc(&fw, bytes);
  if (ce == cudaSuccess) ce = cudaMalloc(&Fw, bytes);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) st = cuda_fail(ce);
  else
    st = autotune_candidates(b, phi, ur, uz, f, F, fw, Fw, bytes, tol, s, stream, e0, e1, &best);
  if (st != SFX_OK) cudaStreamSynchronize(s);   // no copy into the scratch left in flight
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (b->exec) {   // its pointers are the scratch copies freed below
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  if (fw) cudaFree(fw);
  if (Fw) cudaFree(Fw);
  if (st != SFX_OK) {
    sfx_batch_set_schedule(b, block0, sweeps0, iters0);
    return st;
  }
  // the iteration loop ends on the device once every instance converged,
  // so the budget is only a cap: keep room for later steps that need more
  // iterations than the probed one
  // (200 when no candidate converged every instance within the probe's 40)
  const bool found = best.ms < 1e30f;
  const int bb = found ? best.block : block0, bsw = found ? best.sweeps : sweeps0;
  const int bit = found ? std::min(200, std::max(2 * best.iters, 16)) : 200;
  st = sfx_batch_set_schedule(b, bb, bsw, bit);
  if (chosen) {
    chosen[0] = bb;
    chosen[1] = bsw;
    chosen[2] = bit;
  }
  return st;
}

}  // extern "C"
