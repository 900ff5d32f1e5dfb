// Shared launches of the serving engine: one launch per pass and frame size runs the current
// position batch of every active site of that frame size (multi-site batching; the paper
// reconstructs one dataset at a time, so this layer has no counterpart there).
//
// A tick is a sequence of rounds.  In round r every active site with at least r+1 position
// batches contributes its batch r; each pass of the round (row DFT, column DFT + |Psi|^2, loss,
// R^T, adjoint columns, adjoint rows + probe gradient, object gradient) is ONE launch whose
// blocks are split among those sites by a work table: site k owns the launch's blocks
// [start[k], start[k+1]) and reads its own arguments (SiteRound: the kernel arguments of its
// batch and the buffers of its plan).  Each block copies its site's SiteRound into shared
// memory and runs the same device body as the single-site kernel, with its local block index.
// After the rounds, one launch reduces every site's loss, one advances every site's Adam step
// counter and one runs Adam on every site's objects and probes.
//
// Sites share no buffers, and each site's arithmetic (the batches, their order and every
// reduction) does not depend on the other sites, so a site's result is the same alone and in
// any mix.
#pragma once
#include "kernels.cuh"

namespace ptycho {

// One site's share of one round.
struct SiteRound {
  KArgs a;
  LossArgs la;
  AdjArgs aa;
  const float2* O;
  const float2* P;
  float2* S;                     // the site's scratch (one buffer set)
  float* Ipart;
  float2* gO;                    // the site's gradient buffers (zeroed at the start of the tick)
  float2* gP;
};

// Passes of a round; start[pass][k] is the first block of site k in that pass's launch.
enum MultiPass { kMpRowFwd = 0, kMpColFwd, kMpLoss, kMpRemapAdj, kMpColAdj, kMpRowAdj, kMpObjGrad, kMpNum };

struct RoundTab {
  const SiteRound* sr;           // [n]
  const int* start;              // [kMpNum][n + 1]
  int n;
};

// Largest k with start[k] <= blk (sites with no blocks in a pass have start[k] == start[k+1]).
__device__ __forceinline__ int owner_site(const int* start, int n, int blk) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(start + mid) <= blk) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Copies the block's site arguments into shared memory; returns the block index local to the site.
__device__ __forceinline__ int load_site(const RoundTab& rt, int pass, SiteRound& w) {
  const int* start = rt.start + pass * (rt.n + 1);
  const int blk = (int)blockIdx.x;
  const int k = owner_site(start, rt.n, blk);
  const int* src = reinterpret_cast<const int*>(rt.sr + k);
  int* dst = reinterpret_cast<int*>(&w);
  for (int i = threadIdx.x; i < (int)(sizeof(SiteRound) / sizeof(int)); i += blockDim.x) dst[i] = __ldg(src + i);
  __syncthreads();
  return blk - __ldg(start + k);
}

__device__ __forceinline__ uint3 unflatten(int loc, int gx, int gy) {
  return make_uint3(loc % gx, (loc / gx) % gy, loc / (gx * gy));
}

template <int F>
__global__ void __launch_bounds__(RowCfg<F>::threads) k_row_fwd_multi(RoundTab rt) {
  __shared__ SiteRound w;
  const int loc = load_site(rt, kMpRowFwd, w);
  const uint3 u = unflatten(loc, w.a.nb, F / RowCfg<F>::RPB);      // positions fastest (probe rows shared in L2)
  row_fwd_body<F>(w.O, w.P, w.S, w.a, make_uint3(u.y, u.z, u.x));
}

template <int F, bool STORE>
__global__ void __launch_bounds__(ColCfg<F>::threads) k_col_fwd_multi(RoundTab rt) {
  __shared__ SiteRound w;
  const int loc = load_site(rt, kMpColFwd, w);
  col_fwd_body<F, STORE>(w.S, w.Ipart, w.a, 1, unflatten(loc, F / ColCfg<F>::W, w.a.G));
}

template <int F>
__global__ void __launch_bounds__(kLossThreads) k_loss_multi(RoundTab rt) {
  __shared__ SiteRound w;
  const int loc = load_site(rt, kMpLoss, w);
  loss_body<F>(w.a, w.la, unflatten(loc, loss_blocks<F>(), w.a.nb));
}

template <int F>
__global__ void __launch_bounds__(256) k_remap_adj_multi(RoundTab rt) {
  __shared__ SiteRound w;
  const int loc = load_site(rt, kMpRemapAdj, w);
  remap_adj_body<F>(w.a, w.aa, unflatten(loc, F * F / 256, (w.a.nb + kRtPos - 1) / kRtPos));
}

template <int F, bool STORE>
__global__ void __launch_bounds__(ColCfg<F>::threads) k_col_adj_multi(RoundTab rt) {
  __shared__ SiteRound w;
  const int loc = load_site(rt, kMpColAdj, w);
  col_adj_body<F, STORE>(w.S, w.a, w.aa, unflatten(loc, F / ColCfg<F>::W, w.a.G));
}

template <int F>
__global__ void __launch_bounds__(RowAdjCfg<F>::threads, (F <= 256 ? 2 : 1)) k_row_adj_multi(RoundTab rt) {
  __shared__ SiteRound w;
  const int loc = load_site(rt, kMpRowAdj, w);
  row_adj_body<F, false>(w.O, w.P, w.S, w.gP, w.gO, w.a, unflatten(loc, F / RowAdjCfg<F>::RPB, w.a.chunk_len));
}

// grid: for site k, tiles(k) x L(k) blocks (the tiles of its batch's bounding box)
template <int F>
__global__ void __launch_bounds__(256) k_obj_grad_multi(RoundTab rt, const int* __restrict__ tiles) {
  __shared__ SiteRound w;
  const int* start = rt.start + kMpObjGrad * (rt.n + 1);
  const int loc = load_site(rt, kMpObjGrad, w);
  const int k = owner_site(start, rt.n, (int)blockIdx.x);
  obj_grad_body<F>(w.S, w.gO, w.a, unflatten(loc, __ldg(tiles + k), w.a.L));
}

// Per-site arguments of the finishing launches (loss reduction, step counter, Adam), defined
// in serve.cu.
struct SiteFinish {
  const double* loss_part;
  long long nparts;
  double* loss;
  int* t_dev;                    // Adam step counter
  float* theta[2];               // O, P (real views)
  const float* grad[2];
  float* m[2];
  float* v[2];
  long long n[2];
  float lr[2];
  float beta1, beta2, eps;
};

}  // namespace ptycho

namespace ptycho {

// Column passes keep Psi between the forward and the adjoint below 256^2 and recompute the
// column DFT from 256^2 up (the single-site pipeline's measured defaults).
template <int F> constexpr bool kMultiStore = F < 256;

// Dynamic shared memory limits of the shared-launch kernels of frame size F (once per device).
template <int F>
cudaError_t prepare_multi() {
  constexpr int col_adj_smem = ColCfg<F>::smem_xch + F * ColCfg<F>::W * (int)sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(k_row_fwd_multi<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, RowCfg<F>::smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_col_fwd_multi<F, kMultiStore<F>>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             ColCfg<F>::smem_xch);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_col_adj_multi<F, kMultiStore<F>>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             col_adj_smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_row_adj_multi<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, RowAdjCfg<F>::smem);
  return e;
}

// The seven passes of one round; blocks[pass] is the launch's total block count (a pass with
// no blocks, e.g. R^T when no site of the round has the remap, is not launched).
template <int F>
int launch_round_multi(const RoundTab& rt, const int* blocks, const int* d_tiles, cudaStream_t st) {
  constexpr bool STORE = kMultiStore<F>;
  constexpr int col_adj_smem = ColCfg<F>::smem_xch + F * ColCfg<F>::W * (int)sizeof(float);
  if (blocks[kMpRowFwd]) k_row_fwd_multi<F><<<blocks[kMpRowFwd], RowCfg<F>::threads, RowCfg<F>::smem, st>>>(rt);
  if (blocks[kMpColFwd])
    k_col_fwd_multi<F, STORE><<<blocks[kMpColFwd], ColCfg<F>::threads, ColCfg<F>::smem_xch, st>>>(rt);
  if (blocks[kMpLoss]) k_loss_multi<F><<<blocks[kMpLoss], kLossThreads, 0, st>>>(rt);
  if (blocks[kMpRemapAdj]) k_remap_adj_multi<F><<<blocks[kMpRemapAdj], 256, 0, st>>>(rt);
  if (blocks[kMpColAdj]) k_col_adj_multi<F, STORE><<<blocks[kMpColAdj], ColCfg<F>::threads, col_adj_smem, st>>>(rt);
  if (blocks[kMpRowAdj])
    k_row_adj_multi<F><<<blocks[kMpRowAdj], RowAdjCfg<F>::threads, RowAdjCfg<F>::smem, st>>>(rt);
  if (blocks[kMpObjGrad]) k_obj_grad_multi<F><<<blocks[kMpObjGrad], 256, 0, st>>>(rt, d_tiles);
  return cudaGetLastError() == cudaSuccess ? PTYCHO_OK : PTYCHO_ECUDA;
}

}  // namespace ptycho
