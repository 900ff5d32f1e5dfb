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
// The adjoint row pass takes the variant the site's plan chose: per mode (one launch for all
// such sites, then the per-mode object gradient), or fused over the modes of a wavelength (one
// launch per class of block shape: mode count, rows per block and variant; then one launch of
// the mode-summed object gradient for all fused sites).  After the rounds, one launch adds the
// probe-gradient splits of every site that has them, one reduces every site's loss, one
// advances every site's Adam step counter and one runs Adam on every site's objects and probes.
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
  float2* gPs;                   // fused row adjoint: probe-gradient splits (gP itself with one split)
  long long gp_stride;           // elements between splits
  int nsplit;                    // position splits of the fused row adjoint
  int rpb;                       // its rows per block
};

// Passes of a round; start[pass][k] is the first block of site k in that pass's launch.  The
// fused row adjoint's classes follow as passes kMpNum + c.
enum MultiPass { kMpRowFwd = 0, kMpColFwd, kMpLoss, kMpRemapAdj, kMpColAdj, kMpRowAdj, kMpObjGrad, kMpObjGradL, kMpNum };

// One launch of the fused row adjoint: the sites of a round with this block shape.
// var: 0 probe rows in shared memory, 1 probe rows through L1/L2, 2 one warp per row (F = 512).
struct RowAdjClass {
  int M, rpb, var;
  int pass;                      // its start table: kMpNum + class index
  int blocks;
};

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
// (The work tables do not change during a tick, so this may run before the kernel waits for its
// predecessor when the passes are launched as programmatic dependent launches.)
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
  pdl_wait();
  pdl_trigger();
  const uint3 u = unflatten(loc, w.a.nb, F / RowCfg<F>::RPB);      // positions fastest (probe rows shared in L2)
  row_fwd_body<F>(w.O, w.P, w.S, w.a, make_uint3(u.y, u.z, u.x));
}

template <int F, bool STORE>
__global__ void __launch_bounds__(ColCfg<F>::threads) k_col_fwd_multi(RoundTab rt) {
  __shared__ SiteRound w;
  const int loc = load_site(rt, kMpColFwd, w);
  pdl_wait();
  pdl_trigger();
  col_fwd_body<F, STORE>(w.S, w.Ipart, w.a, 1, unflatten(loc, F / ColCfg<F>::W, w.a.G));
}

template <int F>
__global__ void __launch_bounds__(kLossThreads) k_loss_multi(RoundTab rt) {
  __shared__ SiteRound w;
  const int loc = load_site(rt, kMpLoss, w);
  pdl_wait();
  pdl_trigger();
  loss_body<F>(w.a, w.la, unflatten(loc, loss_blocks<F>(), w.a.nb));
}

template <int F>
__global__ void __launch_bounds__(256) k_remap_adj_multi(RoundTab rt) {
  __shared__ SiteRound w;
  const int loc = load_site(rt, kMpRemapAdj, w);
  pdl_wait();
  pdl_trigger();
  remap_adj_body<F>(w.a, w.aa, unflatten(loc, F * F / 256, (w.a.nb + kRtPos - 1) / kRtPos));
}

template <int F, bool STORE>
__global__ void __launch_bounds__(ColCfg<F>::threads) k_col_adj_multi(RoundTab rt) {
  __shared__ SiteRound w;
  const int loc = load_site(rt, kMpColAdj, w);
  pdl_wait();
  pdl_trigger();
  col_adj_body<F, STORE>(w.S, w.a, w.aa, unflatten(loc, F / ColCfg<F>::W, w.a.G));
}

template <int F>
__global__ void __launch_bounds__(RowAdjCfg<F>::threads, (F <= 256 ? 2 : 1)) k_row_adj_multi(RoundTab rt) {
  __shared__ SiteRound w;
  const int loc = load_site(rt, kMpRowAdj, w);
  pdl_wait();
  pdl_trigger();
  row_adj_body<F, false>(w.O, w.P, w.S, w.gP, w.gO, w.a, unflatten(loc, F / RowAdjCfg<F>::RPB, w.a.chunk_len));
}

// Fused row adjoint of one class: for site k, (F/rpb) x L x nsplit blocks.
template <int F, int VAR>
__global__ void __launch_bounds__(VAR == 2 ? kRowAdjWThreads : (VAR == 1 ? kRowAdjL2Threads : 256),
                                  (F <= 256 || VAR >= 1 ? 2 : 1))
k_row_adj_l_multi(RoundTab rt, int pass) {
  __shared__ SiteRound w;
  const int loc = load_site(rt, pass, w);
  pdl_wait();
  pdl_trigger();
  const uint3 bid = unflatten(loc, F / w.rpb, w.a.L);
  if constexpr (VAR == 2)
    row_adj_w_body<F>(w.O, w.P, w.S, w.gPs, w.gp_stride, w.a, w.rpb, w.nsplit, bid);
  else
    row_adj_l_body<F, VAR == 1>(w.O, w.P, w.S, w.gPs, w.gp_stride, w.a, w.rpb, w.nsplit, bid);
}

// Mode-summed object gradient of the fused sites: for site k, tiles(k) x L(k) blocks.
template <int F>
__global__ void __launch_bounds__(256) k_obj_grad_l_multi(RoundTab rt, const int* __restrict__ tiles) {
  __shared__ SiteRound w;
  const int* start = rt.start + kMpObjGradL * (rt.n + 1);
  const int loc = load_site(rt, kMpObjGradL, w);
  pdl_wait();
  pdl_trigger();
  const int k = owner_site(start, rt.n, (int)blockIdx.x);
  obj_grad_l_body<F>(w.S, w.gO, w.a, unflatten(loc, __ldg(tiles + k), w.a.L));
}

// grid: for site k, tiles(k) x L(k) blocks (the tiles of its batch's bounding box)
template <int F>
__global__ void __launch_bounds__(256) k_obj_grad_multi(RoundTab rt, const int* __restrict__ tiles) {
  __shared__ SiteRound w;
  const int* start = rt.start + kMpObjGrad * (rt.n + 1);
  const int loc = load_site(rt, kMpObjGrad, w);
  pdl_wait();
  pdl_trigger();
  const int k = owner_site(start, rt.n, (int)blockIdx.x);
  obj_grad_body<F>(w.S, w.gO, w.a, unflatten(loc, __ldg(tiles + k), w.a.L));
}

// Per-site arguments of the finishing launches (loss reduction, step counter, Adam), defined
// in serve.cu.
struct SiteFinish {
  const float2* gPs;             // probe-gradient splits (nsplit > 1) added into gP in split order
  float2* gP;
  long long nP;
  int nsplit;
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
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_row_adj_l_multi<F, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, kRowAdjLSmemMax);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_row_adj_l_multi<F, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kRowAdjLSmemMax);
  if constexpr (F == 512) {
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_row_adj_l_multi<F, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kRowAdjLSmemMax);
  }
  return e;
}

// Threads and dynamic shared memory of a fused row-adjoint class.
template <int F>
void row_adj_class_shape(const RowAdjClass& c, int& threads, int& smem) {
  if (c.var == 2) {
    threads = 32 * c.M * c.rpb;
    smem = row_adj_w_smem(c.M, c.rpb);
  } else {
    threads = FftShape<F>::N1 * c.M * c.rpb;
    smem = row_adj_l_smem<F>(c.M, c.rpb, c.var == 1);
  }
}

// The passes of one round; blocks[pass] is the launch's total block count (a pass with no
// blocks, e.g. R^T when no site of the round has the remap, is not launched); cls[0..ncls) are
// the fused row adjoint's launches.
template <int F>
int launch_round_multi(const RoundTab& rt, const int* blocks, const int* d_tiles, const RowAdjClass* cls, int ncls,
                       cudaStream_t st) {
  constexpr bool STORE = kMultiStore<F>;
  constexpr int col_adj_smem = ColCfg<F>::smem_xch + F * ColCfg<F>::W * (int)sizeof(float);
  if (blocks[kMpRowFwd] && launch_pdl(k_row_fwd_multi<F>, blocks[kMpRowFwd], RowCfg<F>::threads, RowCfg<F>::smem, st, rt))
    return PTYCHO_ECUDA;
  if (blocks[kMpColFwd] &&
      launch_pdl(k_col_fwd_multi<F, STORE>, blocks[kMpColFwd], ColCfg<F>::threads, ColCfg<F>::smem_xch, st, rt))
    return PTYCHO_ECUDA;
  if (blocks[kMpLoss] && launch_pdl(k_loss_multi<F>, blocks[kMpLoss], kLossThreads, 0, st, rt)) return PTYCHO_ECUDA;
  if (blocks[kMpRemapAdj] && launch_pdl(k_remap_adj_multi<F>, blocks[kMpRemapAdj], 256, 0, st, rt)) return PTYCHO_ECUDA;
  if (blocks[kMpColAdj] &&
      launch_pdl(k_col_adj_multi<F, STORE>, blocks[kMpColAdj], ColCfg<F>::threads, col_adj_smem, st, rt))
    return PTYCHO_ECUDA;
  if (blocks[kMpRowAdj] &&
      launch_pdl(k_row_adj_multi<F>, blocks[kMpRowAdj], RowAdjCfg<F>::threads, RowAdjCfg<F>::smem, st, rt))
    return PTYCHO_ECUDA;
  for (int i = 0; i < ncls; ++i) {
    const RowAdjClass& c = cls[i];
    if (!c.blocks) continue;
    int threads = 0, smem = 0;
    row_adj_class_shape<F>(c, threads, smem);
    cudaError_t e = cudaSuccess;
    if (c.var == 2) {
      if constexpr (F == 512) e = launch_pdl(k_row_adj_l_multi<F, 2>, c.blocks, threads, smem, st, rt, c.pass);
      else return PTYCHO_EUNSUPPORTED;
    } else if (c.var == 1) {
      e = launch_pdl(k_row_adj_l_multi<F, 1>, c.blocks, threads, smem, st, rt, c.pass);
    } else {
      e = launch_pdl(k_row_adj_l_multi<F, 0>, c.blocks, threads, smem, st, rt, c.pass);
    }
    if (e != cudaSuccess) return PTYCHO_ECUDA;
  }
  if (blocks[kMpObjGrad] && launch_pdl(k_obj_grad_multi<F>, blocks[kMpObjGrad], 256, 0, st, rt, d_tiles))
    return PTYCHO_ECUDA;
  if (blocks[kMpObjGradL] && launch_pdl(k_obj_grad_l_multi<F>, blocks[kMpObjGradL], 256, 0, st, rt, d_tiles))
    return PTYCHO_ECUDA;
  return cudaGetLastError() == cudaSuccess ? PTYCHO_OK : PTYCHO_ECUDA;
}

}  // namespace ptycho
