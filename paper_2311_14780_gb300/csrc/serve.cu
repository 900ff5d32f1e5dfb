// Multi-site serving: many reconstructions ("sites", e.g. wafer sites) with different frame
// sizes, position counts, wavelength counts and mode counts stay resident on one GPU; each
// tick runs one optimisation iteration of every active site as ONE graph launch.
//
// Each admitted site owns a plan (its scratch and remap tables), Adam moments, a device step
// counter and a loss word.  Two forms of the tick (ptycho_server_set_mode):
//
//  - shared launches (serve_multi.cuh): the tick graph runs, per frame size and per
//    round of position batches, each pass of the pipeline as one launch over the current batch
//    of every active site of that frame size (a device work table assigns each block to a
//    site), then one launch each for every site's loss reduction, step counter and Adam.  The
//    graph and its tables are built when the active set changes.
//  - one child graph per site (default): each site's own iteration graph (forward, loss,
//    adjoint, gradients, Adam through its plan's pipeline, with its batches in flight on
//    several streams) is captured at admission, and a tick launches a parent graph with one
//    child-graph node per active site and no edges between them.  Measured faster than the
//    shared launches on the 64-request serving stream (659 vs 517 K evals/s): the sites'
//    passes overlap instead of running one shared pass after another.
//
// Sites are admitted between ticks while the HBM budget allows and release their memory when
// done (continuous batching).  Nothing here waits on the device inside a kernel.
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "plan.h"
#include "serve_multi.cuh"

namespace ptycho {
extern template int launch_round_multi<64>(const RoundTab&, const int*, const int*, const RowAdjClass*, int,
                                             cudaStream_t);
extern template int launch_round_multi<128>(const RoundTab&, const int*, const int*, const RowAdjClass*, int,
                                             cudaStream_t);
extern template int launch_round_multi<256>(const RoundTab&, const int*, const int*, const RowAdjClass*, int,
                                             cudaStream_t);
extern template int launch_round_multi<512>(const RoundTab&, const int*, const int*, const RowAdjClass*, int,
                                             cudaStream_t);
extern template cudaError_t prepare_multi<64>();
extern template cudaError_t prepare_multi<128>();
extern template cudaError_t prepare_multi<256>();
extern template cudaError_t prepare_multi<512>();
}  // namespace ptycho

namespace ptycho {

// One block per site: fixed-order FP64 sum of its loss partials.
__global__ void __launch_bounds__(256) k_loss_reduce_multi(const SiteFinish* __restrict__ sf) {
  __shared__ double red[256];
  const SiteFinish& f = sf[blockIdx.x];
  double s = 0.0;
  for (long long i = threadIdx.x; i < f.nparts; i += 256) s += f.loss_part[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *f.loss = red[0];
}

// The fused row adjoint's probe-gradient splits of every site that has several, added in split
// order into its gradient (the single-site pipeline's k_sum_splits, per site).   grid (blocks, n)
__global__ void __launch_bounds__(256) k_sum_splits_multi(const SiteFinish* __restrict__ sf) {
  const SiteFinish& f = sf[blockIdx.y];
  if (f.nsplit <= 1) return;
  for (long long i = blockIdx.x * 256ll + threadIdx.x; i < f.nP; i += (long long)gridDim.x * 256) {
    float2 s = f.gPs[i];
    for (int k = 1; k < f.nsplit; ++k) s = cadd(s, f.gPs[(long long)k * f.nP + i]);
    f.gP[i] = s;
  }
}

// One thread per site: the step counter the bias correction of this tick's Adam reads.
__global__ void k_tick_multi(const SiteFinish* __restrict__ sf, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) *sf[k].t_dev += 1;
}

// Adam on every site's O and P: block row y = 2*site + (0: O, 1: P), blocks of a row stride
// over its parameters.   grid (blocks_per_array, 2 * n)
__global__ void __launch_bounds__(256) k_adam_multi(const SiteFinish* __restrict__ sf) {
  const SiteFinish& f = sf[blockIdx.y >> 1];
  const int q = blockIdx.y & 1;
  const float t = (float)(*f.t_dev);
  const float b1 = f.beta1, b2 = f.beta2;
  const float c1 = 1.0f / (1.0f - powf(b1, t));
  const float c2 = 1.0f / (1.0f - powf(b2, t));
  float* theta = f.theta[q];
  const float* grad = f.grad[q];
  float* m = f.m[q];
  float* v = f.v[q];
  const float lr = f.lr[q], eps = f.eps;
  for (long long i = blockIdx.x * 256ll + threadIdx.x; i < f.n[q]; i += (long long)gridDim.x * 256) {
    const float g = grad[i];
    const float mi = fmaf(b1, m[i], (1.f - b1) * g);
    const float vi = fmaf(b2, v[i], (1.f - b2) * g * g);
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  }
}

}  // namespace ptycho

namespace {

struct Site {
  ptycho_plan* plan = nullptr;
  ptycho_site_t data{};
  float* mom = nullptr;        // mO | vO | mP | vP
  int* t_dev = nullptr;
  double* loss_dev = nullptr;
  cudaGraph_t graph = nullptr; // per-site form only
  long long bytes = 0;         // counted against the budget (own + caller's resident arrays)
  int iters_done = 0;
  int nbatches = 1;
};

// Device tables and the rounds of the shared-launch tick of one active set.
struct TickTables {
  struct Round {
    int F = 0;
    ptycho::RoundTab rt{};
    int blocks[ptycho::kMpNum] = {};
    std::vector<ptycho::RowAdjClass> cls;       // the fused row adjoint's launches
    const int* tiles = nullptr;
  };
  void* mem = nullptr;
  std::vector<Round> rounds;
  ptycho::SiteFinish* finish = nullptr;
  int nsites = 0;
  int adam_blocks = 1;
  void release() {
    if (mem) cudaFree(mem);
    mem = nullptr;
    rounds.clear();
    finish = nullptr;
    nsites = 0;
  }
};

int threads_per_row(int F) {
  switch (F) {
    case 64: return ptycho::FftShape<64>::N1;
    case 128: return ptycho::FftShape<128>::N1;
    case 256: return ptycho::FftShape<256>::N1;
    default: return ptycho::FftShape<512>::N1;
  }
}

// Arguments and block counts of site s in round r (its position batch r); cls receives the
// shape and block count of its fused row adjoint (blocks 0 when the site's plan runs the
// per-mode row adjoint).
void fill_round(Site* s, int r, ptycho::SiteRound& w, int& tiles, int* counts, ptycho::RowAdjClass& cls) {
  using namespace ptycho;
  const ptycho_plan& p = *s->plan;
  const int F = p.F, LM = p.L * p.M, T = threads_per_row(F);
  KArgs a{};
  a.L = p.L; a.M = p.M; a.F = F; a.J = p.J;
  a.pos = p.d_pos;
  for (int l = 0; l < p.L; ++l) { a.obj_off[l] = p.obj_off[l]; a.obj_h[l] = p.obj_h[l]; a.obj_w[l] = p.obj_w[l]; }
  a.bidx = p.d_ident;
  a.nbatch = p.J;
  a.batch_off = r * p.B;
  a.nb = std::min(p.B, p.J - a.batch_off);
  a.sigma = s->data.sigma;
  a.tw = p.d_tw;
  a.C = p.C;
  a.chunk_base = 0;
  a.chunk_len = LM;
  a.MG = p.MG;
  a.G = p.G;
  a.status = p.d_status;
  a.patch = nullptr;
  tiles = 1;
  for (int l = 0; l < p.L; ++l) {                    // the batch's bounding box per wavelength
    int y0 = 1 << 30, x0 = 1 << 30, y1 = -1, x1 = -1;
    for (int q = a.batch_off; q < a.batch_off + a.nb; ++q) {
      const int y = p.pos_host[((size_t)l * p.J + q) * 2], x = p.pos_host[((size_t)l * p.J + q) * 2 + 1];
      y0 = std::min(y0, y); x0 = std::min(x0, x);
      y1 = std::max(y1, y + F); x1 = std::max(x1, x + F);
    }
    a.box[l][0] = y0; a.box[l][1] = x0; a.box[l][2] = y1; a.box[l][3] = x1;
    tiles = std::max(tiles, ((y1 - y0 + kTile - 1) / kTile) * ((x1 - x0 + kTile - 1) / kTile));
  }
  LossArgs la{};
  la.Ipart = p.d_Ipart;
  la.bg = s->data.bg;
  la.tap_base = p.d_tap_base;
  la.tap_w = p.d_tap_w;
  la.Imeas = s->data.I_meas;
  la.mask = s->data.mask;
  la.mask_per_frame = s->data.mask_per_frame ? 1 : 0;
  la.eps = p.eps;
  la.loss_kind = p.loss_kind;
  la.read_var = p.read_var;
  la.D = p.d_D;
  la.loss_part = p.d_loss_part;
  la.remap = p.remap;
  la.Gsum = p.G;
  la.tap_dz = p.d_tap_dz;
  AdjArgs aa{};
  aa.D = p.d_D;
  aa.rt_ptr = p.d_rt_ptr;
  aa.rt_idx = p.d_rt_idx;
  aa.rt_w = p.d_rt_w;
  aa.Gt = p.d_Gt;
  aa.remap = p.remap;
  w.a = a;
  w.la = la;
  w.aa = aa;
  w.O = reinterpret_cast<const float2*>(s->data.O);
  w.P = reinterpret_cast<const float2*>(s->data.P);
  w.S = p.d_S;
  w.Ipart = p.d_Ipart;
  w.gO = p.d_gO;
  w.gP = p.d_gP;
  // the row adjoint the site's plan chose (the same variant, rows per block and position splits)
  const bool fused = p.adj_l != 0;
  const int nsplit = fused ? std::max(1, p.nsplit_adj) : 1;
  w.gPs = nsplit > 1 ? p.d_gPs : p.d_gP;
  w.gp_stride = p.P_numel;
  w.nsplit = nsplit;
  w.rpb = p.rpb_adj;
  cls.M = p.M;
  cls.rpb = p.rpb_adj;
  cls.var = (F == 512 && p.adj_l_w) ? 2 : (p.adj_l_pl2 ? 1 : 0);
  cls.pass = -1;
  cls.blocks = fused ? (F / p.rpb_adj) * p.L * nsplit : 0;
  int rows = 0, cols = 0;                           // RowCfg<F>::RPB, ColCfg<F>::W
  switch (F) {
    case 64: rows = RowCfg<64>::RPB; cols = ColCfg<64>::W; break;
    case 128: rows = RowCfg<128>::RPB; cols = ColCfg<128>::W; break;
    case 256: rows = RowCfg<256>::RPB; cols = ColCfg<256>::W; break;
    default: rows = RowCfg<512>::RPB; cols = ColCfg<512>::W; break;
  }
  counts[kMpRowFwd] = (F / rows) * p.L * a.nb;
  counts[kMpColFwd] = (F / cols) * p.G * a.nb;
  counts[kMpLoss] = (F * F / (kLossThreads * kLossPx)) * a.nb;
  counts[kMpRemapAdj] = p.remap ? (F * F / 256) * ((a.nb + kRtPos - 1) / kRtPos) : 0;
  counts[kMpColAdj] = counts[kMpColFwd];
  counts[kMpRowAdj] = fused ? 0 : (F / (256 / (T * kAdjSlots))) * LM;
  counts[kMpObjGrad] = fused ? 0 : tiles * p.L;
  counts[kMpObjGradL] = fused ? tiles * p.L : 0;
}

long long align256(long long x) { return (x + 255) & ~255ll; }

// Builds the rounds and uploads the work tables of the active set (synchronous).
int build_tables(const std::vector<Site*>& sites, TickTables& tt) {
  using namespace ptycho;
  tt.release();
  struct HostRound { int F; size_t sr, start, tiles; int n; int blocks[kMpNum]; std::vector<RowAdjClass> cls; };
  std::vector<SiteRound> hsr;
  std::vector<int> hstart, htiles;
  std::vector<HostRound> hr;
  for (int F : {64, 128, 256, 512}) {
    int R = 0;
    for (Site* s : sites)
      if (s->plan->F == F) R = std::max(R, s->nbatches);
    for (int r = 0; r < R; ++r) {
      HostRound h{F, hsr.size(), hstart.size(), htiles.size(), 0, {}, {}};
      std::vector<std::vector<int>> cnt(kMpNum);
      std::vector<RowAdjClass> site_cls;
      for (Site* s : sites) {
        if (s->plan->F != F || s->nbatches <= r) continue;
        SiteRound w;
        int tiles = 1, c[kMpNum];
        RowAdjClass sc{};
        fill_round(s, r, w, tiles, c, sc);
        hsr.push_back(w);
        htiles.push_back(tiles);
        for (int q = 0; q < kMpNum; ++q) cnt[q].push_back(c[q]);
        site_cls.push_back(sc);
        ++h.n;
        if (sc.blocks) {                              // a new block shape opens a launch of its own
          bool known = false;
          for (const RowAdjClass& k : h.cls) known = known || (k.M == sc.M && k.rpb == sc.rpb && k.var == sc.var);
          if (!known) {
            sc.pass = kMpNum + (int)h.cls.size();
            sc.blocks = 0;
            h.cls.push_back(sc);
          }
        }
      }
      for (RowAdjClass& k : h.cls) {                  // the class passes' counts: 0 for other sites
        std::vector<int> c;
        for (const RowAdjClass& sc : site_cls)
          c.push_back(sc.blocks && sc.M == k.M && sc.rpb == k.rpb && sc.var == k.var ? sc.blocks : 0);
        cnt.push_back(c);
      }
      for (size_t q = 0; q < cnt.size(); ++q) {
        long long acc = 0;
        for (int k = 0; k < h.n; ++k) {
          hstart.push_back((int)acc);
          acc += cnt[q][k];
        }
        hstart.push_back((int)acc);
        if (acc >= (1ll << 31)) return PTYCHO_EUNSUPPORTED;
        if (q < (size_t)kMpNum) h.blocks[q] = (int)acc;
        else h.cls[q - kMpNum].blocks = (int)acc;
      }
      hr.push_back(h);
    }
  }
  std::vector<SiteFinish> hf;
  long long max_n = 1;
  for (Site* s : sites) {
    ptycho_plan& p = *s->plan;
    SiteFinish f{};
    const int nsplit = p.adj_l ? std::max(1, p.nsplit_adj) : 1;
    f.gPs = nsplit > 1 ? p.d_gPs : nullptr;
    f.gP = p.d_gP;
    f.nP = p.P_numel;
    f.nsplit = nsplit;
    f.loss_part = p.d_loss_part;
    f.nparts = (long long)p.J * (p.F * p.F / (kLossThreads * kLossPx));
    f.loss = s->loss_dev;
    f.t_dev = s->t_dev;
    const long long nO = 2 * p.O_numel, nP = 2 * p.P_numel;
    f.theta[0] = s->data.O;
    f.theta[1] = s->data.P;
    f.grad[0] = reinterpret_cast<const float*>(p.d_gO);
    f.grad[1] = reinterpret_cast<const float*>(p.d_gP);
    f.m[0] = s->mom;
    f.v[0] = s->mom + nO;
    f.m[1] = s->mom + 2 * nO;
    f.v[1] = s->mom + 2 * nO + nP;
    f.n[0] = nO;
    f.n[1] = nP;
    f.lr[0] = s->data.lr_O;
    f.lr[1] = s->data.lr_P;
    f.beta1 = s->data.beta1;
    f.beta2 = s->data.beta2;
    f.eps = s->data.eps;
    max_n = std::max(max_n, std::max(nO, nP));
    hf.push_back(f);
  }
  const long long b_sr = align256((long long)(hsr.size() * sizeof(SiteRound)));
  const long long b_st = align256((long long)(hstart.size() * sizeof(int)));
  const long long b_ti = align256((long long)(htiles.size() * sizeof(int)));
  const long long b_fi = align256((long long)(hf.size() * sizeof(SiteFinish)));
  if (cudaMalloc(&tt.mem, (size_t)(b_sr + b_st + b_ti + b_fi)) != cudaSuccess) {
    cudaGetLastError();
    tt.mem = nullptr;
    return PTYCHO_ENOMEM;
  }
  char* base = static_cast<char*>(tt.mem);
  SiteRound* d_sr = reinterpret_cast<SiteRound*>(base);
  int* d_st = reinterpret_cast<int*>(base + b_sr);
  int* d_ti = reinterpret_cast<int*>(base + b_sr + b_st);
  SiteFinish* d_fi = reinterpret_cast<SiteFinish*>(base + b_sr + b_st + b_ti);
  if ((!hsr.empty() && cudaMemcpy(d_sr, hsr.data(), hsr.size() * sizeof(SiteRound), cudaMemcpyHostToDevice)) ||
      (!hstart.empty() && cudaMemcpy(d_st, hstart.data(), hstart.size() * sizeof(int), cudaMemcpyHostToDevice)) ||
      (!htiles.empty() && cudaMemcpy(d_ti, htiles.data(), htiles.size() * sizeof(int), cudaMemcpyHostToDevice)) ||
      cudaMemcpy(d_fi, hf.data(), hf.size() * sizeof(SiteFinish), cudaMemcpyHostToDevice)) {
    tt.release();
    return PTYCHO_ECUDA;
  }
  for (const HostRound& h : hr) {
    TickTables::Round r;
    r.F = h.F;
    r.rt.sr = d_sr + h.sr;
    r.rt.start = d_st + h.start;
    r.rt.n = h.n;
    for (int q = 0; q < kMpNum; ++q) r.blocks[q] = h.blocks[q];
    r.cls = h.cls;
    r.tiles = d_ti + h.tiles;
    tt.rounds.push_back(r);
  }
  tt.finish = d_fi;
  tt.nsites = (int)sites.size();
  tt.adam_blocks = (int)std::min<long long>(256, (max_n + 256 * 8 - 1) / (256 * 8));
  return PTYCHO_OK;
}

int launch_round(const TickTables::Round& r, cudaStream_t st) {
  switch (r.F) {
    case 64: return ptycho::launch_round_multi<64>(r.rt, r.blocks, r.tiles, r.cls.data(), (int)r.cls.size(), st);
    case 128: return ptycho::launch_round_multi<128>(r.rt, r.blocks, r.tiles, r.cls.data(), (int)r.cls.size(), st);
    case 256: return ptycho::launch_round_multi<256>(r.rt, r.blocks, r.tiles, r.cls.data(), (int)r.cls.size(), st);
    default: return ptycho::launch_round_multi<512>(r.rt, r.blocks, r.tiles, r.cls.data(), (int)r.cls.size(), st);
  }
}

// The shared-launch tick of the active sites, captured on st.
int enqueue_shared_tick(const std::vector<Site*>& sites, const TickTables& tt, cudaStream_t st) {
  // ordinary launches: as programmatic dependent launches the shared passes measured 9 % slower on
  // the 64-request serving stream (472 vs 517 K evals/s, two runs each)
  ptycho::pdl_enabled() = false;
  bool splits = false;
  for (Site* s : sites) {
    ptycho_plan* p = s->plan;
    const int nsplit = p->adj_l ? std::max(1, p->nsplit_adj) : 1;
    if (cudaMemsetAsync(p->d_gO, 0, sizeof(float2) * (size_t)p->O_numel, st) != cudaSuccess ||
        cudaMemsetAsync(nsplit > 1 ? p->d_gPs : p->d_gP, 0, sizeof(float2) * (size_t)p->P_numel * nsplit, st) !=
            cudaSuccess)
      return PTYCHO_ECUDA;
    splits = splits || nsplit > 1;
  }
  for (const TickTables::Round& r : tt.rounds) {
    const int rc = launch_round(r, st);
    if (rc) return rc;
  }
  if (splits) ptycho::k_sum_splits_multi<<<dim3(tt.adam_blocks, tt.nsites), 256, 0, st>>>(tt.finish);
  ptycho::k_loss_reduce_multi<<<tt.nsites, 256, 0, st>>>(tt.finish);
  ptycho::k_tick_multi<<<(tt.nsites + 255) / 256, 256, 0, st>>>(tt.finish, tt.nsites);
  ptycho::k_adam_multi<<<dim3(tt.adam_blocks, 2 * tt.nsites), 256, 0, st>>>(tt.finish);
  return cudaGetLastError() == cudaSuccess ? PTYCHO_OK : PTYCHO_ECUDA;
}

int run_pipeline_dispatch(ptycho_plan* p, const ptycho::CallArgs& c, cudaStream_t st) {
  switch (p->F) {
    case 64: return ptycho::run_pipeline<64>(*p, c, st);
    case 128: return ptycho::run_pipeline<128>(*p, c, st);
    case 256: return ptycho::run_pipeline<256>(*p, c, st);
    case 512: return ptycho::run_pipeline<512>(*p, c, st);
  }
  return PTYCHO_EUNSUPPORTED;
}

int prepare_dispatch(int F) {
  int rc = PTYCHO_EUNSUPPORTED;
  cudaError_t e = cudaSuccess;
  switch (F) {
    case 64: rc = ptycho::prepare_kernels<64>(); e = ptycho::prepare_multi<64>(); break;
    case 128: rc = ptycho::prepare_kernels<128>(); e = ptycho::prepare_multi<128>(); break;
    case 256: rc = ptycho::prepare_kernels<256>(); e = ptycho::prepare_multi<256>(); break;
    case 512: rc = ptycho::prepare_kernels<512>(); e = ptycho::prepare_multi<512>(); break;
  }
  if (rc) return rc;
  return e == cudaSuccess ? PTYCHO_OK : PTYCHO_ECUDA;
}

// Launches one full iteration of a site on ``st`` (captured into its graph).
int enqueue_iteration(Site* s, cudaStream_t st) {
  ptycho_plan* p = s->plan;
  ptycho::CallArgs c{};
  c.kind = ptycho::CallKind::Adjoint;
  c.O = reinterpret_cast<const float2*>(s->data.O);
  c.P = reinterpret_cast<const float2*>(s->data.P);
  c.sigma = s->data.sigma;
  c.bg = s->data.bg;
  c.Imeas = s->data.I_meas;
  c.mask = s->data.mask;
  c.mask_per_frame = s->data.mask_per_frame ? 1 : 0;
  c.bidx = p->d_ident;
  c.nbatch = p->J;
  c.gO = p->d_gO;
  c.gP = p->d_gP;
  c.loss = s->loss_dev;
  int rc = run_pipeline_dispatch(p, c, st);
  if (rc) return rc;
  ptycho::k_tick<<<1, 32, 0, st>>>(s->t_dev);
  if (cudaGetLastError() != cudaSuccess) return PTYCHO_ECUDA;
  const long long nO = 2 * p->O_numel, nP = 2 * p->P_numel;
  float* mO = s->mom;
  float* vO = mO + nO;
  float* mP = vO + nO;
  float* vP = mP + nP;
  const int grid = 4 * p->sms;
  ptycho::k_adam_dev<<<grid, 256, 0, st>>>(s->data.O, reinterpret_cast<const float*>(p->d_gO), mO, vO, nO,
                                           s->data.lr_O, s->data.beta1, s->data.beta2, s->data.eps, s->t_dev);
  if (cudaGetLastError() != cudaSuccess) return PTYCHO_ECUDA;
  ptycho::k_adam_dev<<<grid, 256, 0, st>>>(s->data.P, reinterpret_cast<const float*>(p->d_gP), mP, vP, nP,
                                           s->data.lr_P, s->data.beta1, s->data.beta2, s->data.eps, s->t_dev);
  if (cudaGetLastError() != cudaSuccess) return PTYCHO_ECUDA;
  return PTYCHO_OK;
}

void free_site(Site* s) {
  if (!s) return;
  if (s->graph) cudaGraphDestroy(s->graph);
  if (s->mom) cudaFree(s->mom);
  if (s->t_dev) cudaFree(s->t_dev);
  if (s->loss_dev) cudaFree(s->loss_dev);
  if (s->plan) ptycho_plan_destroy(s->plan);
  delete s;
}

}  // namespace

struct ptycho_server {
  int dev = 0;
  int mode = PTYCHO_SERVE_SITE_GRAPHS;
  long long budget = 0, used = 0;
  std::vector<Site*> slots;
  TickTables tables;                          // shared-launch tables of the last active set
  cudaStream_t cap = nullptr;                 // capture stream
  cudaGraphExec_t exec = nullptr;             // parent graph of the last active set
  std::vector<int> exec_set;
  long long epoch = 0;                        // bumped by every admission and release: a slot
  long long exec_epoch = -1;                  // number can be reused by a different site
  long long last_launch_nodes = 0;
};

extern "C" {

int ptycho_server_create(int64_t hbm_budget_bytes, int32_t max_sites, ptycho_server_t** out) {
  if (!out || hbm_budget_bytes <= 0 || max_sites < 1) return PTYCHO_EINVAL;
  *out = nullptr;
  ptycho_server* sv = new (std::nothrow) ptycho_server();
  if (!sv) return PTYCHO_ENOMEM;
  if (cudaGetDevice(&sv->dev) != cudaSuccess ||
      cudaStreamCreateWithFlags(&sv->cap, cudaStreamNonBlocking) != cudaSuccess) {
    delete sv;
    return PTYCHO_ECUDA;
  }
  sv->budget = hbm_budget_bytes;
  sv->slots.assign((size_t)max_sites, nullptr);
  *out = sv;
  return PTYCHO_OK;
}

int ptycho_server_destroy(ptycho_server_t* sv) {
  if (!sv) return PTYCHO_OK;
  cudaDeviceSynchronize();
  for (Site* s : sv->slots) free_site(s);
  if (sv->exec) cudaGraphExecDestroy(sv->exec);
  sv->tables.release();
  if (sv->cap) cudaStreamDestroy(sv->cap);
  delete sv;
  return PTYCHO_OK;
}

int ptycho_server_admit(ptycho_server_t* sv, const ptycho_geom_t* geom, const ptycho_site_t* site, int32_t* slot_out) {
  if (!sv || !geom || !site || !slot_out || !site->O || !site->P || !site->I_meas || site->iterations < 1)
    return PTYCHO_EINVAL;
  if (!(site->beta1 >= 0.f && site->beta1 < 1.f && site->beta2 >= 0.f && site->beta2 < 1.f)) return PTYCHO_EINVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != sv->dev) return PTYCHO_EINVAL;
  int slot = -1;
  for (size_t i = 0; i < sv->slots.size(); ++i)
    if (!sv->slots[i]) { slot = (int)i; break; }
  if (slot < 0) return PTYCHO_EBUSY;
  Site* s = new (std::nothrow) Site();
  if (!s) return PTYCHO_ENOMEM;
  s->data = *site;
  const bool shared = sv->mode == PTYCHO_SERVE_SHARED_LAUNCHES;
  int rc = PTYCHO_OK;
  if (shared) {
    // the shared launches use one scratch set per site and the default pipeline variants
    ptycho_geom_t g = *geom;
    g.overlap = 1;
    g.flags = 0;
    g.col_groups = 0;
    g.zoom = nullptr;
    if (geom->zoom || geom->flags) { delete s; return PTYCHO_EUNSUPPORTED; }
    rc = ptycho::create_plan(&g, ptycho::kServeBatchTarget, &s->plan);
  } else {
    rc = ptycho::create_plan(geom, ptycho::kServeBatchTarget, &s->plan);
  }
  if (rc) { delete s; return rc; }
  ptycho_plan* p = s->plan;
  if (shared && (!p->store || p->nchunks != 1)) { free_site(s); return PTYCHO_EUNSUPPORTED; }
  s->nbatches = (p->J + p->B - 1) / p->B;
  const long long FF = (long long)p->F * p->F;
  const long long mom_floats = 4 * (p->O_numel + p->P_numel);     // 2 moments x 2 floats per complex
  s->bytes = p->bytes + mom_floats * 4 + 64 +
             8 * (p->O_numel + p->P_numel) + 4 * (long long)p->J * FF +      // caller's O, P, I_meas
             (site->mask ? (site->mask_per_frame ? (long long)p->J * FF : FF) : 0);
  if (sv->used + s->bytes > sv->budget) {
    free_site(s);
    return PTYCHO_EBUSY;
  }
  if (cudaMalloc((void**)&s->mom, sizeof(float) * (size_t)mom_floats) != cudaSuccess ||
      cudaMalloc((void**)&s->t_dev, sizeof(int)) != cudaSuccess ||
      cudaMalloc((void**)&s->loss_dev, sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    free_site(s);
    return PTYCHO_ENOMEM;
  }
  if (cudaMemsetAsync(s->mom, 0, sizeof(float) * (size_t)mom_floats, sv->cap) != cudaSuccess ||
      cudaMemsetAsync(s->t_dev, 0, sizeof(int), sv->cap) != cudaSuccess ||
      cudaMemsetAsync(s->loss_dev, 0, sizeof(double), sv->cap) != cudaSuccess ||
      cudaStreamSynchronize(sv->cap) != cudaSuccess) {
    free_site(s);
    return PTYCHO_ECUDA;
  }
  rc = prepare_dispatch(p->F);
  if (rc) { free_site(s); return rc; }
  if (shared) {                                 // the tick graph is built per active set
    sv->slots[(size_t)slot] = s;
    sv->used += s->bytes;
    sv->epoch += 1;
    *slot_out = slot;
    return PTYCHO_OK;
  }
  // capture one iteration
  if (cudaStreamBeginCapture(sv->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    free_site(s);
    return PTYCHO_ECUDA;
  }
  rc = enqueue_iteration(s, sv->cap);
  cudaGraph_t g = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(sv->cap, &g);
  if (rc || ec != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    free_site(s);
    return rc ? rc : PTYCHO_ECUDA;
  }
  s->graph = g;
  sv->slots[(size_t)slot] = s;
  sv->used += s->bytes;
  sv->epoch += 1;
  *slot_out = slot;
  return PTYCHO_OK;
}

int ptycho_server_tick(ptycho_server_t* sv, void* stream, int32_t* n_sites) {
  if (!sv) return PTYCHO_EINVAL;
  std::vector<int> active;
  for (size_t i = 0; i < sv->slots.size(); ++i) {
    Site* s = sv->slots[i];
    if (s && s->iters_done < s->data.iterations) active.push_back((int)i);
  }
  if (n_sites) *n_sites = (int32_t)active.size();
  if (active.empty()) return PTYCHO_OK;
  if (!sv->exec || sv->exec_epoch != sv->epoch || active != sv->exec_set) {
    if (sv->exec) {
      cudaGraphExecDestroy(sv->exec);
      sv->exec = nullptr;
    }
    cudaGraph_t parent = nullptr;
    if (sv->mode == PTYCHO_SERVE_SHARED_LAUNCHES) {
      std::vector<Site*> sites;
      for (int i : active) sites.push_back(sv->slots[(size_t)i]);
      // the previous tick may still read the old tables
      if (cudaDeviceSynchronize() != cudaSuccess) return PTYCHO_ECUDA;
      int rc = build_tables(sites, sv->tables);
      if (rc) return rc;
      if (cudaStreamBeginCapture(sv->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return PTYCHO_ECUDA;
      rc = enqueue_shared_tick(sites, sv->tables, sv->cap);
      const cudaError_t ec = cudaStreamEndCapture(sv->cap, &parent);
      if (rc || ec != cudaSuccess || !parent) {
        if (parent) cudaGraphDestroy(parent);
        cudaGetLastError();
        return rc ? rc : PTYCHO_ECUDA;
      }
    } else {
      if (cudaGraphCreate(&parent, 0) != cudaSuccess) return PTYCHO_ECUDA;
      for (int i : active) {
        cudaGraphNode_t node;
        if (cudaGraphAddChildGraphNode(&node, parent, nullptr, 0, sv->slots[(size_t)i]->graph) != cudaSuccess) {
          cudaGraphDestroy(parent);
          return PTYCHO_ECUDA;
        }
      }
    }
    const cudaError_t e = cudaGraphInstantiate(&sv->exec, parent, 0);
    cudaGraphDestroy(parent);
    if (e != cudaSuccess) {
      sv->exec = nullptr;
      cudaGetLastError();
      return PTYCHO_ECUDA;
    }
    sv->exec_set = active;
    sv->exec_epoch = sv->epoch;
  }
  if (cudaGraphLaunch(sv->exec, (cudaStream_t)stream) != cudaSuccess) return PTYCHO_ECUDA;
  for (int i : active) sv->slots[(size_t)i]->iters_done += 1;
  return PTYCHO_OK;
}

int ptycho_server_site_status(ptycho_server_t* sv, int32_t slot, int32_t* iters_done, double* loss) {
  if (!sv || slot < 0 || (size_t)slot >= sv->slots.size() || !sv->slots[(size_t)slot]) return PTYCHO_EINVAL;
  Site* s = sv->slots[(size_t)slot];
  if (iters_done) *iters_done = s->iters_done;
  if (loss && cudaMemcpy(loss, s->loss_dev, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
    return PTYCHO_ECUDA;
  return PTYCHO_OK;
}

int ptycho_server_release(ptycho_server_t* sv, int32_t slot) {
  if (!sv || slot < 0 || (size_t)slot >= sv->slots.size() || !sv->slots[(size_t)slot]) return PTYCHO_EINVAL;
  // the tick stream may still run this site's graph: finish the device work first
  if (cudaDeviceSynchronize() != cudaSuccess) return PTYCHO_ECUDA;
  Site* s = sv->slots[(size_t)slot];
  sv->used -= s->bytes;
  sv->slots[(size_t)slot] = nullptr;
  sv->epoch += 1;
  if (sv->exec) {                             // it may contain this site's graph
    cudaGraphExecDestroy(sv->exec);
    sv->exec = nullptr;
  }
  free_site(s);
  return PTYCHO_OK;
}

int64_t ptycho_server_used_bytes(const ptycho_server_t* sv) { return sv ? sv->used : 0; }

int ptycho_server_set_mode(ptycho_server_t* sv, int32_t mode) {
  if (!sv || (mode != PTYCHO_SERVE_SHARED_LAUNCHES && mode != PTYCHO_SERVE_SITE_GRAPHS)) return PTYCHO_EINVAL;
  for (Site* s : sv->slots)
    if (s) return PTYCHO_EINVAL;                // only while no site is admitted
  sv->mode = mode;
  return PTYCHO_OK;
}

}  // extern "C"
