// Multi-site serving: many reconstructions ("sites", e.g. wafer sites) with different frame
// sizes, position counts, wavelength counts and mode counts stay resident on one GPU; each
// tick runs one optimisation iteration of every active site as ONE graph launch.
//
// Each admitted site owns a plan (its L2-staged scratch and remap tables), Adam moments, a
// device step counter and a loss word, and a CUDA graph of one full iteration (forward,
// loss, adjoint, object/probe gradients, Adam) captured once at admission.  A tick
// instantiates (and caches, per active set) a parent graph with one child-graph node per
// active site and no edges between them, so the sites' kernels overlap on the device.
// Sites are admitted between ticks while the HBM budget allows and release their memory
// when done (continuous batching).  Nothing here waits on the device inside a kernel.
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "plan.h"


namespace {

struct Site {
  ptycho_plan* plan = nullptr;
  ptycho_site_t data{};
  float* mom = nullptr;        // mO | vO | mP | vP
  int* t_dev = nullptr;
  double* loss_dev = nullptr;
  cudaGraph_t graph = nullptr;
  long long bytes = 0;         // counted against the budget (own + caller's resident arrays)
  int iters_done = 0;
};

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
  switch (F) {
    case 64: return ptycho::prepare_kernels<64>();
    case 128: return ptycho::prepare_kernels<128>();
    case 256: return ptycho::prepare_kernels<256>();
    case 512: return ptycho::prepare_kernels<512>();
  }
  return PTYCHO_EUNSUPPORTED;
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
  long long budget = 0, used = 0;
  std::vector<Site*> slots;
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
  int rc = ptycho::create_plan(geom, ptycho::kServeBatchEvals, &s->plan);
  if (rc) { delete s; return rc; }
  ptycho_plan* p = s->plan;
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
    if (cudaGraphCreate(&parent, 0) != cudaSuccess) return PTYCHO_ECUDA;
    for (int i : active) {
      cudaGraphNode_t node;
      if (cudaGraphAddChildGraphNode(&node, parent, nullptr, 0, sv->slots[(size_t)i]->graph) != cudaSuccess) {
        cudaGraphDestroy(parent);
        return PTYCHO_ECUDA;
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

}  // extern "C"
