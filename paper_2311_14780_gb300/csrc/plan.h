// Host-side plan: geometry, validated positions, remap tables, batching decisions and the
// device workspace.  Shared by the C-ABI front end and the per-frame-size pipelines.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <vector>

#include "../../include/ptycho.h"
#include "kernels.cuh"
#include "shift.cuh"
#include "czt.cuh"

struct ptycho_plan {
  int dev = 0;
  int sms = 0;
  int L = 0, M = 0, F = 0, J = 0;
  int remap = 0, loss_kind = 0;
  float read_var = 0.f;                        // read-noise variance of the mixed loss
  // chirp-z propagator (geometry zoom != NULL): Bluestein tables on the device
  int czt = 0;
  float2* d_czt_chirp = nullptr;               // [L][F]
  float2* d_czt_hf = nullptr;                  // [L][2F]
  float2* d_czt_ha = nullptr;                  // [L][2F]
  float2* d_czt_tw2 = nullptr;                 // [2F]
  int flags = 0;                               // PTYCHO_FLAG_* variants
  float eps = 0.f;
  int obj_h[ptycho::kMaxL] = {}, obj_w[ptycho::kMaxL] = {};
  long long obj_off[ptycho::kMaxL] = {};
  long long O_numel = 0, P_numel = 0;          // complex elements
  std::vector<int32_t> pos_host;               // [L][J][2]

  // batching: B positions per batch, modes split into chunks of C, columns kernels use
  // G groups of MG modes; store = 1 keeps Psi in S between the forward and the adjoint.
  int store = 1, B = 1, C = 1, nchunks = 1, G = 1, MG = 1;
  // adjoint row pass over all modes of a wavelength per block (k_row_adj_l): rows per block,
  // position splits (each with its own probe-gradient buffer when nsplit > 1)
  int adj_l = 0, rpb_adj = 1, nsplit_adj = 1;
  int adj_l_ok = 0;                            // k_row_adj_l can run (all modes fit a block and the scratch)
  int adj_l_pl2 = 0;                           // its probe rows through L1/L2, two blocks per SM
  int adj_l_w = 0;                             // F = 512: one warp per row (k_row_adj_w)
  int fwd_l_w = 0;                             // F = 512: one warp per row (k_row_fwd_w)
  int col_tma2 = 0;                            // F = 512: staged columns, half exchange, two blocks per SM
  // forward row pass over all modes of a wavelength per block (k_row_fwd_l), same rows per block
  int fwd_l = 0, nsplit_fwd = 1;
  // staged column passes (k_col_fwd_s / k_col_adj_s): one block per W columns of a position
  // runs over all its modes, so the column passes leave a single intensity slice (G = 1)
  int col_staged = 0;
  // frame-resident passes (F <= 128, resident.cuh): the forward over G_res mode groups of MG_res
  // modes per position, the adjoint over nsplit_res position splits per probe mode
  int res = 0, G_res = 1, MG_res = 1, nsplit_res = 1;
  long long scratch_budget = 0;

  // nsets buffer sets let consecutive position batches overlap: batch k runs on stream
  // k % nsets (the caller's stream, then side[0..]) with buffer set k % nsets; events keep the
  // probe- and object-gradient accumulations in batch order
  static constexpr int kMaxSets = 4;
  int nsets = 1;
  cudaStream_t side[kMaxSets - 1] = {};
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_join[kMaxSets - 1] = {};
  cudaEvent_t ev_radj[kMaxSets] = {};
  cudaEvent_t ev_og[kMaxSets] = {};

  // device workspace (all owned by the plan)
  int32_t* d_pos = nullptr;
  int32_t* d_ident = nullptr;
  float2* d_tw = nullptr;
  int32_t* d_tap_base = nullptr;
  float2* d_tap_w = nullptr;
  int32_t* d_rt_ptr = nullptr;
  int32_t* d_rt_idx = nullptr;
  float* d_rt_w = nullptr;
  float2* d_S = nullptr;                       // [nsets][B][C][F][F]
  float* d_Ipart = nullptr;                    // [nsets][B][G][F][F]
  float* d_D = nullptr;                        // [nsets][B][F][F]
  float* d_Gt = nullptr;                       // [nsets][B][F][F] R^T D (remap only)
  double* d_loss_part = nullptr;
  double* d_sig_part = nullptr;                // [J][loss_blocks] sigma-gradient partials
  float* d_gbg_set = nullptr;                  // [nsets][F][F] background-gradient accumulators
  float* d_gsig = nullptr;                     // [J] sigma gradient (ptycho_step)
  float* d_gbg = nullptr;                      // [F][F] background gradient (ptycho_step)
  float2* d_gO = nullptr;
  float2* d_gP = nullptr;
  float2* d_gPs = nullptr;                     // [nsplit_adj][L][M][F][F] probe-gradient partials
  int* d_status = nullptr;                     // device status word, see ptycho_plan_status
  // fractional scan offsets (ptycho_plan_set_offsets): the caller's [L][J][2] array and the
  // per-set workspaces of the Fourier shift (allocated on first registration)
  float* d_delta = nullptr;
  // remap geometry (rebuilt by ptycho_plan_set_distance) and the z-gradient workspace
  double z = 0.0, det_pixel = 0.0, tilt_rad = 0.0;
  float2* d_tap_dz = nullptr;                  // [F*F] d(row, col tap index)/dz
  double* d_z_part = nullptr;                  // [J][loss_blocks] z-gradient partials
  long long rt_cap = 0;                        // capacity of d_rt_idx / d_rt_w
  float2* d_shT = nullptr;                     // [nsets][B][L][F][F] transform workspace
  float2* d_shQ = nullptr;                     // [nsets][B][L][F][F] ramp * spectrum of the windows
  float2* d_shP = nullptr;                     // [nsets][B][L][F][F] shifted patches
  double* d_dpart = nullptr;                   // [J][L][F/W][2] position-gradient partials
  float* d_gdelta = nullptr;                   // [L][J][2] position gradient (ptycho_step)
  double* d_reg_part = nullptr;                // [L][tiles] regulariser partials (allocated on first use)
  long long reg_cap = 0;                       // capacity of d_reg_part

  // TMA tensor maps of each scratch set, viewed as [B*C*F rows][F columns] of 8-byte elements
  // with a W x min(F, 256) box (column passes); has_tma = 0 falls back to plain loads
  int has_tma = 0;
  alignas(64) CUtensorMap tmap_S[4];
  long long bytes = 0;
  long long last_launches = 0;

  // opt-in per-kernel timing: an event pair around every launch, read back on request
  int prof = 0;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<int> ev_kind;                    // kind of the launch of each event pair

  // ptycho_step_host: the measured patterns are copied batch by batch on copy_st; the loss kernel
  // of position batch k waits for ev_copy[k] (set only for the duration of that call)
  cudaStream_t copy_st = nullptr;
  cudaEvent_t ev_copy_start = nullptr;
  std::vector<cudaEvent_t> ev_copy;
  const cudaEvent_t* imeas_ready = nullptr;
};

namespace ptycho {

enum class CallKind { Forward, Loss, Adjoint };

struct CallArgs {
  CallKind kind;
  const float2* O;
  const float2* P;
  const float* sigma;
  const float* bg;
  const float* Imeas;
  const uint8_t* mask;
  int mask_per_frame;
  const int32_t* bidx;     // device; never null here (the front end substitutes d_ident)
  int nbatch;
  float* I_pred;
  float2* gO;
  float2* gP;
  float* g_sigma;          // [J] or null
  float* g_bg;             // [F][F] or null
  float* g_delta;          // [L][J][2] or null (requires registered offsets)
  double* g_z;             // [1] dL/dz (device) or null (requires the remap)
  double* loss;
};

// Kernel kinds reported by ptycho_plan_profile_read (order matches PTYCHO_K_* in ptycho.h).
enum KernelKind { kRowFwd = 0, kColFwd, kLoss, kColAdj, kRowAdj, kObjGrad, kLossReduce, kAdam, kRemapAdj, kShift, kReg,
                  kResFwd, kResAdj, kNumKinds };

// Records the start event of a profiled launch (no-op unless profiling); returns the pair index.
long long prof_begin(ptycho_plan& p, int kind, cudaStream_t st);
void prof_end(ptycho_plan& p, long long idx, cudaStream_t st);

// How the default batching sizes a plan's position batches (ignored with an explicit scratch_bytes):
// about ``evals`` evaluations per batch, but at least ``min_positions`` positions, with one buffer
// set of at most ``max_set_bytes``.
struct BatchTarget {
  long long evals;
  long long min_positions;
  long long max_set_bytes;
};
// ptycho_plan_create with a batching target.
int create_plan(const ptycho_geom_t* g, const BatchTarget& target, ptycho_plan_t** out);
// Evaluations per position batch of a served site, in both tick forms.  Measured on the
// 64-request serving stream: per-site graphs 576 / 649 / 659 K evals/s with 128 / 600 / 1200;
// shared launches 468 / 500 / 519 / 524 K with 300 / 600 / 1200 / 2400.  1200 is also the
// single-site default, so a site's scratch is what its own plan would take.
constexpr long long kServeBatchEvals = 1200;
constexpr BatchTarget kServeBatchTarget{kServeBatchEvals, 1, 2ll << 30};

// Object regulariser (reg.cu): adds R to *loss (if not null) and dR to gO on stream st.
bool reg_args_ok(float mu_l1, float mu_tv, float eta);
int regularise(ptycho_plan& p, const float2* O, float mu_l1, float mu_tv, float eta, float2* gO, double* loss,
               cudaStream_t st);

// Defined once per frame size in kern_<F>.cu.
template <int F> int run_pipeline(ptycho_plan& p, const CallArgs& c, cudaStream_t st);
template <int F> int prepare_kernels();
// Plain (unfused) adjoint of one site, in plain.cuh; psi, Ibuf, Dbuf and Gbuf hold Bp positions.
template <int F> int plain_adjoint(ptycho_plan& p, const CallArgs& c, float2* psi, float* Ibuf, float* Dbuf,
                                   float* Gbuf, int Bp, cudaStream_t st);

}  // namespace ptycho
