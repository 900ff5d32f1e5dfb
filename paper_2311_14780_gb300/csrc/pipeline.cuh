// Orchestration of one compute call for a fixed frame size F: loops over position batches
// and mode chunks and launches the kernels of kernels.cuh on the caller's stream.
#pragma once
#include <mutex>

#include "plan.h"
#include "resident.cuh"
#include "serve_multi.cuh"

namespace ptycho {

// Launch a kernel of the given kind on stream st, count it, bracket it with profiling
// events when enabled, and turn a launch failure into PTYCHO_ECUDA.
#define PTY_LAUNCH(p, kind, st, ...)                                 \
  do {                                                               \
    const long long pty_ev = prof_begin((p), (kind), (st));          \
    __VA_ARGS__;                                                     \
    ++(p).last_launches;                                             \
    if (cudaGetLastError() != cudaSuccess) return PTYCHO_ECUDA;      \
    prof_end((p), pty_ev, (st));                                     \
  } while (0)

template <int F, int WN>
cudaError_t set_cols_smem() {
  cudaError_t e = cudaFuncSetAttribute(k_col_fwd_s<F, true, WN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       ColSCfg<F, WN>::smem_fwd);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_col_fwd_s<F, false, WN>, cudaFuncAttributeMaxDynamicSharedMemorySize, ColSCfg<F, WN>::smem_fwd);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_col_adj_s<F, true, WN>, cudaFuncAttributeMaxDynamicSharedMemorySize, ColSCfg<F, WN>::smem_adj);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_col_adj_s<F, false, WN>, cudaFuncAttributeMaxDynamicSharedMemorySize, ColSCfg<F, WN>::smem_adj);
  return e;
}

// Staged column passes with WN columns per block (0 = the frame size's default).
template <int F, int WN>
int launch_cols_s(ptycho_plan& p, bool fwd, bool store, cudaStream_t cs, float2* S, float* Ip, const KArgs& a,
                  const AdjArgs& aa) {
  using Cfg = ColSCfg<F, WN>;
  const dim3 grid(F / Cfg::W, a.nb), blk(Cfg::threads);
  if (fwd && store)
    PTY_LAUNCH(p, kColFwd, cs, launch_pdl(k_col_fwd_s<F, true, WN>, grid, blk, Cfg::smem_fwd, cs, S, Ip, a));
  else if (fwd)
    PTY_LAUNCH(p, kColFwd, cs, launch_pdl(k_col_fwd_s<F, false, WN>, grid, blk, Cfg::smem_fwd, cs, S, Ip, a));
  else if (store)
    PTY_LAUNCH(p, kColAdj, cs, launch_pdl(k_col_adj_s<F, true, WN>, grid, blk, Cfg::smem_adj, cs, S, a, aa));
  else
    PTY_LAUNCH(p, kColAdj, cs, launch_pdl(k_col_adj_s<F, false, WN>, grid, blk, Cfg::smem_adj, cs, S, a, aa));
  return PTYCHO_OK;
}

// Raises the dynamic shared-memory limit of every kernel of frame size F on the current device
// (cudaFuncSetAttribute acts per device), once per device; thread-safe.
template <int F>
int prepare_kernels() {
  constexpr int kMaxDevices = 64;
  static std::mutex mu;
  static bool done[kMaxDevices] = {};
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return PTYCHO_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return PTYCHO_EINVAL;
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return PTYCHO_OK;
  const int col_adj_smem = ColCfg<F>::smem_xch + F * ColCfg<F>::W * (int)sizeof(float);
  cudaError_t e = cudaSuccess;
  e = cudaFuncSetAttribute(k_row_fwd<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, RowCfg<F>::smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_row_adj<F, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, RowAdjCfg<F>::smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_row_adj<F, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, RowAdjCfg<F>::smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_col_fwd<F, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, ColCfg<F>::smem_xch);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_col_fwd<F, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, ColCfg<F>::smem_xch);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_col_adj<F, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, col_adj_smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_col_adj<F, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, col_adj_smem);
  if constexpr (F >= 512) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_col_fwd_2b<F, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, ColCfg<F>::smem_xch);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_col_fwd_2b<F, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, ColCfg<F>::smem_xch);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_col_adj_2b<F, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, col_adj_smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_col_adj_2b<F, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, col_adj_smem);
  }
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_col_fwd_tma<F, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, ColTma<F>::smem_fwd);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_col_fwd_tma<F, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, ColTma<F>::smem_fwd);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_col_adj_tma<F, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, ColTma<F>::smem_adj);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_col_adj_tma<F, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, ColTma<F>::smem_adj);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_row_adj_l<F, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kRowAdjLSmemMax);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_row_adj_l<F, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kRowAdjLSmemMax);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_row_fwd_l<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, kRowAdjLSmemMax);
  if constexpr (F == 512) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_row_adj_w<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, kRowAdjLSmemMax);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_row_fwd_w<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, kRowAdjLSmemMax);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_col_fwd_tma2<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, ColTma2<F>::smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_col_adj_tma2<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, ColTma2<F>::smem);
  }
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_shift_rows<F, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, RowCfg<F>::smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_shift_rows<F, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, RowCfg<F>::smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_shift_rows<F, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, RowCfg<F>::smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_shift_cols<F, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, ColCfg<F>::smem_xch);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_shift_cols<F, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, ColCfg<F>::smem_xch);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_czt_row_fwd<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, CztRowCfg<F>::smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_czt_col_fwd<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, CztColCfg<F>::smem_fwd);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_czt_col_adj<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, CztColCfg<F>::smem_adj);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_czt_row_adj<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, CztRowAdjCfg<F>::smem);
  if (e == cudaSuccess) e = set_cols_smem<F, 0>();
  if (e == cudaSuccess) e = set_cols_smem<F, 4>();
  if constexpr (ResSupported<F>::value) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_res_fwd<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, ResCfg<F>::smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_res_adj<F>, cudaFuncAttributeMaxDynamicSharedMemorySize, ResCfg<F>::smem);
  }
  if (e != cudaSuccess) return PTYCHO_ECUDA;
  done[dev] = true;
  return PTYCHO_OK;
}

template <int F>
int run_pipeline(ptycho_plan& p, const CallArgs& c, cudaStream_t st) {
  int rc = prepare_kernels<F>();
  if (rc) return rc;
  pdl_enabled() = !(p.flags & PTYCHO_FLAG_NO_PDL);
  constexpr int FF = F * F;
  const bool grad = c.kind == CallKind::Adjoint;
  const bool need_loss = c.kind != CallKind::Forward;
  // keep Psi between the passes only when an adjoint follows and the variant asks for it;
  // otherwise the adjoint recomputes the column DFT from the kept row-pass output
  const bool store = grad && p.store && !(p.flags & PTYCHO_FLAG_RECOMPUTE_COLUMNS);
  const bool rerun_rows = !p.store;     // modes in chunks: the row pass is rerun as well
  const bool obj_atomic = (p.flags & PTYCHO_FLAG_OBJ_GRAD_ATOMIC) != 0;
  // all modes of a wavelength per adjoint row block; with several position splits the probe
  // gradient is summed per split and the splits are added in order at the end
  // fractional scan offsets: the Fourier-shift passes, the fused row adjoint (it forms the
  // mode-summed object-gradient patch that the adjoint shift transforms)
  const bool shifted = p.d_delta != nullptr;
  if (shifted && (p.nchunks != 1 || !p.adj_l_ok)) return PTYCHO_EUNSUPPORTED;
  const bool adj_l = (p.adj_l && !obj_atomic && p.nchunks == 1) || shifted;
  const bool col_staged = p.col_staged && p.nchunks == 1;
  const bool fwd_l = p.fwd_l && p.nchunks == 1 && !shifted;
  const bool narrow = (p.flags & PTYCHO_FLAG_NARROW_COLUMNS) != 0;
  // frame-resident passes (F <= 128, PTYCHO_FLAG_RESIDENT_FRAMES): fields stay in one block's
  // shared memory
  const bool res = ResSupported<F>::value && p.res && !shifted && !p.czt && p.nchunks == 1 && !obj_atomic;
  const int nsplit = res ? p.nsplit_res : adj_l ? p.nsplit_adj : 1;
  float2* gPs = nsplit > 1 ? p.d_gPs : c.gP;

  KArgs a{};
  a.L = p.L; a.M = p.M; a.F = F; a.J = p.J;
  a.pos = p.d_pos;
  for (int l = 0; l < p.L; ++l) { a.obj_off[l] = p.obj_off[l]; a.obj_h[l] = p.obj_h[l]; a.obj_w[l] = p.obj_w[l]; }
  a.bidx = c.bidx;
  a.nbatch = c.nbatch;
  a.sigma = c.sigma;
  a.tw = p.d_tw;
  a.C = p.C;
  a.MG = res ? p.MG_res : p.MG;
  a.G = res ? p.G_res : p.G;
  a.status = p.d_status;

  LossArgs la{};
  la.Ipart = p.d_Ipart;
  la.bg = c.bg;
  la.tap_base = p.d_tap_base;
  la.tap_w = p.d_tap_w;
  la.Imeas = c.Imeas;
  la.mask = c.mask;
  la.mask_per_frame = c.mask_per_frame;
  la.eps = p.eps;
  la.loss_kind = p.loss_kind;
  la.read_var = p.read_var;
  la.D = grad ? p.d_D : nullptr;
  la.loss_part = need_loss ? p.d_loss_part : nullptr;
  la.sig_part = grad && c.g_sigma ? p.d_sig_part : nullptr;
  la.I_pred = c.kind == CallKind::Forward ? c.I_pred : nullptr;
  la.remap = p.remap;
  la.Gsum = a.G;
  la.tap_dz = p.d_tap_dz;
  la.z_part = grad && c.g_z ? p.d_z_part : nullptr;

  CztArgs ct{p.d_czt_chirp, p.d_czt_hf, p.d_czt_ha, p.d_czt_tw2};
  if (p.czt && (p.nchunks != 1 || p.d_delta)) return PTYCHO_EUNSUPPORTED;
  AdjArgs aa{};
  aa.D = p.d_D;
  aa.rt_ptr = p.d_rt_ptr;
  aa.rt_idx = p.d_rt_idx;
  aa.rt_w = p.d_rt_w;
  aa.Gt = p.d_Gt;
  aa.remap = p.remap;
  // batches in identity order have host-known positions (plan-owned table)
  const bool identity = c.bidx == p.d_ident && p.pos_host.size() >= (size_t)p.L * p.J * 2;

  p.last_launches = 0;
  if (grad) {
    if (cudaMemsetAsync(c.gO, 0, sizeof(float2) * p.O_numel, st) != cudaSuccess) return PTYCHO_ECUDA;
    if (cudaMemsetAsync(gPs, 0, sizeof(float2) * p.P_numel * nsplit, st) != cudaSuccess) return PTYCHO_ECUDA;
    if (c.g_bg && cudaMemsetAsync(p.d_gbg_set, 0, sizeof(float) * p.nsets * FF, st) != cudaSuccess)
      return PTYCHO_ECUDA;
  }
  const int LM = p.L * p.M;
  const dim3 row_blk(RowCfg<F>::threads), col_blk(ColCfg<F>::threads);
  const int col_adj_smem = ColCfg<F>::smem_xch + F * ColCfg<F>::W * (int)sizeof(float);
  const int nbatches = (c.nbatch + p.B - 1) / p.B;
  const int nsets = p.nsets < nbatches ? p.nsets : nbatches;
  const long long set_S = (long long)p.B * p.C * FF, set_I = (long long)p.B * a.G * FF, set_F = (long long)p.B * FF;
  cudaStream_t streams[ptycho_plan::kMaxSets] = {st};
  for (int i = 1; i < nsets; ++i) streams[i] = p.side[i - 1];
  if (nsets > 1) {                                    // the side streams follow the caller's work so far
    if (cudaEventRecord(p.ev_fork, st) != cudaSuccess) return PTYCHO_ECUDA;
    for (int i = 1; i < nsets; ++i)
      if (cudaStreamWaitEvent(streams[i], p.ev_fork, 0) != cudaSuccess) return PTYCHO_ECUDA;
  }

  for (int k = 0, off = 0; off < c.nbatch; ++k, off += p.B) {
    const int set = k % nsets;
    cudaStream_t cs = streams[set];
    float2* S = p.d_S + set * set_S;
    float* Ip = p.d_Ipart + set * set_I;
    la.Ipart = Ip;
    la.D = grad ? p.d_D + set * set_F : nullptr;
    aa.D = p.d_D + set * set_F;
    aa.Gt = p.d_Gt ? p.d_Gt + set * set_F : nullptr;
    a.batch_off = off;
    a.nb = (c.nbatch - off < p.B) ? (c.nbatch - off) : p.B;
    // region of each object the batch's patches cover (exact for the identity order, else
    // the whole object); the object-gradient kernel tiles it
    int max_tiles = 1;
    for (int l = 0; l < p.L && grad; ++l) {
      int y0 = 0, x0 = 0, y1 = p.obj_h[l], x1 = p.obj_w[l];
      if (identity) {
        y0 = x0 = 1 << 30;
        y1 = x1 = -1;
        for (int q = off; q < off + a.nb; ++q) {
          const int y = p.pos_host[((size_t)l * p.J + q) * 2], x = p.pos_host[((size_t)l * p.J + q) * 2 + 1];
          y0 = y < y0 ? y : y0; x0 = x < x0 ? x : x0;
          y1 = y + F > y1 ? y + F : y1; x1 = x + F > x1 ? x + F : x1;
        }
      }
      a.box[l][0] = y0; a.box[l][1] = x0; a.box[l][2] = y1; a.box[l][3] = x1;
      const int tiles = ((y1 - y0 + kTile - 1) / kTile) * ((x1 - x0 + kTile - 1) / kTile);
      max_tiles = tiles > max_tiles ? tiles : max_tiles;
    }
    // forward: all chunks accumulate the model intensity
    // fractional offsets: shift the batch's object windows into the patch buffer
    const long long set_P = (long long)p.B * p.L * FF;
    ShiftArgs sh{};
    if (shifted) {
      sh.delta = p.d_delta;
      sh.T = p.d_shT + set * set_P;
      sh.Q = p.d_shQ + set * set_P;
      float2* Pt = p.d_shP + set * set_P;
      const dim3 rgrid(F / RowCfg<F>::RPB, p.L, a.nb), cgrid(F / ColCfg<F>::W, p.L, a.nb);
      sh.dst = sh.T; sh.dst_b = (long long)p.L * FF; sh.dst_l = FF; sh.scale = 1.0f;
      PTY_LAUNCH(p, kShift, cs, launch_pdl(k_shift_rows<F, false, true>, rgrid, row_blk, RowCfg<F>::smem, cs, c.O, a, sh));
      PTY_LAUNCH(p, kShift, cs, launch_pdl(k_shift_cols<F, false>, cgrid, col_blk, ColCfg<F>::smem_xch, cs, a, sh));
      sh.src = sh.T; sh.src_b = (long long)p.L * FF; sh.src_l = FF;
      sh.dst = Pt; sh.scale = 1.0f / (float)FF;
      PTY_LAUNCH(p, kShift, cs, launch_pdl(k_shift_rows<F, true, false>, rgrid, row_blk, RowCfg<F>::smem, cs, c.O, a, sh));
      a.patch = Pt;
    }
    if constexpr (ResSupported<F>::value) {
      if (res) {                                      // all modes of the batch, frames on chip
        a.chunk_base = 0;
        a.chunk_len = LM;
        PTY_LAUNCH(p, kResFwd, cs, launch_pdl(k_res_fwd<F>, dim3(a.nb, a.G), ResCfg<F>::threads, ResCfg<F>::smem, cs,
                                              c.O, c.P, Ip, a));
      }
    }
    for (int ch = 0; ch < p.nchunks && !res; ++ch) {
      a.chunk_base = ch * p.C;
      a.chunk_len = (LM - a.chunk_base < p.C) ? (LM - a.chunk_base) : p.C;
      {
        if (p.czt) {                                  // chirp-z propagator
          PTY_LAUNCH(p, kRowFwd, cs, launch_pdl(k_czt_row_fwd<F>, dim3(a.nb, F / CztRowCfg<F>::RPB, p.L),
                                                CztRowCfg<F>::threads, CztRowCfg<F>::smem, cs, c.O, c.P, S, a, ct));
          PTY_LAUNCH(p, kColFwd, cs, launch_pdl(k_czt_col_fwd<F>, dim3(F / CztColCfg<F>::W, p.G, a.nb),
                                                CztColCfg<F>::threads, CztColCfg<F>::smem_fwd, cs, (const float2*)S, Ip,
                                                a, ct));
          continue;
        }
      }
      bool warp_rows_fwd = false;
      if constexpr (F == 512) {
        if (fwd_l && p.fwd_l_w) {
          PTY_LAUNCH(p, kRowFwd, cs,
                     launch_pdl(k_row_fwd_w<F>, dim3(F / p.rpb_adj, p.L, p.nsplit_fwd), 32 * p.M * p.rpb_adj,
                                row_fwd_w_smem(p.M, p.rpb_adj), cs, c.O, c.P, S, a, p.rpb_adj, p.nsplit_fwd));
          warp_rows_fwd = true;
        }
      }
      if (warp_rows_fwd)
        ;
      else if (fwd_l)
        PTY_LAUNCH(p, kRowFwd, cs,
                   launch_pdl(k_row_fwd_l<F>, dim3(F / p.rpb_adj, p.L, p.nsplit_fwd), FftShape<F>::N1 * p.M * p.rpb_adj,
                              row_fwd_l_smem<F>(p.M, p.rpb_adj), cs, c.O, c.P, S, a, p.rpb_adj, p.nsplit_fwd));
      else
        PTY_LAUNCH(p, kRowFwd, cs,
                   launch_pdl(k_row_fwd<F>, dim3(a.nb, F / RowCfg<F>::RPB, p.L), row_blk, RowCfg<F>::smem, cs, c.O, c.P, S, a));
      const dim3 col_grid(F / ColCfg<F>::W, p.G, a.nb);
      if (col_staged) {
        rc = narrow ? launch_cols_s<F, 4>(p, true, store, cs, S, Ip, a, aa) : launch_cols_s<F, 0>(p, true, store, cs, S, Ip, a, aa);
        if (rc) return rc;
      } else if (F == 512 && p.has_tma && p.col_tma2 && !store) {
        if constexpr (F == 512)
          PTY_LAUNCH(p, kColFwd, cs, launch_pdl(k_col_fwd_tma2<F>, col_grid, col_blk, ColTma2<F>::smem, cs,
                                                p.tmap_S[set], Ip, a, (int)(ch == 0)));
      } else if (p.has_tma && store)
        PTY_LAUNCH(p, kColFwd, cs, launch_pdl(k_col_fwd_tma<F, true>, col_grid, col_blk, ColTma<F>::smem_fwd, cs,
                                              p.tmap_S[set], S, Ip, a, (int)(ch == 0)));
      else if (p.has_tma)
        PTY_LAUNCH(p, kColFwd, cs, launch_pdl(k_col_fwd_tma<F, false>, col_grid, col_blk, ColTma<F>::smem_fwd, cs,
                                              p.tmap_S[set], S, Ip, a, (int)(ch == 0)));
      else if (F >= 512 && store)
        PTY_LAUNCH(p, kColFwd, cs, launch_pdl(k_col_fwd_2b<F, true>, col_grid, col_blk, ColCfg<F>::smem_xch, cs, S, Ip,
                                              a, (int)(ch == 0)));
      else if (F >= 512)
        PTY_LAUNCH(p, kColFwd, cs, launch_pdl(k_col_fwd_2b<F, false>, col_grid, col_blk, ColCfg<F>::smem_xch, cs, S, Ip,
                                              a, (int)(ch == 0)));
      else if (store)
        PTY_LAUNCH(p, kColFwd, cs, launch_pdl(k_col_fwd<F, true>, col_grid, col_blk, ColCfg<F>::smem_xch, cs, S, Ip, a,
                                              (int)(ch == 0)));
      else
        PTY_LAUNCH(p, kColFwd, cs, launch_pdl(k_col_fwd<F, false>, col_grid, col_blk, ColCfg<F>::smem_xch, cs, S, Ip, a,
                                              (int)(ch == 0)));
    }
    if (p.imeas_ready && cudaStreamWaitEvent(cs, p.imeas_ready[k], 0) != cudaSuccess) return PTYCHO_ECUDA;
    PTY_LAUNCH(p, kLoss, cs, launch_pdl(k_loss<F>, dim3(loss_blocks<F>(), a.nb), kLossThreads, 0, cs, a, la));
    if (!grad) continue;
    if (p.remap) PTY_LAUNCH(p, kRemapAdj, cs, launch_pdl(k_remap_adj<F>, dim3(FF / 256, (a.nb + kRtPos - 1) / kRtPos), 256, 0, cs, a, aa));
    if (c.g_bg)                                       // per-set background-gradient sum, batch order
      PTY_LAUNCH(p, kRemapAdj, cs, launch_pdl(k_bg_accum<F>, dim3(FF / 256), 256, 0, cs,
                                              (const float*)(p.remap ? aa.Gt : aa.D), a.nb, p.d_gbg_set + set * FF));
    for (int ch = 0; ch < p.nchunks; ++ch) {
      a.chunk_base = ch * p.C;
      a.chunk_len = (LM - a.chunk_base < p.C) ? (LM - a.chunk_base) : p.C;
      const dim3 col_grid(F / ColCfg<F>::W, p.G, a.nb);
      if constexpr (ResSupported<F>::value) {
        if (res) {                                    // Psi recomputed on chip, chi, both gradients
          if (nsets > 1 && k > 0 && cudaStreamWaitEvent(cs, p.ev_radj[(k - 1) % nsets], 0) != cudaSuccess)
            return PTYCHO_ECUDA;
          PTY_LAUNCH(p, kResAdj, cs, launch_pdl(k_res_adj<F>, dim3(LM, nsplit), ResCfg<F>::threads, ResCfg<F>::smem, cs,
                                                c.O, c.P, S, gPs, (long long)p.P_numel, a, aa, nsplit));
          if (nsets > 1 && cudaEventRecord(p.ev_radj[k % nsets], cs) != cudaSuccess) return PTYCHO_ECUDA;
          if (nsets > 1 && k > 0 && cudaStreamWaitEvent(cs, p.ev_og[(k - 1) % nsets], 0) != cudaSuccess)
            return PTYCHO_ECUDA;
          PTY_LAUNCH(p, kObjGrad, cs, launch_pdl(k_obj_grad<F>, dim3(max_tiles, p.L), 256, 0, cs, S, c.gO, a));
          if (nsets > 1 && cudaEventRecord(p.ev_og[k % nsets], cs) != cudaSuccess) return PTYCHO_ECUDA;
          continue;
        }
      }
      {
        if (p.czt) {                                  // chirp-z propagator
          PTY_LAUNCH(p, kColAdj, cs, launch_pdl(k_czt_col_adj<F>, dim3(F / CztColCfg<F>::W, p.G, a.nb),
                                                CztColCfg<F>::threads, CztColCfg<F>::smem_adj, cs, S, a, aa, ct));
          if (nsets > 1 && k > 0 && cudaStreamWaitEvent(cs, p.ev_radj[(k - 1) % nsets], 0) != cudaSuccess)
            return PTYCHO_ECUDA;
          PTY_LAUNCH(p, kRowAdj, cs, launch_pdl(k_czt_row_adj<F>, dim3(F / CztRowAdjCfg<F>::RPB, a.chunk_len),
                                                CztRowAdjCfg<F>::threads, CztRowAdjCfg<F>::smem, cs, c.O, c.P, S, c.gP,
                                                a, ct));
          if (nsets > 1 && cudaEventRecord(p.ev_radj[k % nsets], cs) != cudaSuccess) return PTYCHO_ECUDA;
          if (nsets > 1 && k > 0 && cudaStreamWaitEvent(cs, p.ev_og[(k - 1) % nsets], 0) != cudaSuccess)
            return PTYCHO_ECUDA;
          PTY_LAUNCH(p, kObjGrad, cs, launch_pdl(k_obj_grad<F>, dim3(max_tiles, p.L), 256, 0, cs, S, c.gO, a));
          if (nsets > 1 && cudaEventRecord(p.ev_og[k % nsets], cs) != cudaSuccess) return PTYCHO_ECUDA;
          continue;
        }
      }
      if (!store && rerun_rows)
        PTY_LAUNCH(p, kRowFwd, cs,
                   launch_pdl(k_row_fwd<F>, dim3(a.nb, F / RowCfg<F>::RPB, p.L), row_blk, RowCfg<F>::smem, cs, c.O, c.P, S, a));
      if (col_staged) {
        rc = narrow ? launch_cols_s<F, 4>(p, false, store, cs, S, Ip, a, aa) : launch_cols_s<F, 0>(p, false, store, cs, S, Ip, a, aa);
        if (rc) return rc;
      } else if (F == 512 && p.has_tma && p.col_tma2 && !store) {
        if constexpr (F == 512)
          PTY_LAUNCH(p, kColAdj, cs, launch_pdl(k_col_adj_tma2<F>, col_grid, col_blk, ColTma2<F>::smem, cs,
                                                p.tmap_S[set], S, a, aa));
      } else if (p.has_tma && store)
        PTY_LAUNCH(p, kColAdj, cs, launch_pdl(k_col_adj_tma<F, true>, col_grid, col_blk, ColTma<F>::smem_adj, cs,
                                              p.tmap_S[set], S, a, aa));
      else if (p.has_tma)
        PTY_LAUNCH(p, kColAdj, cs, launch_pdl(k_col_adj_tma<F, false>, col_grid, col_blk, ColTma<F>::smem_adj, cs,
                                              p.tmap_S[set], S, a, aa));
      else if (F >= 512 && store)
        PTY_LAUNCH(p, kColAdj, cs, launch_pdl(k_col_adj_2b<F, true>, col_grid, col_blk, col_adj_smem, cs, S, a, aa));
      else if (F >= 512)
        PTY_LAUNCH(p, kColAdj, cs, launch_pdl(k_col_adj_2b<F, false>, col_grid, col_blk, col_adj_smem, cs, S, a, aa));
      else if (store)
        PTY_LAUNCH(p, kColAdj, cs, launch_pdl(k_col_adj<F, true>, col_grid, col_blk, col_adj_smem, cs, S, a, aa));
      else
        PTY_LAUNCH(p, kColAdj, cs, launch_pdl(k_col_adj<F, false>, col_grid, col_blk, col_adj_smem, cs, S, a, aa));
      // the probe and object gradients accumulate in batch order across the streams
      if (nsets > 1 && k > 0 && cudaStreamWaitEvent(cs, p.ev_radj[(k - 1) % nsets], 0) != cudaSuccess)
        return PTYCHO_ECUDA;
      if (adj_l) {
        constexpr int T = FftShape<F>::N1;
        bool warp_rows = false;
        if constexpr (F == 512) {
          if (p.adj_l_w) {
            PTY_LAUNCH(p, kRowAdj, cs,
                       launch_pdl(k_row_adj_w<F>, dim3(F / p.rpb_adj, p.L, nsplit), 32 * p.M * p.rpb_adj,
                                  row_adj_w_smem(p.M, p.rpb_adj), cs, c.O, c.P, S, gPs, (long long)p.P_numel, a,
                                  p.rpb_adj, nsplit));
            warp_rows = true;
          }
        }
        if (warp_rows)
          ;
        else if (p.adj_l_pl2)
          PTY_LAUNCH(p, kRowAdj, cs,
                     launch_pdl(k_row_adj_l<F, true>, dim3(F / p.rpb_adj, p.L, nsplit), T * p.M * p.rpb_adj,
                                row_adj_l_smem<F>(p.M, p.rpb_adj, true), cs, c.O, c.P, S, gPs, (long long)p.P_numel,
                                a, p.rpb_adj, nsplit));
        else
          PTY_LAUNCH(p, kRowAdj, cs,
                     launch_pdl(k_row_adj_l<F, false>, dim3(F / p.rpb_adj, p.L, nsplit), T * p.M * p.rpb_adj,
                                row_adj_l_smem<F>(p.M, p.rpb_adj), cs, c.O, c.P, S, gPs, (long long)p.P_numel, a,
                                p.rpb_adj, nsplit));
        if (nsets > 1 && cudaEventRecord(p.ev_radj[k % nsets], cs) != cudaSuccess) return PTYCHO_ECUDA;
        if (shifted) {                                // adjoint shift of the mode-summed patch gradients
          const dim3 rgrid(F / RowCfg<F>::RPB, p.L, a.nb), cgrid(F / ColCfg<F>::W, p.L, a.nb);
          sh.src = S; sh.src_b = (long long)p.C * FF; sh.src_l = (long long)p.M * FF;
          sh.dst = sh.T; sh.dst_b = (long long)p.L * FF; sh.dst_l = FF; sh.scale = 1.0f;
          PTY_LAUNCH(p, kShift, cs, launch_pdl(k_shift_rows<F, false, false>, rgrid, row_blk, RowCfg<F>::smem, cs, c.O, a, sh));
          sh.dpart = c.g_delta ? p.d_dpart : nullptr;
          PTY_LAUNCH(p, kShift, cs, launch_pdl(k_shift_cols<F, true>, cgrid, col_blk, ColCfg<F>::smem_xch, cs, a, sh));
          sh.src = sh.T; sh.src_b = (long long)p.L * FF; sh.src_l = FF;
          sh.dst = S; sh.dst_b = (long long)p.C * FF; sh.dst_l = (long long)p.M * FF; sh.scale = 1.0f / (float)FF;
          PTY_LAUNCH(p, kShift, cs, launch_pdl(k_shift_rows<F, true, false>, rgrid, row_blk, RowCfg<F>::smem, cs, c.O, a, sh));
          sh.dpart = nullptr;
        }
        if (nsets > 1 && k > 0 && cudaStreamWaitEvent(cs, p.ev_og[(k - 1) % nsets], 0) != cudaSuccess)
          return PTYCHO_ECUDA;
        PTY_LAUNCH(p, kObjGrad, cs, launch_pdl(k_obj_grad_l<F>, dim3(max_tiles, p.L), 256, 0, cs, S, c.gO, a));
        if (nsets > 1 && cudaEventRecord(p.ev_og[k % nsets], cs) != cudaSuccess) return PTYCHO_ECUDA;
        continue;
      }
      if (obj_atomic)
        PTY_LAUNCH(p, kRowAdj, cs,
                   launch_pdl(k_row_adj<F, true>, dim3(F / RowAdjCfg<F>::RPB, a.chunk_len), RowAdjCfg<F>::threads, RowAdjCfg<F>::smem, cs, c.O, c.P, S, c.gP, c.gO, a));
      else
        PTY_LAUNCH(p, kRowAdj, cs,
                   launch_pdl(k_row_adj<F, false>, dim3(F / RowAdjCfg<F>::RPB, a.chunk_len), RowAdjCfg<F>::threads, RowAdjCfg<F>::smem, cs, c.O, c.P, S, c.gP, c.gO, a));
      if (nsets > 1 && cudaEventRecord(p.ev_radj[k % nsets], cs) != cudaSuccess) return PTYCHO_ECUDA;
      if (obj_atomic) continue;
      if (nsets > 1 && k > 0 && cudaStreamWaitEvent(cs, p.ev_og[(k - 1) % nsets], 0) != cudaSuccess)
        return PTYCHO_ECUDA;
      PTY_LAUNCH(p, kObjGrad, cs, launch_pdl(k_obj_grad<F>, dim3(max_tiles, p.L), 256, 0, cs, S, c.gO, a));
      if (nsets > 1 && cudaEventRecord(p.ev_og[k % nsets], cs) != cudaSuccess) return PTYCHO_ECUDA;
    }
  }
  for (int i = 1; i < nsets; ++i) {                   // join the side streams back
    if (cudaEventRecord(p.ev_join[i - 1], streams[i]) != cudaSuccess ||
        cudaStreamWaitEvent(st, p.ev_join[i - 1], 0) != cudaSuccess)
      return PTYCHO_ECUDA;
  }
  if (grad && nsplit > 1)
    PTY_LAUNCH(p, kRowAdj, st,
               launch_pdl(k_sum_splits, dim3(4 * p.sms), 256, 0, st, (const float2*)gPs, nsplit, p.P_numel, c.gP));
  if (grad && c.g_z)
    PTY_LAUNCH(p, kLossReduce, st,
               launch_pdl(k_loss_reduce, 1, 256, 0, st, (const double*)p.d_z_part,
                          (long long)c.nbatch * loss_blocks<F>(), c.g_z));
  if (grad && c.g_delta)
    PTY_LAUNCH(p, kShift, st,
               launch_pdl(k_delta_grad, dim3((p.L * p.J + 255) / 256), 256, 0, st, (const int32_t*)c.bidx, c.nbatch,
                          p.L, p.J, (const double*)p.d_dpart, F / ColCfg<F>::W, c.g_delta));
  if (grad && c.g_sigma)
    PTY_LAUNCH(p, kLossReduce, st,
               launch_pdl(k_sigma_grad, dim3((p.J + 255) / 256), 256, 0, st, (const int32_t*)c.bidx, c.nbatch, p.J,
                          (const double*)p.d_sig_part, loss_blocks<F>(), c.sigma, c.g_sigma));
  if (grad && c.g_bg)
    PTY_LAUNCH(p, kLossReduce, st,
               launch_pdl(k_sum_sets, dim3(FF / 256), 256, 0, st, (const float*)p.d_gbg_set, nsets, (long long)FF,
                          c.g_bg));
  if (need_loss) {
    double* out = c.loss;
    if (out) {
      PTY_LAUNCH(p, kLossReduce, st,
                 launch_pdl(k_loss_reduce, 1, 256, 0, st, p.d_loss_part, (long long)c.nbatch * loss_blocks<F>(), out));
    }
  }
  return PTYCHO_OK;
}

}  // namespace ptycho
