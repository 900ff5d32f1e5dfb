// Plain (unfused) form of one optimisation step, kept as the baseline the fused and served
// paths are measured against: one site at a time, every stage a separate kernel with its
// result in a device buffer, the same in-register FFT code, and the object / probe
// gradients scattered with FP32 atomics.
//
//   k_pl_exit      psi[b][mode] = sigma P_mode * O_l(patch)              (gather, f1-f3)
//   k_pl_rows      1D DFT of every row of every frame (forward or inverse, in place)
//   k_pl_cols      1D DFT of every column of every frame (in place), optional scale
//   k_pl_intensity I[b] = sum over modes |Psi|^2 on the centred model grid
//   k_loss / k_remap_adj   measurement, loss and R^T (shared with the fused path)
//   k_pl_mul       Psi <- (2/F) G Psi                                      (centred G)
//   k_pl_scatter   grad P += conj(sigma p) chi, grad O += conj(sigma P) chi (atomics)
//   k_adam         Adam
#pragma once
#include <algorithm>

#include "pipeline.cuh"

namespace ptycho {

template <int F>
__global__ void __launch_bounds__(256) k_pl_exit(const float2* __restrict__ O, const float2* __restrict__ P,
                                                 float2* __restrict__ psi, KArgs a, int LM) {
  const int b = blockIdx.z, mode = blockIdx.y;
  const int l = mode / a.M;
  const int j = batch_pos(a, a.batch_off + b);
  if (j < 0) return;
  const int y = a.pos[(l * a.J + j) * 2], x = a.pos[(l * a.J + j) * 2 + 1];
  const float s = sigma_of(a, j);
  float2* out = psi + ((long long)b * LM + mode) * F * F;
  for (int e = blockIdx.x * 256 + threadIdx.x; e < F * F; e += gridDim.x * 256) {
    const int r = e / F, c = e % F;
    const float2 p = O[a.obj_off[l] + (long long)(y + r) * a.obj_w[l] + x + c];
    out[e] = cscale(cmul(P[((long long)mode * F + r) * F + c], p), s);
  }
}

// rows: INV = false takes layout I and stores natural order (layout O); INV = true reads
// natural order in layout O and stores layout I.   grid (F/RPB, nframes)
template <int F, bool INV>
__global__ void __launch_bounds__(RowCfg<F>::threads) k_pl_rows(float2* __restrict__ buf, const float2* __restrict__ tw) {
  constexpr int N1 = FftShape<F>::N1, N2 = FftShape<F>::N2, T = RowCfg<F>::T;
  extern __shared__ float2 smem[];
  const int vec = threadIdx.x / T, t = threadIdx.x % T;
  float2* row = buf + ((long long)blockIdx.y * F + blockIdx.x * RowCfg<F>::RPB + vec) * F;
  float2 v[N2];
  if (!INV) {
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) v[n2] = row[idxI<F>(t, n2)];
    fft_fwd_I2O<F>(v, t, smem + vec * Xch<F>::region_rows, tw, WarpSync{});
#pragma unroll
    for (int sl = 0; sl < N2; ++sl) row[idxO<F>(t, sl)] = v[sl];
  } else {
#pragma unroll
    for (int sl = 0; sl < N2; ++sl) v[sl] = row[idxO<F>(t, sl)];
    fft_inv_O2I<F>(v, t, smem + vec * Xch<F>::region_rows, tw, WarpSync{});
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) row[idxI<F>(t, n2)] = v[n2];
  }
}

template <int F, bool INV>
__global__ void __launch_bounds__(ColCfg<F>::threads) k_pl_cols(float2* __restrict__ buf, const float2* __restrict__ tw,
                                                                float scale) {
  constexpr int N1 = FftShape<F>::N1, N2 = FftShape<F>::N2, W = ColCfg<F>::W;
  extern __shared__ float2 smem[];
  const int c = threadIdx.x % W, t = threadIdx.x / W;
  float2* base = buf + (long long)blockIdx.y * F * F + blockIdx.x * W + c;
  float2 v[N2];
  if (!INV) {
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) v[n2] = base[(long long)idxI<F>(t, n2) * F];
    fft_fwd_I2O<F>(v, t, smem + c * Xch<F>::region_cols, tw, BlockSync{});
#pragma unroll
    for (int sl = 0; sl < N2; ++sl) base[(long long)idxO<F>(t, sl) * F] = cscale(v[sl], scale);
  } else {
#pragma unroll
    for (int sl = 0; sl < N2; ++sl) v[sl] = base[(long long)idxO<F>(t, sl) * F];
    fft_inv_O2I<F>(v, t, smem + c * Xch<F>::region_cols, tw, BlockSync{});
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) base[(long long)idxI<F>(t, n2) * F] = cscale(v[n2], scale);
  }
}

// grid (F*F/256, nb)
template <int F>
__global__ void __launch_bounds__(256) k_pl_intensity(const float2* __restrict__ psi, float* __restrict__ I, int LM) {
  const int b = blockIdx.y;
  const int e = blockIdx.x * 256 + threadIdx.x;
  float acc = 0.f;
  for (int mode = 0; mode < LM; ++mode) {
    const float2 v = psi[((long long)b * LM + mode) * F * F + e];
    acc = fmaf(v.x, v.x, fmaf(v.y, v.y, acc));
  }
  const int r = e / F, c = e % F;
  I[(long long)b * F * F + ((r + F / 2) & (F - 1)) * F + ((c + F / 2) & (F - 1))] = acc;
}

// grid (F*F/256, LM, nb)
template <int F>
__global__ void __launch_bounds__(256) k_pl_mul(float2* __restrict__ psi, const float* __restrict__ G, int LM) {
  const int b = blockIdx.z, mode = blockIdx.y;
  const int e = blockIdx.x * 256 + threadIdx.x;
  const int r = e / F, c = e % F;
  const float g = G[(long long)b * F * F + ((r + F / 2) & (F - 1)) * F + ((c + F / 2) & (F - 1))] * (2.0f / F);
  float2* p = psi + ((long long)b * LM + mode) * F * F + e;
  *p = cscale(*p, g);
}

// grid (F*F/256, LM, nb)
template <int F>
__global__ void __launch_bounds__(256) k_pl_scatter(const float2* __restrict__ O, const float2* __restrict__ P,
                                                    const float2* __restrict__ chi, float2* __restrict__ gO,
                                                    float2* __restrict__ gP, KArgs a, int LM) {
  const int b = blockIdx.z, mode = blockIdx.y;
  const int l = mode / a.M;
  const int j = batch_pos(a, a.batch_off + b);
  if (j < 0) return;
  const int y = a.pos[(l * a.J + j) * 2], x = a.pos[(l * a.J + j) * 2 + 1];
  const float s = sigma_of(a, j);
  const int e = blockIdx.x * 256 + threadIdx.x;
  const int r = e / F, c = e % F;
  const float2 ch = chi[((long long)b * LM + mode) * F * F + e];
  const long long oi = a.obj_off[l] + (long long)(y + r) * a.obj_w[l] + x + c;
  const long long pi = ((long long)mode * F + r) * F + c;
  const float2 gp = cscale(cconjmul(O[oi], ch), s);
  const float2 go = cscale(cconjmul(P[pi], ch), s);
  atomicAdd(&gP[pi].x, gp.x);
  atomicAdd(&gP[pi].y, gp.y);
  atomicAdd(&gO[oi].x, go.x);
  atomicAdd(&gO[oi].y, go.y);
}

template <int F>
int plain_adjoint(ptycho_plan& p, const CallArgs& c, float2* psi, float* Ibuf, float* Dbuf, float* Gbuf, int Bp,
                  cudaStream_t st) {
  const int LM = p.L * p.M;
  constexpr int FF = F * F;
  {
    cudaError_t e = cudaFuncSetAttribute(k_pl_rows<F, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, RowCfg<F>::smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pl_rows<F, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, RowCfg<F>::smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pl_cols<F, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, ColCfg<F>::smem_xch);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_pl_cols<F, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, ColCfg<F>::smem_xch);
    if (e != cudaSuccess) return PTYCHO_ECUDA;
  }
  KArgs a{};
  a.L = p.L; a.M = p.M; a.F = F; a.J = p.J;
  a.pos = p.d_pos;
  for (int l = 0; l < p.L; ++l) { a.obj_off[l] = p.obj_off[l]; a.obj_h[l] = p.obj_h[l]; a.obj_w[l] = p.obj_w[l]; }
  a.bidx = c.bidx;
  a.nbatch = c.nbatch;
  a.sigma = c.sigma;
  a.tw = p.d_tw;
  a.G = 1;
  a.status = p.d_status;
  LossArgs la{};
  la.Ipart = Ibuf;
  la.bg = c.bg;
  la.tap_base = p.d_tap_base;
  la.tap_w = p.d_tap_w;
  la.Imeas = c.Imeas;
  la.mask = c.mask;
  la.mask_per_frame = c.mask_per_frame;
  la.eps = p.eps;
  la.loss_kind = p.loss_kind;
  la.read_var = p.read_var;
  la.D = Dbuf;                                        // [Bp][F][F], sized by the caller
  la.loss_part = p.d_loss_part;
  la.remap = p.remap;
  la.Gsum = 1;
  AdjArgs aa{};
  aa.D = Dbuf;
  aa.rt_ptr = p.d_rt_ptr;
  aa.rt_idx = p.d_rt_idx;
  aa.rt_w = p.d_rt_w;
  aa.Gt = Gbuf;                                       // [Bp][F][F]
  aa.remap = p.remap;
  if (cudaMemsetAsync(c.gO, 0, sizeof(float2) * p.O_numel, st) != cudaSuccess) return PTYCHO_ECUDA;
  if (cudaMemsetAsync(c.gP, 0, sizeof(float2) * p.P_numel, st) != cudaSuccess) return PTYCHO_ECUDA;
  p.last_launches = 0;
  const float inv = 1.0f / (float)F;
  for (int off = 0; off < c.nbatch; off += Bp) {
    a.batch_off = off;
    a.nb = std::min(Bp, c.nbatch - off);
    const int frames = a.nb * LM;
    PTY_LAUNCH(p, kRowFwd, st, k_pl_exit<F><<<dim3(std::max(1, FF / 4096), LM, a.nb), 256, 0, st>>>(c.O, c.P, psi, a, LM));
    PTY_LAUNCH(p, kRowFwd, st, k_pl_rows<F, false><<<dim3(F / RowCfg<F>::RPB, frames), RowCfg<F>::threads, RowCfg<F>::smem, st>>>(psi, p.d_tw));
    PTY_LAUNCH(p, kColFwd, st, k_pl_cols<F, false><<<dim3(F / ColCfg<F>::W, frames), ColCfg<F>::threads, ColCfg<F>::smem_xch, st>>>(psi, p.d_tw, inv));
    PTY_LAUNCH(p, kColFwd, st, k_pl_intensity<F><<<dim3(FF / 256, a.nb), 256, 0, st>>>(psi, Ibuf, LM));
    PTY_LAUNCH(p, kLoss, st, k_loss<F><<<dim3(loss_blocks<F>(), a.nb), kLossThreads, 0, st>>>(a, la));
    if (p.remap) PTY_LAUNCH(p, kRemapAdj, st, k_remap_adj<F><<<dim3(FF / 256, (a.nb + kRtPos - 1) / kRtPos), 256, 0, st>>>(a, aa));
    PTY_LAUNCH(p, kColAdj, st, k_pl_mul<F><<<dim3(FF / 256, LM, a.nb), 256, 0, st>>>(psi, p.remap ? Gbuf : Dbuf, LM));
    PTY_LAUNCH(p, kColAdj, st, k_pl_cols<F, true><<<dim3(F / ColCfg<F>::W, frames), ColCfg<F>::threads, ColCfg<F>::smem_xch, st>>>(psi, p.d_tw, inv));
    PTY_LAUNCH(p, kRowAdj, st, k_pl_rows<F, true><<<dim3(F / RowCfg<F>::RPB, frames), RowCfg<F>::threads, RowCfg<F>::smem, st>>>(psi, p.d_tw));
    PTY_LAUNCH(p, kObjGrad, st, k_pl_scatter<F><<<dim3(FF / 256, LM, a.nb), 256, 0, st>>>(c.O, c.P, psi, c.gO, c.gP, a, LM));
  }
  if (c.loss) {
    PTY_LAUNCH(p, kLossReduce, st,
               k_loss_reduce<<<1, 256, 0, st>>>(p.d_loss_part, (long long)c.nbatch * loss_blocks<F>(), c.loss));
  }
  return PTYCHO_OK;
}

}  // namespace ptycho
