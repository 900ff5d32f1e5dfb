// Kernels of the batched multi-wavelength, multi-mode ptychography forward model and its
// adjoint (Eq. 1 written as f5(f4(f3(f1(sigma_j), f2(s_j)))) of Eq. 2).
//
// Work is organised per *position batch* (B scan positions) and per *mode chunk* (a run of
// the L*M (wavelength, probe-mode) pairs, index mode = l*M + m).  For a batch the 2D DFT of
// every exit wave goes through a scratch buffer S[B][C][F][F] (complex64) sized to stay in
// the GPU's L2 cache:
//
//   k_row_fwd   psi = sigma_j P_lm * O_l(r - s_j) for one row of every mode of a wavelength
//               (the object row is read once); 1D FFT along the row -> S
//   k_col_fwd   1D FFT along columns of S -> Psi (scaled by 1/F); accumulate |Psi|^2 over
//               the modes of a group into Ipart; optionally keep Psi in S for the adjoint
//   k_loss      I = sum of groups (+ background) on the model grid; tilted-plane remap to the
//               camera grid; mask; loss terms (FP64 block partials) and D = mask dL/dI
//   k_remap_adj G = R^T D on the model grid (only with the remap; otherwise G = D)
//   k_col_adj   Psi (kept, or recomputed from S); (2/F) G Psi; inverse column DFT -> S
//   k_row_adj   inverse 1D FFT along rows -> chi = dL/dpsi; grad P_lm += conj(sigma p) chi
//               summed over the batch in registers; S <- conj(sigma P_lm) chi
//   k_obj_grad  grad O_l tile += sum over the batch's overlapping patches and the chunk's
//               modes of S (each object tile is owned by one thread block: deterministic)
//   k_loss_reduce  fixed-order FP64 sum of the per-block loss partials
//   k_sigma_grad, k_bg_accum, k_sum_sets  gradients of the power coefficients and of the
//               background (optional outputs of the adjoint)
//   k_adam      Adam on the real and imaginary parts of O and P
#pragma once
#include "fft_regs.cuh"
#include "tma.cuh"

namespace ptycho {

constexpr int kMaxL = 16;
constexpr int kLossThreads = 256;
constexpr int kTile = 32;        // object-gradient tile side
constexpr int kMaxB = 512;       // positions per batch (upper bound)

struct KArgs {
  int L, M, F, J;
  const int32_t* pos;            // [L][J][2] (row, col) of the patch corner, device
  long long obj_off[kMaxL];      // complex offset of O_l in the packed object buffer
  int obj_h[kMaxL], obj_w[kMaxL];
  const int32_t* bidx;           // positions of this call, in processing order
  int nbatch;                    // number of entries in bidx
  int batch_off;                 // first entry of the current position batch
  int nb;                        // positions in the current batch (<= B <= kMaxB)
  const float* sigma;            // [J] power coefficients or null
  const float2* tw;              // W_F^(t*k2) table
  int C;                         // stride (modes) of the scratch buffer
  int chunk_base, chunk_len;     // global modes [chunk_base, chunk_base + chunk_len)
  int MG;                        // modes per column-kernel group
  int G;                         // groups per chunk (Ipart has G slices per position)
  int* status;                   // device status word (bit 0: a position index was out of range)
  int box[kMaxL][4];             // per wavelength: rows [box0, box2) x cols [box1, box3) covered by
                                 // the batch's patches (the whole object when not known on the host)
};

// Programmatic dependent launch: the pipeline launches each kernel so that it may start
// while the previous kernel of its stream finishes.  pdl_wait() blocks until that kernel
// has completed and its writes are visible (a no-op for an ordinary launch); every pipeline
// kernel calls it before touching global memory.  pdl_trigger() lets the next kernel start
// launching its blocks.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" :::); }

// Position index of batch entry i, or -1 (and the status bit set) if out of range.
__device__ __forceinline__ int batch_pos(const KArgs& a, int i) {
  const int j = a.bidx[i];
  if (j < 0 || j >= a.J) {
    atomicOr(a.status, 1);
    return -1;
  }
  return j;
}

// Scan positions (row, col) of the current batch for wavelength l and their power
// coefficients, staged in shared memory (block-strided); invalid entries become (-1, -1).
// Ends with a block barrier.
__device__ __forceinline__ void stage_batch(const KArgs& a, int l, int2* spos, float* ssig) {
  for (int b = threadIdx.x; b < a.nb; b += blockDim.x) {
    const int j = batch_pos(a, a.batch_off + b);
    if (j < 0) {
      spos[b] = make_int2(-1, -1);
      ssig[b] = 0.f;
    } else {
      spos[b] = make_int2(a.pos[(l * a.J + j) * 2], a.pos[(l * a.J + j) * 2 + 1]);
      ssig[b] = a.sigma ? __ldg(a.sigma + j) : 1.0f;
    }
  }
  __syncthreads();
}

template <int F> struct RowCfg {
  static constexpr int T = FftShape<F>::N1;
  static constexpr int RPB = 256 / T;            // rows per block
  static constexpr int threads = RPB * T;
  static constexpr int smem = RPB * Xch<F>::region_rows * (int)sizeof(float2);
};
template <int F> struct ColCfg {
  static constexpr int T = FftShape<F>::N1;
  static constexpr int W = 256 / T;              // columns per block
  static constexpr int threads = W * T;
  static constexpr int smem_xch = W * Xch<F>::region_cols * (int)sizeof(float2);
};

__device__ __forceinline__ float sigma_of(const KArgs& a, int j) { return a.sigma ? __ldg(a.sigma + j) : 1.0f; }

// ---------------------------------------------------------------------------------------
// forward row pass: exit waves (f1, f2, f3) of every mode of wavelength l in the chunk and
// the row DFT (first half of f4).   grid (F/RPB, L, nb)
// ---------------------------------------------------------------------------------------
template <int F>
__global__ void __launch_bounds__(RowCfg<F>::threads)
k_row_fwd(const float2* __restrict__ O, const float2* __restrict__ P, float2* __restrict__ S, KArgs a) {
  pdl_wait();
  pdl_trigger();
  constexpr int N1 = FftShape<F>::N1, N2 = FftShape<F>::N2, T = RowCfg<F>::T;
  extern __shared__ float2 smem[];
  const int vec = threadIdx.x / T, t = threadIdx.x % T;
  const int r = blockIdx.x * RowCfg<F>::RPB + vec;
  const int l = blockIdx.y, b = blockIdx.z;
  const int mlo = max(a.chunk_base, l * a.M), mhi = min(a.chunk_base + a.chunk_len, (l + 1) * a.M);
  if (mlo >= mhi) return;                             // uniform over the block
  const int j = batch_pos(a, a.batch_off + b);
  if (j < 0) return;                                  // uniform over the block
  const int y = a.pos[(l * a.J + j) * 2], x = a.pos[(l * a.J + j) * 2 + 1];
  const float s = sigma_of(a, j);
  const float2* Orow = O + a.obj_off[l] + (long long)(y + r) * a.obj_w[l] + x;
  float2 p[N2];
#pragma unroll
  for (int n2 = 0; n2 < N2; ++n2) p[n2] = cscale(__ldg(Orow + t + N1 * n2), s);
  for (int mode = mlo; mode < mhi; ++mode) {
    const float2* Prow = P + ((long long)mode * F + r) * F;
    float2 v[N2];
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) v[n2] = cmul(__ldg(Prow + t + N1 * n2), p[n2]);
    fft_fwd_I2O<F>(v, t, smem + vec * Xch<F>::region_rows, a.tw, WarpSync{});
    float2* out = S + (((long long)b * a.C + (mode - a.chunk_base)) * F + r) * F;
#pragma unroll
    for (int sl = 0; sl < N2; ++sl) out[idxO<F>(t, sl)] = v[sl];
  }
}

// ---------------------------------------------------------------------------------------
// forward column pass: column DFT (second half of f4), |Psi|^2 summed over a mode group
// grid (F/W, G, nb)
// ---------------------------------------------------------------------------------------
template <int F, bool STORE>
__global__ void __launch_bounds__(ColCfg<F>::threads)
k_col_fwd(float2* __restrict__ S, float* __restrict__ Ipart, KArgs a, int first_chunk) {
  pdl_wait();
  pdl_trigger();
  constexpr int N1 = FftShape<F>::N1, N2 = FftShape<F>::N2, W = ColCfg<F>::W;
  extern __shared__ float2 smem[];
  const int c = threadIdx.x % W, t = threadIdx.x / W;
  const int col = blockIdx.x * W + c;
  const int g = blockIdx.y, b = blockIdx.z;
  const int m0 = g * a.MG, m1 = min(a.chunk_len, m0 + a.MG);
  float acc[N2];
#pragma unroll
  for (int i = 0; i < N2; ++i) acc[i] = 0.f;
  const float inv = 1.0f / (float)F;
  for (int cm = m0; cm < m1; ++cm) {
    float2* base = S + ((long long)b * a.C + cm) * F * F + col;
    float2 v[N2];
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) v[n2] = base[(long long)(t + N1 * n2) * F];
    fft_fwd_I2O<F>(v, t, smem + c * Xch<F>::region_cols, a.tw, BlockSync{});
#pragma unroll
    for (int sl = 0; sl < N2; ++sl) {
      acc[sl] = fmaf(v[sl].x, v[sl].x, fmaf(v[sl].y, v[sl].y, acc[sl]));
      if (STORE) base[(long long)idxO<F>(t, sl) * F] = cscale(v[sl], inv);
    }
  }
  float* dst = Ipart + ((long long)b * a.G + g) * F * F;
  const int cc = (col + F / 2) & (F - 1);
#pragma unroll
  for (int sl = 0; sl < N2; ++sl) {
    const int rc = (idxO<F>(t, sl) + F / 2) & (F - 1);
    float val = acc[sl] * (inv * inv);
    if (!first_chunk) val += dst[rc * F + cc];
    dst[rc * F + cc] = val;
  }
}

// ---------------------------------------------------------------------------------------
// TMA-staged column passes.  The W x F column block of one mode (W*F*8 bytes) arrives in
// shared memory through cp.async.bulk.tensor (2D tensor map over S viewed as
// [B*C*F rows][F columns] of 8-byte elements); the next mode's block is requested as soon as
// every thread has read the current one into registers, so the copy overlaps the FFT.
// ---------------------------------------------------------------------------------------
template <int F> struct ColTma {
  static constexpr int W = ColCfg<F>::W;
  static constexpr int box_rows = F < 256 ? F : 256;
  static constexpr int stage_bytes = F * W * (int)sizeof(float2);
  static constexpr int smem_fwd = stage_bytes + ColCfg<F>::smem_xch + 16;
  static constexpr int smem_adj = smem_fwd + F * W * (int)sizeof(float);
};

template <int F>
__device__ __forceinline__ void col_tma_issue(float2* stage, const CUtensorMap* map, int col0, int row0, uint64_t* bar) {
  fence_proxy_async_smem();                    // earlier generic reads of the stage come first
  mbar_arrive_expect_tx(bar, ColTma<F>::stage_bytes);
#pragma unroll
  for (int h = 0; h < F / ColTma<F>::box_rows; ++h)
    tma_load_2d(stage + h * ColTma<F>::box_rows * ColTma<F>::W, map, col0, row0 + h * ColTma<F>::box_rows, bar);
}

// grid (F/W, G, nb); same results as k_col_fwd
template <int F, bool STORE>
__global__ void __launch_bounds__(ColCfg<F>::threads)
k_col_fwd_tma(const __grid_constant__ CUtensorMap map, float2* __restrict__ S, float* __restrict__ Ipart, KArgs a,
              int first_chunk) {
  pdl_wait();
  pdl_trigger();
  constexpr int N1 = FftShape<F>::N1, N2 = FftShape<F>::N2, W = ColCfg<F>::W;
  extern __shared__ __align__(128) float2 smem[];
  float2* stage = smem;
  float2* xch = smem + F * W;
  uint64_t* bar = reinterpret_cast<uint64_t*>(xch + W * Xch<F>::region_cols);
  const int c = threadIdx.x % W, t = threadIdx.x / W;
  const int col0 = blockIdx.x * W, col = col0 + c;
  const int g = blockIdx.y, b = blockIdx.z;
  const int m0 = g * a.MG, m1 = min(a.chunk_len, m0 + a.MG);
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && m0 < m1) col_tma_issue<F>(stage, &map, col0, ((long long)b * a.C + m0) * F, bar);
  float acc[N2];
#pragma unroll
  for (int i = 0; i < N2; ++i) acc[i] = 0.f;
  const float inv = 1.0f / (float)F;
  uint32_t phase = 0;
  bool ok = true;
  for (int cm = m0; cm < m1; ++cm) {
    ok = __syncthreads_and(mbar_wait_bounded(bar, phase, a.status));
    if (!ok) break;
    phase ^= 1;
    float2 v[N2];
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) v[n2] = stage[(t + N1 * n2) * W + c];
    __syncthreads();                           // the stage is free for the next mode
    if (threadIdx.x == 0 && cm + 1 < m1) col_tma_issue<F>(stage, &map, col0, ((long long)b * a.C + cm + 1) * F, bar);
    fft_fwd_I2O<F>(v, t, xch + c * Xch<F>::region_cols, a.tw, BlockSync{});
    float2* base = S + ((long long)b * a.C + cm) * F * F + col;
#pragma unroll
    for (int sl = 0; sl < N2; ++sl) {
      acc[sl] = fmaf(v[sl].x, v[sl].x, fmaf(v[sl].y, v[sl].y, acc[sl]));
      if (STORE) base[(long long)idxO<F>(t, sl) * F] = cscale(v[sl], inv);
    }
  }
  if (!ok) {                                   // give a lost copy a bounded chance to land, then stop
    if (threadIdx.x == 0) mbar_wait_bounded(bar, phase, a.status);
    return;
  }
  float* dst = Ipart + ((long long)b * a.G + g) * F * F;
  const int cc = (col + F / 2) & (F - 1);
#pragma unroll
  for (int sl = 0; sl < N2; ++sl) {
    const int rc = (idxO<F>(t, sl) + F / 2) & (F - 1);
    float val = acc[sl] * (inv * inv);
    if (!first_chunk) val += dst[rc * F + cc];
    dst[rc * F + cc] = val;
  }
}

// ---------------------------------------------------------------------------------------
// measurement (f5) and loss: camera-grid prediction, masked loss partials, D = mask dL/dI.
// grid (F*F/256, nb)
// ---------------------------------------------------------------------------------------
struct LossArgs {
  const float* Ipart;            // [B][G][F][F] model grid (centred)
  const float* bg;               // [F][F] model grid or null
  const int32_t* tap_base;       // [F*F] top-left model tap of each camera pixel, -1 invalid
  const float2* tap_w;           // [F*F] (wy, wx)
  const float* Imeas;            // [J][F][F] camera grid
  const uint8_t* mask;           // null, [F][F] or [J][F][F]
  int mask_per_frame;
  float eps;
  int loss_kind;                 // 0 amplitude, 1 Poisson
  float* D;                      // [B][F][F] mask * dL/dI (camera grid), null if not needed
  double* loss_part;             // [nbatch][F*F/256] or null
  double* sig_part;              // [nbatch][F*F/256] sums of D * (remapped sum |Psi|^2), or null
  float* I_pred;                 // [J][F][F] or null
  int remap;
};

__device__ __forceinline__ float model_I(const float* Ip, const float* bg, int G, int FF, int u) {
  float s = 0.f;
  for (int g = 0; g < G; ++g) s += Ip[(long long)g * FF + u];
  if (bg) s += __ldg(bg + u);
  return s;
}

// Poisson deviance per pixel, I_hat * (r - 1 - log r) with r = Ie / I_hat, without the
// cancellation of the direct form near r = 1 (series of u - log(1+u), u = r - 1).
__device__ __forceinline__ float poisson_term(float Ie, float Ih) {
  if (Ih <= 0.f) return Ie;
  const float u = (Ie - Ih) / Ih;
  float f;
  if (fabsf(u) < 0.25f) {
    // u - log(1+u) = sum_{n>=2} (-1)^n u^n / n
    float p = 0.f;
#pragma unroll
    for (int n = 12; n >= 2; --n) p = fmaf(p, u, ((n & 1) ? -1.0f : 1.0f) / (float)n);
    f = p * u * u;
  } else {
    f = u - log1pf(u);
  }
  return Ih * f;
}

template <int F>
__global__ void __launch_bounds__(kLossThreads)
k_loss(KArgs a, LossArgs la) {
  pdl_wait();
  pdl_trigger();
  constexpr int FF = F * F;
  __shared__ double red[kLossThreads / 32];
  const int b = blockIdx.y;
  const int i = a.batch_off + b;
  const int q = blockIdx.x * kLossThreads + threadIdx.x;
  const int j = batch_pos(a, i);                     // uniform over the block
  if (j < 0) {
    if (la.loss_part && threadIdx.x == 0) la.loss_part[(long long)i * (FF / kLossThreads) + blockIdx.x] = 0.0;
    if (la.sig_part && threadIdx.x == 0) la.sig_part[(long long)i * (FF / kLossThreads) + blockIdx.x] = 0.0;
    if (la.D) la.D[(long long)b * FF + q] = 0.f;
    return;
  }
  const float* Ip = la.Ipart + (long long)b * a.G * FF;
  float Is = 0.f, Ib = 0.f;                          // field part and background part of the prediction
  bool valid = true;
  if (la.remap) {
    const int u = la.tap_base[q];
    valid = u >= 0;
    if (valid) {
      const float2 w = la.tap_w[q];
      const float i00 = model_I(Ip, nullptr, a.G, FF, u), i01 = model_I(Ip, nullptr, a.G, FF, u + 1);
      const float i10 = model_I(Ip, nullptr, a.G, FF, u + F), i11 = model_I(Ip, nullptr, a.G, FF, u + F + 1);
      Is = (1.f - w.x) * ((1.f - w.y) * i00 + w.y * i01) + w.x * ((1.f - w.y) * i10 + w.y * i11);
      if (la.bg) {
        const float b00 = __ldg(la.bg + u), b01 = __ldg(la.bg + u + 1);
        const float b10 = __ldg(la.bg + u + F), b11 = __ldg(la.bg + u + F + 1);
        Ib = (1.f - w.x) * ((1.f - w.y) * b00 + w.y * b01) + w.x * ((1.f - w.y) * b10 + w.y * b11);
      }
    }
  } else {
    Is = model_I(Ip, nullptr, a.G, FF, q);
    if (la.bg) Ib = __ldg(la.bg + q);
  }
  const float Ic = Is + Ib;
  if (la.I_pred) la.I_pred[(long long)j * FF + q] = valid ? Ic : 0.f;
  double term = 0.0, sterm = 0.0;
  if (la.D || la.loss_part) {
    bool use = valid;
    if (la.mask) use = use && (la.mask[(la.mask_per_frame ? (long long)j * FF : 0) + q] != 0);
    float d = 0.f;
    if (use) {
      const float Ih = __ldg(la.Imeas + (long long)j * FF + q);
      const float Ie = Ic + la.eps;
      if (la.loss_kind == 0) {
        const float se = sqrtf(Ie), diff = se - sqrtf(Ih);
        term = (double)(diff * diff);
        d = diff / se;
      } else {
        term = (double)poisson_term(Ie, Ih);
        d = (Ie - Ih) / Ie;
      }
    }
    if (la.D) la.D[(long long)b * FF + q] = d;
    sterm = (double)(d * Is);
  }
  if (la.sig_part) {                                  // before the loss reduction reuses red
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sterm += __shfl_down_sync(0xffffffffu, sterm, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sterm;
    __syncthreads();
    if (threadIdx.x == 0) {
      double sum = 0.0;
      for (int wi = 0; wi < kLossThreads / 32; ++wi) sum += red[wi];
      la.sig_part[(long long)i * (FF / kLossThreads) + blockIdx.x] = sum;
    }
    __syncthreads();
  }
  if (la.loss_part) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) term += __shfl_down_sync(0xffffffffu, term, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = term;
    __syncthreads();
    if (threadIdx.x == 0) {
      double sum = 0.0;
      for (int wi = 0; wi < kLossThreads / 32; ++wi) sum += red[wi];
      la.loss_part[(long long)i * (FF / kLossThreads) + blockIdx.x] = sum;
    }
  }
}

// ---------------------------------------------------------------------------------------
// R^T of the tilted-plane remap: G[b][u] = sum over the camera pixels q that sample model
// pixel u of w_uq D[b][q] (CSR rows in increasing q: a fixed order).   grid (F*F/256, nb)
// ---------------------------------------------------------------------------------------
struct AdjArgs {
  const float* D;                // [B][F][F] camera grid
  const int32_t* rt_ptr;         // [F*F+1] CSR of R^T over centred model pixels (remap only)
  const int32_t* rt_idx;         // camera pixel of each entry
  const float* rt_w;             // weight of each entry
  float* Gt;                     // [B][F][F] R^T D on the model grid (remap only)
  int remap;
};

template <int F>
__global__ void __launch_bounds__(256)
k_remap_adj(KArgs a, AdjArgs aa) {
  pdl_wait();
  pdl_trigger();
  constexpr int FF = F * F;
  const int u = blockIdx.x * 256 + threadIdx.x;
  const int b = blockIdx.y;
  const int e0 = __ldg(aa.rt_ptr + u), e1 = __ldg(aa.rt_ptr + u + 1);
  const float* Db = aa.D + (long long)b * FF;
  float gv = 0.f;
  for (int e = e0; e < e1; ++e) gv = fmaf(__ldg(aa.rt_w + e), Db[__ldg(aa.rt_idx + e)], gv);
  aa.Gt[(long long)b * FF + u] = gv;
}

// Background gradient, Eq. 1 (N is added before the remap): acc[u] += sum over the batch of
// G[b][u] (R^T D, or D without the remap), in batch order.   grid (F*F/256)
template <int F>
__global__ void __launch_bounds__(256)
k_bg_accum(const float* __restrict__ G, int nb, float* __restrict__ acc) {
  pdl_wait();
  pdl_trigger();
  constexpr int FF = F * F;
  const int u = blockIdx.x * 256 + threadIdx.x;
  float s = acc[u];
  for (int b = 0; b < nb; ++b) s += G[(long long)b * FF + u];
  acc[u] = s;
}

// ---------------------------------------------------------------------------------------
// adjoint column pass: (2/F) G Psi, inverse column DFT.   grid (F/W, G, nb)
// ---------------------------------------------------------------------------------------
template <int F, bool STORE>
__global__ void __launch_bounds__(ColCfg<F>::threads)
k_col_adj(float2* __restrict__ S, KArgs a, AdjArgs aa) {
  pdl_wait();
  pdl_trigger();
  constexpr int N1 = FftShape<F>::N1, N2 = FftShape<F>::N2, W = ColCfg<F>::W;
  extern __shared__ float2 smem[];
  float* gt = reinterpret_cast<float*>(smem + W * Xch<F>::region_cols);   // [F][W]
  const int c = threadIdx.x % W, t = threadIdx.x / W;
  const int col0 = blockIdx.x * W;
  const int g = blockIdx.y, b = blockIdx.z;
  const float* Gb = (aa.remap ? aa.Gt : aa.D) + (long long)b * F * F;
  const float scale = 2.0f / (float)F;
  for (int e = threadIdx.x; e < F * W; e += blockDim.x) {
    const int k = e / W, ce = e % W;
    const int u = ((k + F / 2) & (F - 1)) * F + ((col0 + ce + F / 2) & (F - 1));
    gt[k * W + ce] = Gb[u] * scale;
  }
  __syncthreads();
  const int col = col0 + c;
  const int m0 = g * a.MG, m1 = min(a.chunk_len, m0 + a.MG);
  const float inv = 1.0f / (float)F;
  for (int cm = m0; cm < m1; ++cm) {
    float2* base = S + ((long long)b * a.C + cm) * F * F + col;
    float2 v[N2];
    if (STORE) {
#pragma unroll
      for (int sl = 0; sl < N2; ++sl) v[sl] = base[(long long)idxO<F>(t, sl) * F];
    } else {
#pragma unroll
      for (int n2 = 0; n2 < N2; ++n2) v[n2] = base[(long long)(t + N1 * n2) * F];
      fft_fwd_I2O<F>(v, t, smem + c * Xch<F>::region_cols, a.tw, BlockSync{});
#pragma unroll
      for (int sl = 0; sl < N2; ++sl) v[sl] = cscale(v[sl], inv);
    }
#pragma unroll
    for (int sl = 0; sl < N2; ++sl) v[sl] = cscale(v[sl], gt[idxO<F>(t, sl) * W + c]);
    fft_inv_O2I<F>(v, t, smem + c * Xch<F>::region_cols, a.tw, BlockSync{});
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) base[(long long)(t + N1 * n2) * F] = v[n2];
  }
}

// grid (F/W, G, nb); same results as k_col_adj
template <int F, bool STORE>
__global__ void __launch_bounds__(ColCfg<F>::threads)
k_col_adj_tma(const __grid_constant__ CUtensorMap map, float2* __restrict__ S, KArgs a, AdjArgs aa) {
  pdl_wait();
  pdl_trigger();
  constexpr int N1 = FftShape<F>::N1, N2 = FftShape<F>::N2, W = ColCfg<F>::W;
  extern __shared__ __align__(128) float2 smem[];
  float2* stage = smem;
  float2* xch = smem + F * W;
  uint64_t* bar = reinterpret_cast<uint64_t*>(xch + W * Xch<F>::region_cols);
  float* gt = reinterpret_cast<float*>(bar + 2);                    // [F][W]
  const int c = threadIdx.x % W, t = threadIdx.x / W;
  const int col0 = blockIdx.x * W, col = col0 + c;
  const int g = blockIdx.y, b = blockIdx.z;
  const int m0 = g * a.MG, m1 = min(a.chunk_len, m0 + a.MG);
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && m0 < m1) col_tma_issue<F>(stage, &map, col0, ((long long)b * a.C + m0) * F, bar);
  const float* Gb = (aa.remap ? aa.Gt : aa.D) + (long long)b * F * F;
  const float scale = 2.0f / (float)F;
  for (int e = threadIdx.x; e < F * W; e += blockDim.x) {
    const int k = e / W, ce = e % W;
    const int u = ((k + F / 2) & (F - 1)) * F + ((col0 + ce + F / 2) & (F - 1));
    gt[k * W + ce] = Gb[u] * scale;
  }
  __syncthreads();
  const float inv = 1.0f / (float)F;
  uint32_t phase = 0;
  bool ok = true;
  for (int cm = m0; cm < m1; ++cm) {
    ok = __syncthreads_and(mbar_wait_bounded(bar, phase, a.status));
    if (!ok) break;
    phase ^= 1;
    float2 v[N2];
    if (STORE) {
#pragma unroll
      for (int sl = 0; sl < N2; ++sl) v[sl] = stage[idxO<F>(t, sl) * W + c];
    } else {
#pragma unroll
      for (int n2 = 0; n2 < N2; ++n2) v[n2] = stage[(t + N1 * n2) * W + c];
    }
    __syncthreads();                           // the stage is free for the next mode
    if (threadIdx.x == 0 && cm + 1 < m1) col_tma_issue<F>(stage, &map, col0, ((long long)b * a.C + cm + 1) * F, bar);
    if (!STORE) {
      fft_fwd_I2O<F>(v, t, xch + c * Xch<F>::region_cols, a.tw, BlockSync{});
#pragma unroll
      for (int sl = 0; sl < N2; ++sl) v[sl] = cscale(v[sl], inv);
    }
#pragma unroll
    for (int sl = 0; sl < N2; ++sl) v[sl] = cscale(v[sl], gt[idxO<F>(t, sl) * W + c]);
    fft_inv_O2I<F>(v, t, xch + c * Xch<F>::region_cols, a.tw, BlockSync{});
    float2* base = S + ((long long)b * a.C + cm) * F * F + col;
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) base[(long long)(t + N1 * n2) * F] = v[n2];
  }
  if (!ok && threadIdx.x == 0) mbar_wait_bounded(bar, phase, a.status);
}

// ---------------------------------------------------------------------------------------
// adjoint row pass: chi = dL/dpsi; probe gradient summed over the batch; object-gradient
// contributions conj(sigma P) chi left in S (or, with ATOMIC, added to grad O with FP32
// atomics).  The batch is split over kAdjSlots groups of
// warps (slot s takes positions s, s + kAdjSlots, ...); their probe-gradient sums are added
// in slot order through shared memory, so the result does not depend on timing.
// grid (F/RPB, chunk_len)
// ---------------------------------------------------------------------------------------
constexpr int kAdjSlots = 4;
template <int F> struct RowAdjCfg {
  static constexpr int T = FftShape<F>::N1;
  static constexpr int RPB = 256 / (T * kAdjSlots);   // rows per block
  static constexpr int threads = RPB * T * kAdjSlots;
  static constexpr int vecs = RPB * kAdjSlots;
  static constexpr int smem_xch = vecs * Xch<F>::region_rows * (int)sizeof(float2);
  static constexpr int smem_red = (kAdjSlots - 1) * RPB * F * (int)sizeof(float2);
  static constexpr int smem = smem_xch > smem_red ? smem_xch : smem_red;
};

template <int F, bool ATOMIC>
__global__ void __launch_bounds__(RowAdjCfg<F>::threads, (F <= 256 ? 2 : 1))
k_row_adj(const float2* __restrict__ O, const float2* __restrict__ P, float2* __restrict__ S,
          float2* __restrict__ gP, float2* __restrict__ gO, KArgs a) {
  pdl_wait();
  pdl_trigger();
  constexpr int N1 = FftShape<F>::N1, N2 = FftShape<F>::N2, T = RowAdjCfg<F>::T, RPB = RowAdjCfg<F>::RPB;
  extern __shared__ float2 smem[];
  __shared__ int2 spos[kMaxB];
  __shared__ float ssig[kMaxB];
  const int vec = threadIdx.x / T, t = threadIdx.x % T;
  const int slot = vec / RPB, rr = vec % RPB;
  const int r = blockIdx.x * RPB + rr;
  const int cm = blockIdx.y;
  const int mode = a.chunk_base + cm;
  const int l = mode / a.M;
  stage_batch(a, l, spos, ssig);
  const float2* Prow = P + ((long long)mode * F + r) * F;
  const float2* Ol = O + a.obj_off[l];
  const int Wl = a.obj_w[l];
  float2 acc[N2];
#pragma unroll
  for (int n2 = 0; n2 < N2; ++n2) acc[n2] = make_float2(0.f, 0.f);
  for (int b = slot; b < a.nb; b += kAdjSlots) {
    const int2 yx = spos[b];
    if (yx.x < 0) continue;                           // uniform over the slot's warps
    const float s = ssig[b];
    float2* row = S + (((long long)b * a.C + cm) * F + r) * F;
    const float2* Orow = Ol + (long long)(yx.x + r) * Wl + yx.y;
    float2 v[N2], p[N2];
#pragma unroll
    for (int sl = 0; sl < N2; ++sl) v[sl] = row[idxO<F>(t, sl)];
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) p[n2] = __ldg(Orow + t + N1 * n2);
    fft_inv_O2I<F>(v, t, smem + vec * Xch<F>::region_rows, a.tw, WarpSync{});
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) {
      const float2 gp = cconjmul(p[n2], v[n2]);     // conj(p) chi
      acc[n2].x = fmaf(s, gp.x, acc[n2].x);
      acc[n2].y = fmaf(s, gp.y, acc[n2].y);
      const float2 go = cscale(cconjmul(__ldg(Prow + t + N1 * n2), v[n2]), s);   // conj(sigma P) chi
      if (ATOMIC)
        atomicAdd(gO + a.obj_off[l] + (long long)(yx.x + r) * Wl + yx.y + t + N1 * n2, go);
      else
        row[t + N1 * n2] = go;
    }
  }
  // slots 1.. hand their sums to slot 0 through shared memory (the exchange area is free now)
  __syncthreads();
  float2* red = smem;                                 // [kAdjSlots-1][RPB][F]
  if (slot > 0) {
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) red[((slot - 1) * RPB + rr) * F + t + N1 * n2] = acc[n2];
  }
  __syncthreads();
  if (slot == 0) {
    float2* g = gP + ((long long)mode * F + r) * F;
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) {
      const int c = t + N1 * n2;
      float2 sum = acc[n2];
      for (int s2 = 1; s2 < kAdjSlots; ++s2) sum = cadd(sum, red[((s2 - 1) * RPB + rr) * F + c]);
      g[c] = cadd(g[c], sum);
    }
  }
}

// ---------------------------------------------------------------------------------------
// object gradient: one block per 32x32 tile of grad O_l inside the batch's bounding box; it
// adds, in a fixed order, every overlapping patch contribution of the chunk's modes.
// grid (tiles of the largest box, L)
// ---------------------------------------------------------------------------------------
template <int F>
__global__ void __launch_bounds__(256)
k_obj_grad(const float2* __restrict__ S, float2* __restrict__ gO, KArgs a) {
  pdl_wait();
  pdl_trigger();
  __shared__ int2 spos[kMaxB];
  __shared__ float ssig[kMaxB];
  const int l = blockIdx.y;
  const int mlo = max(a.chunk_base, l * a.M), mhi = min(a.chunk_base + a.chunk_len, (l + 1) * a.M);
  if (mlo >= mhi) return;                             // uniform over the block
  const int by0 = a.box[l][0], bx0 = a.box[l][1];
  const int ntx = (a.box[l][3] - bx0 + kTile - 1) / kTile;
  const int nty = (a.box[l][2] - by0 + kTile - 1) / kTile;
  if ((int)blockIdx.x >= ntx * nty) return;          // uniform over the block
  stage_batch(a, l, spos, ssig);
  const int oy0 = by0 + ((int)blockIdx.x / ntx) * kTile, ox0 = bx0 + ((int)blockIdx.x % ntx) * kTile;
  const int H = a.obj_h[l], Wd = a.obj_w[l];
  const int tx = threadIdx.x % kTile, ty0 = threadIdx.x / kTile;   // 8 row slots
  const int ox = ox0 + tx;
  float2 acc[kTile / 8];
#pragma unroll
  for (int k = 0; k < kTile / 8; ++k) acc[k] = make_float2(0.f, 0.f);
  for (int b = 0; b < a.nb; ++b) {
    const int y = spos[b].x, x = spos[b].y;
    if (y < 0 || y >= oy0 + kTile || y + F <= oy0 || x >= ox0 + kTile || x + F <= ox0) continue;
    const bool in_x = ox >= x && ox < x + F;
    const float2* src = S + ((long long)b * a.C + (mlo - a.chunk_base)) * F * F + (ox - x);
    for (int m0 = mlo; m0 < mhi; m0 += 4, src += 4ll * F * F) {
      float2 v[4][kTile / 8];
#pragma unroll
      for (int mm = 0; mm < 4; ++mm)
#pragma unroll
        for (int k = 0; k < kTile / 8; ++k) {
          const int oy = oy0 + ty0 + 8 * k;
          const bool ok = m0 + mm < mhi && in_x && oy >= y && oy < y + F;
          v[mm][k] = ok ? src[(long long)mm * F * F + (long long)(oy - y) * F] : make_float2(0.f, 0.f);
        }
#pragma unroll
      for (int mm = 0; mm < 4; ++mm)
#pragma unroll
        for (int k = 0; k < kTile / 8; ++k) acc[k] = cadd(acc[k], v[mm][k]);
    }
  }
  float2* g = gO + a.obj_off[l];
#pragma unroll
  for (int k = 0; k < kTile / 8; ++k) {
    const int oy = oy0 + ty0 + 8 * k;
    if (oy < H && ox < Wd) {
      float2* p = g + (long long)oy * Wd + ox;
      *p = cadd(*p, acc[k]);
    }
  }
}

// ---------------------------------------------------------------------------------------
// loss reduction and Adam (defined in ptycho_capi.cu)
// ---------------------------------------------------------------------------------------
__global__ void k_loss_reduce(const double* __restrict__ part, long long n, double* out);
__global__ void k_sigma_grad(const int32_t* __restrict__ bidx, int nbatch, int J, const double* __restrict__ part,
                             int nblk, const float* __restrict__ sigma, float* __restrict__ g);
__global__ void k_sum_sets(const float* __restrict__ acc, int nsets, long long n, float* __restrict__ out);
__global__ void k_tick(int* t);
__global__ void k_adam_dev(float* __restrict__ theta, const float* __restrict__ grad, float* __restrict__ m,
                           float* __restrict__ v, long long n, float lr, float b1, float b2, float eps,
                           const int* __restrict__ t_dev);
__global__ void k_adam(float* __restrict__ theta, const float* __restrict__ grad, float* __restrict__ m,
                       float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1,
                       float c2);

}  // namespace ptycho
