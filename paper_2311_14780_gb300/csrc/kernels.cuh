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
constexpr int kLossPx = 4;       // camera pixels per thread in the loss kernel (a multiple of 4)
template <int F> __host__ __device__ constexpr int loss_blocks() { return F * F / (kLossThreads * kLossPx); }
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
  const float2* patch;           // [B][L][F][F] object patches shifted by fractional offsets, or null
                                 // (the row passes then gather the patch from O at the integer position)
};

// Programmatic dependent launch: the pipeline launches each kernel so that it may start
// while the previous kernel of its stream finishes.  pdl_wait() blocks until that kernel
// has completed and its writes are visible (a no-op for an ordinary launch); every pipeline
// kernel calls it before touching global memory.  pdl_trigger() lets the next kernel start
// launching its blocks.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" :::); }

// Whether launch_pdl asks for programmatic stream serialisation (per host thread; each
// compute call sets it from its plan's flags).
inline bool& pdl_enabled() {
  static thread_local bool on = true;
  return on;
}

// Launch with programmatic stream serialisation (see pdl_wait above).
template <typename... KP, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KP...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KP>(args)...);
}

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
// the row DFT (first half of f4).   block index (row block, l, position b)
// ---------------------------------------------------------------------------------------
template <int F>
__device__ __forceinline__ void row_fwd_body(const float2* __restrict__ O, const float2* __restrict__ P, float2* __restrict__ S, const KArgs& a, const uint3 bid) {
  constexpr int N1 = FftShape<F>::N1, N2 = FftShape<F>::N2, T = RowCfg<F>::T;
  extern __shared__ float2 smem[];
  const int vec = threadIdx.x / T, t = threadIdx.x % T;
  const int r = bid.x * RowCfg<F>::RPB + vec;
  const int l = bid.y, b = bid.z;
  const int mlo = max(a.chunk_base, l * a.M), mhi = min(a.chunk_base + a.chunk_len, (l + 1) * a.M);
  if (mlo >= mhi) return;                             // uniform over the block
  const int j = batch_pos(a, a.batch_off + b);
  if (j < 0) return;                                  // uniform over the block
  const int y = a.pos[(l * a.J + j) * 2], x = a.pos[(l * a.J + j) * 2 + 1];
  const float s = sigma_of(a, j);
  const float2* Orow = a.patch ? a.patch + (((long long)b * a.L + l) * F + r) * F
                               : O + a.obj_off[l] + (long long)(y + r) * a.obj_w[l] + x;
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

// grid (nb, F/RPB, L): the positions of a batch vary fastest, so that the blocks running at the
// same time share probe rows in L2 (the probes of all modes can exceed the L2: 120 MB at 512^2
// with 6 wavelengths x 10 modes)
template <int F>
__global__ void __launch_bounds__(RowCfg<F>::threads)
k_row_fwd(const float2* __restrict__ O, const float2* __restrict__ P, float2* __restrict__ S, KArgs a) {
  pdl_wait();
  pdl_trigger();
  row_fwd_body<F>(O, P, S, a, make_uint3(blockIdx.y, blockIdx.z, blockIdx.x));
}

// ---------------------------------------------------------------------------------------
// forward column pass: column DFT (second half of f4), |Psi|^2 summed over a mode group
// grid (F/W, G, nb)
// ---------------------------------------------------------------------------------------
template <int F, bool STORE>
__device__ __forceinline__ void col_fwd_body(float2* __restrict__ S, float* __restrict__ Ipart, const KArgs& a, int first_chunk, const uint3 bid) {
  constexpr int N1 = FftShape<F>::N1, N2 = FftShape<F>::N2, W = ColCfg<F>::W;
  extern __shared__ float2 smem[];
  const int c = threadIdx.x % W, t = threadIdx.x / W;
  const int col = bid.x * W + c;
  const int g = bid.y, b = bid.z;
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

template <int F, bool STORE>
__global__ void __launch_bounds__(ColCfg<F>::threads)
k_col_fwd(float2* __restrict__ S, float* __restrict__ Ipart, KArgs a, int first_chunk) {
  pdl_wait();
  pdl_trigger();
  col_fwd_body<F, STORE>(S, Ipart, a, first_chunk, blockIdx);
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
  // + 128: the stage is placed on a 128-byte boundary inside the dynamic shared memory (whose
  // start moves with the kernel's static shared variables)
  static constexpr int smem_fwd = stage_bytes + ColCfg<F>::smem_xch + 16 + 128;
  static constexpr int smem_adj = smem_fwd + F * W * (int)sizeof(float);
};

// The first 128-byte-aligned address (in the shared window) at or after p: the destination of
// a bulk tensor copy must be 128-byte aligned.
__device__ __forceinline__ float2* align_tma_stage(unsigned char* p) {
  const uint32_t pad = (128u - (smem_addr(p) & 127u)) & 127u;
  return reinterpret_cast<float2*>(p + pad);
}

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
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float2* smem = align_tma_stage(smem_raw);
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
// Staged column passes (one mode chunk holding every mode, one group: G = 1).  A block
// takes W columns of one position and runs over all its modes; the W x F column block of
// the next mode is copied into shared memory (cp.async, double-buffered) while the current
// one is transformed, so a block always has one mode's data in flight.
// grid (F/W, nb), block W*T
// ---------------------------------------------------------------------------------------
template <int F, int WN = 0> struct ColSCfg {
  static constexpr int T = FftShape<F>::N1;
  static constexpr int W = WN > 0 ? WN : (F >= 256 ? 8 : 128 / T);   // columns per block
  static constexpr int threads = W * T;
  static constexpr int stage = F * W;                // float2 per stage
  // exchange-region stride: a warp holds columns c < W and 32/W threads t of each; with the
  // stride = 32/W (mod 16) the offsets c*R + t fall on every 8-byte bank pair exactly twice
  // (two wavefronts, the minimum for 32 x 8 bytes); W >= 32 only needs an odd stride
  static constexpr int R = W >= 32 ? (Xch<F>::base | 1)
                                   : Xch<F>::base + (((32 / W) - Xch<F>::base) % 16 + 16) % 16;
  static constexpr int smem_fwd = (2 * stage + W * R) * (int)sizeof(float2);
  static constexpr int smem_adj = smem_fwd + F * W * (int)sizeof(float);
};

// Issue the copies of mode slot cm's W x F column block (from column col0) into dst.
template <int F, int WN>
__device__ __forceinline__ void col_prefetch(const float2* __restrict__ Sb, int cm, int col0, float2* dst) {
  constexpr int W = ColSCfg<F, WN>::W, CH = F * W / 2;  // 16-byte chunks
  const float2* src = Sb + (long long)cm * F * F + col0;
  for (int e = threadIdx.x; e < CH; e += ColSCfg<F, WN>::threads) {
    const int row = e / (W / 2), cc = (e % (W / 2)) * 2;
    cp_async16(dst + row * W + cc, src + (long long)row * F + cc);
  }
  cp_async_commit();
}

template <int F, bool STORE, int WN>
__global__ void __launch_bounds__(ColSCfg<F, WN>::threads)
k_col_fwd_s(float2* __restrict__ S, float* __restrict__ Ipart, KArgs a) {
  pdl_wait();
  pdl_trigger();
  constexpr int N1 = FftShape<F>::N1, N2 = FftShape<F>::N2, W = ColSCfg<F, WN>::W, ST = ColSCfg<F, WN>::stage;
  extern __shared__ __align__(16) float2 smem[];
  float2* stage = smem;                               // [2][F][W]
  float2* xch = smem + 2 * ST;
  const int c = threadIdx.x % W, t = threadIdx.x / W;
  const int col0 = blockIdx.x * W, col = col0 + c;
  const int b = blockIdx.y;
  const int nm = a.chunk_len;
  float2* Sb = S + (long long)b * a.C * F * F;
  float acc[N2];
#pragma unroll
  for (int i = 0; i < N2; ++i) acc[i] = 0.f;
  const float inv = 1.0f / (float)F;
  if (nm > 0) col_prefetch<F, WN>(Sb, 0, col0, stage);
  for (int cm = 0; cm < nm; ++cm) {
    const float2* cur = stage + (cm & 1) * ST;
    if (cm + 1 < nm) {
      col_prefetch<F, WN>(Sb, cm + 1, col0, stage + ((cm + 1) & 1) * ST);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    float2 v[N2];
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) v[n2] = cur[(t + N1 * n2) * W + c];
    fft_fwd_I2O<F>(v, t, xch + c * ColSCfg<F, WN>::R, a.tw, BlockSync{});   // its first barrier frees cur
    float2* base = Sb + (long long)cm * F * F + col;
#pragma unroll
    for (int sl = 0; sl < N2; ++sl) {
      acc[sl] = fmaf(v[sl].x, v[sl].x, fmaf(v[sl].y, v[sl].y, acc[sl]));
      if (STORE) base[(long long)idxO<F>(t, sl) * F] = cscale(v[sl], inv);
    }
  }
  float* dst = Ipart + (long long)b * F * F;
  const int cc = (col + F / 2) & (F - 1);
#pragma unroll
  for (int sl = 0; sl < N2; ++sl) {
    const int rc = (idxO<F>(t, sl) + F / 2) & (F - 1);
    dst[rc * F + cc] = acc[sl] * (inv * inv);
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
  int loss_kind;                 // 0 amplitude, 1 Poisson, 2 mixed Poisson-Gaussian
  float read_var;                // s2 of the mixed loss
  float* D;                      // [B][F][F] mask * dL/dI (camera grid), null if not needed
  double* loss_part;             // [nbatch][loss_blocks] or null
  double* sig_part;              // [nbatch][loss_blocks] sums of D * (remapped sum |Psi|^2), or null
  float* I_pred;                 // [J][F][F] or null
  int remap;
  int Gsum;                      // intensity slices (mode groups) to add
  const float2* tap_dz;          // [F*F] d(row, col index of the taps)/dz (remap only)
  double* z_part;                // [nbatch][loss_blocks] sums of D * d(R I)/dz, or null
};

// Model intensity at pixel u: the G intensity slices added in slice order (small G unrolled; the
// rounding is that of the loop, which starts from 0 + slice 0).
__device__ __forceinline__ float model_I(const float* Ip, int G, int FF, int u) {
  const float* p = Ip + u;
  switch (G) {
    case 1: return p[0];
    case 2: return p[0] + p[FF];
    case 3: return (p[0] + p[FF]) + p[2 * FF];
    case 4: return ((p[0] + p[FF]) + p[2 * FF]) + p[3 * FF];
    default: {
      float s = 0.f;
      for (int g = 0; g < G; ++g, p += FF) s += *p;
      return s;
    }
  }
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

// Camera-grid prediction of one pixel q (remap: bilinear in the four model taps of q).
// Is is the field part, Ib the background part; valid = false outside the remap's grid.
// With the remap, srow / scol are the slopes of the bilinear interpolant of the full model
// intensity (field + background) along the row and column fractions of the taps.
template <int F>
__device__ __forceinline__ void predict_pixel(const LossArgs& la, const float* Ip, int G, int q, int tb, float2 w,
                                              float& Is, float& Ib, bool& valid, float& srow, float& scol) {
  constexpr int FF = F * F;
  Is = 0.f;
  Ib = 0.f;
  srow = scol = 0.f;
  valid = true;
  if (la.remap) {
    valid = tb >= 0;
    if (!valid) return;
    float i00, i01, i10, i11;
    if (G == 1) {                                     // one intensity slice (uniform branch)
      i00 = Ip[tb];
      i01 = Ip[tb + 1];
      i10 = Ip[tb + F];
      i11 = Ip[tb + F + 1];
    } else {
      i00 = model_I(Ip, G, FF, tb);
      i01 = model_I(Ip, G, FF, tb + 1);
      i10 = model_I(Ip, G, FF, tb + F);
      i11 = model_I(Ip, G, FF, tb + F + 1);
    }
    Is = (1.f - w.x) * ((1.f - w.y) * i00 + w.y * i01) + w.x * ((1.f - w.y) * i10 + w.y * i11);
    if (la.bg) {
      const float b00 = __ldg(la.bg + tb), b01 = __ldg(la.bg + tb + 1);
      const float b10 = __ldg(la.bg + tb + F), b11 = __ldg(la.bg + tb + F + 1);
      Ib = (1.f - w.x) * ((1.f - w.y) * b00 + w.y * b01) + w.x * ((1.f - w.y) * b10 + w.y * b11);
      i00 += b00; i01 += b01; i10 += b10; i11 += b11;
    }
    srow = ((1.f - w.y) * i10 + w.y * i11) - ((1.f - w.y) * i00 + w.y * i01);
    scol = (1.f - w.x) * (i01 - i00) + w.x * (i11 - i10);
  } else {
    Is = model_I(Ip, G, FF, q);
    if (la.bg) Ib = __ldg(la.bg + q);
  }
}

// Compensated FP32 sums ("double-float": value = hi + lo).  Knuth's TwoSum gives the exact
// rounding error of an addition, so the pair carries about twice the FP32 mantissa without
// FP64 arithmetic (slow on this part).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void df_add(float& hi, float& lo, float x) {
  float s, e;
  two_sum(hi, x, s, e);
  hi = s;
  lo += e;
}
__device__ __forceinline__ void df_add_df(float& hi, float& lo, float bhi, float blo) {
  float s, e;
  two_sum(hi, bhi, s, e);
  e += lo + blo;
  hi = s + e;                                    // renormalise (Fast2Sum, |s| >= |e|)
  lo = e - (hi - s);
}
// Warp-tree sum of a double-float (fixed pairing: the result does not depend on timing).
__device__ __forceinline__ void df_warp_sum(float& hi, float& lo) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float bh = __shfl_down_sync(0xffffffffu, hi, o), bl = __shfl_down_sync(0xffffffffu, lo, o);
    df_add_df(hi, lo, bh, bl);
  }
}

// Each thread takes kLossPx consecutive camera pixels; the loss terms and the sigma-gradient
// terms of a block are summed as double-floats (per thread, then a warp tree) and the eight
// warp sums in FP64, in a fixed order, into one partial per (call entry, block).
// grid (F*F/(kLossThreads*kLossPx), nb)
template <int F>
__device__ __forceinline__ void loss_body(const KArgs& a, const LossArgs& la, const uint3 bid) {
  constexpr int FF = F * F, NB = loss_blocks<F>();
  __shared__ float red[6][kLossThreads / 32];
  const int b = bid.y;
  const int i = a.batch_off + b;
  const int q0 = (bid.x * kLossThreads + threadIdx.x) * kLossPx;
  const int j = batch_pos(a, i);                     // uniform over the block
  if (j < 0) {
    if (la.loss_part && threadIdx.x == 0) la.loss_part[(long long)i * NB + bid.x] = 0.0;
    if (la.sig_part && threadIdx.x == 0) la.sig_part[(long long)i * NB + bid.x] = 0.0;
    if (la.z_part && threadIdx.x == 0) la.z_part[(long long)i * NB + bid.x] = 0.0;
    if (la.D)
#pragma unroll
      for (int k = 0; k < kLossPx; k += 4)
        *reinterpret_cast<float4*>(la.D + (long long)b * FF + q0 + k) = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  const float* Ip = la.Ipart + (long long)b * a.G * FF;
  int tb[kLossPx];
  float2 tw[kLossPx];
  if (la.remap) {
#pragma unroll
    for (int k = 0; k < kLossPx; k += 4) {
      const int4 t4 = *reinterpret_cast<const int4*>(la.tap_base + q0 + k);
      const float4 w01 = *reinterpret_cast<const float4*>(la.tap_w + q0 + k);
      const float4 w23 = *reinterpret_cast<const float4*>(la.tap_w + q0 + k + 2);
      tb[k] = t4.x; tb[k + 1] = t4.y; tb[k + 2] = t4.z; tb[k + 3] = t4.w;
      tw[k] = make_float2(w01.x, w01.y); tw[k + 1] = make_float2(w01.z, w01.w);
      tw[k + 2] = make_float2(w23.x, w23.y); tw[k + 3] = make_float2(w23.z, w23.w);
    }
  } else {
#pragma unroll
    for (int k = 0; k < kLossPx; ++k) { tb[k] = 0; tw[k] = make_float2(0.f, 0.f); }
  }
  float d[kLossPx];
  float th = 0.f, tl = 0.f, sh = 0.f, sl = 0.f;   // double-float sums of the loss and sigma terms
  float zh = 0.f, zl = 0.f;                       // and of the z terms
#pragma unroll
  for (int k = 0; k < kLossPx; ++k) {
    const int q = q0 + k;
    float Is, Ib, srow, scol;
    bool valid;
    predict_pixel<F>(la, Ip, la.Gsum, q, tb[k], tw[k], Is, Ib, valid, srow, scol);
    const float Ic = Is + Ib;
    if (la.I_pred) la.I_pred[(long long)j * FF + q] = valid ? Ic : 0.f;
    d[k] = 0.f;
    if (la.D || la.loss_part) {
      bool use = valid;
      if (la.mask) use = use && (la.mask[(la.mask_per_frame ? (long long)j * FF : 0) + q] != 0);
      if (use) {
        float Ih = __ldg(la.Imeas + (long long)j * FF + q);
        float Ie = Ic + la.eps;
        if (la.loss_kind == 2) {                       // shifted Poisson
          Ie += la.read_var;
          Ih = fmaxf(Ih + la.read_var, 0.f);
        }
        if (la.loss_kind == 0) {
          const float se = sqrtf(Ie), diff = se - sqrtf(Ih);
          df_add(th, tl, diff * diff);
          d[k] = __fdividef(diff, se);                 // 2 ulp: ample for a gradient
        } else {
          df_add(th, tl, poisson_term(Ie, Ih));
          d[k] = __fdividef(Ie - Ih, Ie);
        }
      }
      if (la.sig_part) df_add(sh, sl, d[k] * Is);
      if (la.z_part && d[k] != 0.f) {
        const float2 rz = __ldg(la.tap_dz + q);
        df_add(zh, zl, d[k] * fmaf(srow, rz.x, scol * rz.y));
      }
    }
  }
  if (la.D)
#pragma unroll
    for (int k = 0; k < kLossPx; k += 4)
      *reinterpret_cast<float4*>(la.D + (long long)b * FF + q0 + k) = make_float4(d[k], d[k + 1], d[k + 2], d[k + 3]);
  if (!la.loss_part && !la.sig_part && !la.z_part) return;
  if (la.loss_part) df_warp_sum(th, tl);           // each sum only when its output is requested
  if (la.sig_part) df_warp_sum(sh, sl);            // (uniform branches)
  if (la.z_part) df_warp_sum(zh, zl);
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = th;
    red[1][threadIdx.x >> 5] = tl;
    red[2][threadIdx.x >> 5] = sh;
    red[3][threadIdx.x >> 5] = sl;
    red[4][threadIdx.x >> 5] = zh;
    red[5][threadIdx.x >> 5] = zl;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double sum = 0.0;
    for (int wi = 0; wi < kLossThreads / 32; ++wi)
      sum += (double)red[2 * threadIdx.x][wi] + (double)red[2 * threadIdx.x + 1][wi];
    double* out = threadIdx.x == 0 ? la.loss_part : (threadIdx.x == 1 ? la.sig_part : la.z_part);
    if (out) out[(long long)i * NB + bid.x] = sum;
  }
}

template <int F>
__global__ void __launch_bounds__(kLossThreads)
k_loss(KArgs a, LossArgs la) {
  pdl_wait();
  pdl_trigger();
  loss_body<F>(a, la, blockIdx);
}

// ---------------------------------------------------------------------------------------
// R^T of the tilted-plane remap: G[b][u] = sum over the camera pixels q that sample model
// pixel u of w_uq D[b][q] (CSR rows in increasing q: a fixed order).
// ---------------------------------------------------------------------------------------
struct AdjArgs {
  const float* D;                // [B][F][F] camera grid
  const int32_t* rt_ptr;         // [F*F+1] CSR of R^T over centred model pixels (remap only)
  const int32_t* rt_idx;         // camera pixel of each entry
  const float* rt_w;             // weight of each entry
  float* Gt;                     // [B][F][F] R^T D on the model grid (remap only)
  int remap;
};

// One thread per model pixel u and kRtPos positions of the batch: the CSR entries of u are
// read once and the positions' D loads are independent.   grid (F*F/256, ceil(nb/kRtPos))
constexpr int kRtPos = 8;
template <int F>
__device__ __forceinline__ void remap_adj_body(const KArgs& a, const AdjArgs& aa, const uint3 bid) {
  constexpr int FF = F * F;
  const int u = bid.x * 256 + threadIdx.x;
  const int b0 = bid.y * kRtPos;
  const int nbk = min(kRtPos, a.nb - b0);
  const int e0 = __ldg(aa.rt_ptr + u), e1 = __ldg(aa.rt_ptr + u + 1);
  const float* Db = aa.D + (long long)b0 * FF;
  float gv[kRtPos];
#pragma unroll
  for (int k = 0; k < kRtPos; ++k) gv[k] = 0.f;
  for (int e = e0; e < e1; ++e) {
    const float w = __ldg(aa.rt_w + e);
    const int q = __ldg(aa.rt_idx + e);
#pragma unroll
    for (int k = 0; k < kRtPos; ++k)
      if (k < nbk) gv[k] = fmaf(w, Db[(long long)k * FF + q], gv[k]);
  }
#pragma unroll
  for (int k = 0; k < kRtPos; ++k)
    if (k < nbk) aa.Gt[(long long)(b0 + k) * FF + u] = gv[k];
}

template <int F>
__global__ void __launch_bounds__(256)
k_remap_adj(KArgs a, AdjArgs aa) {
  pdl_wait();
  pdl_trigger();
  remap_adj_body<F>(a, aa, blockIdx);
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
__device__ __forceinline__ void col_adj_body(float2* __restrict__ S, const KArgs& a, const AdjArgs& aa, const uint3 bid) {
  constexpr int N1 = FftShape<F>::N1, N2 = FftShape<F>::N2, W = ColCfg<F>::W;
  extern __shared__ float2 smem[];
  float* gt = reinterpret_cast<float*>(smem + W * Xch<F>::region_cols);   // [F][W]
  const int c = threadIdx.x % W, t = threadIdx.x / W;
  const int col0 = bid.x * W;
  const int g = bid.y, b = bid.z;
  const float* Gb = (aa.remap ? aa.Gt : aa.D) + (long long)b * F * F;
  const float scale = 2.0f / (float)F;
  for (int e = threadIdx.x; e < F * W; e += blockDim.x) {
    const int k = e / W, ce = e % W;
    const int u = ((k + F / 2) & (F - 1)) * F + ((col0 + ce + F / 2) & (F - 1));
    gt[k * W + ce] = Gb[u] * (STORE ? scale : scale / (float)F);   // recomputed Psi: the 1/F folded in
  }
  __syncthreads();
  const int col = col0 + c;
  const int m0 = g * a.MG, m1 = min(a.chunk_len, m0 + a.MG);
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
    }
#pragma unroll
    for (int sl = 0; sl < N2; ++sl) v[sl] = cscale(v[sl], gt[idxO<F>(t, sl) * W + c]);
    fft_inv_O2I<F>(v, t, smem + c * Xch<F>::region_cols, a.tw, BlockSync{});
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) base[(long long)(t + N1 * n2) * F] = v[n2];
  }
}

template <int F, bool STORE>
__global__ void __launch_bounds__(ColCfg<F>::threads)
k_col_adj(float2* __restrict__ S, KArgs a, AdjArgs aa) {
  pdl_wait();
  pdl_trigger();
  col_adj_body<F, STORE>(S, a, aa, blockIdx);
}

// The plain-load column passes compiled for two blocks per SM: at 512^2 (32 values per thread)
// they fit 128 registers without spills and measured 10 % faster than the TMA-staged passes (one
// block per SM) with one field per position; from two fields on the TMA-staged passes are faster.
// (Below 512^2 the compiler's own choice is kept: a two-block bound measured 5 % slower at 256^2.)
template <int F, bool STORE>
__global__ void __launch_bounds__(ColCfg<F>::threads, 2)
k_col_fwd_2b(float2* __restrict__ S, float* __restrict__ Ipart, KArgs a, int first_chunk) {
  pdl_wait();
  pdl_trigger();
  col_fwd_body<F, STORE>(S, Ipart, a, first_chunk, blockIdx);
}

template <int F, bool STORE>
__global__ void __launch_bounds__(ColCfg<F>::threads, 2)
k_col_adj_2b(float2* __restrict__ S, KArgs a, AdjArgs aa) {
  pdl_wait();
  pdl_trigger();
  col_adj_body<F, STORE>(S, a, aa, blockIdx);
}

// Staged adjoint column pass (see k_col_fwd_s).   grid (F/W, nb), block W*T
template <int F, bool STORE, int WN>
__global__ void __launch_bounds__(ColSCfg<F, WN>::threads)
k_col_adj_s(float2* __restrict__ S, KArgs a, AdjArgs aa) {
  pdl_wait();
  pdl_trigger();
  constexpr int N1 = FftShape<F>::N1, N2 = FftShape<F>::N2, W = ColSCfg<F, WN>::W, ST = ColSCfg<F, WN>::stage;
  extern __shared__ __align__(16) float2 smem[];
  float2* stage = smem;                               // [2][F][W]
  float2* xch = smem + 2 * ST;
  float* gt = reinterpret_cast<float*>(xch + W * ColSCfg<F, WN>::R);   // [F][W]
  const int c = threadIdx.x % W, t = threadIdx.x / W;
  const int col0 = blockIdx.x * W, col = col0 + c;
  const int b = blockIdx.y;
  const int nm = a.chunk_len;
  float2* Sb = S + (long long)b * a.C * F * F;
  if (nm > 0) col_prefetch<F, WN>(Sb, 0, col0, stage);
  const float* Gb = (aa.remap ? aa.Gt : aa.D) + (long long)b * F * F;
  const float scale = 2.0f / (float)F;
  for (int e = threadIdx.x; e < F * W; e += ColSCfg<F, WN>::threads) {
    const int k = e / W, ce = e % W;
    const int u = ((k + F / 2) & (F - 1)) * F + ((col0 + ce + F / 2) & (F - 1));
    gt[k * W + ce] = Gb[u] * scale;
  }
  const float inv = 1.0f / (float)F;
  for (int cm = 0; cm < nm; ++cm) {
    const float2* cur = stage + (cm & 1) * ST;
    if (cm + 1 < nm) {
      col_prefetch<F, WN>(Sb, cm + 1, col0, stage + ((cm + 1) & 1) * ST);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    float2 v[N2];
    if (STORE) {
#pragma unroll
      for (int sl = 0; sl < N2; ++sl) v[sl] = cur[idxO<F>(t, sl) * W + c];
    } else {
#pragma unroll
      for (int n2 = 0; n2 < N2; ++n2) v[n2] = cur[(t + N1 * n2) * W + c];
      fft_fwd_I2O<F>(v, t, xch + c * ColSCfg<F, WN>::R, a.tw, BlockSync{});
#pragma unroll
      for (int sl = 0; sl < N2; ++sl) v[sl] = cscale(v[sl], inv);
    }
#pragma unroll
    for (int sl = 0; sl < N2; ++sl) v[sl] = cscale(v[sl], gt[idxO<F>(t, sl) * W + c]);
    fft_inv_O2I<F>(v, t, xch + c * ColSCfg<F, WN>::R, a.tw, BlockSync{});   // its first barrier frees cur
    float2* base = Sb + (long long)cm * F * F + col;
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
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float2* smem = align_tma_stage(smem_raw);
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

// TMA-staged column passes with the half-size exchange (fft_*_half; F = 512) and, in the adjoint,
// the dL/dI factors read through L1/L2 instead of being staged: 99 KB of shared memory per block
// instead of 134 / 166 KB, so two 8-warp blocks fit on an SM.  Same arithmetic as
// k_col_fwd_tma / k_col_adj_tma without STORE.   grid (F/W, G, nb)
template <int F> struct ColTma2 {
  static constexpr int W = ColCfg<F>::W;
  static constexpr int smem = ColTma<F>::stage_bytes + W * XchHalf<F>::region_cols * (int)sizeof(float2) + 16 + 128;
};

template <int F>
__global__ void __launch_bounds__(ColCfg<F>::threads, 2)
k_col_fwd_tma2(const __grid_constant__ CUtensorMap map, float* __restrict__ Ipart, KArgs a, int first_chunk) {
  pdl_wait();
  pdl_trigger();
  constexpr int N1 = FftShape<F>::N1, N2 = FftShape<F>::N2, W = ColCfg<F>::W, R = XchHalf<F>::region_cols;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float2* stage = align_tma_stage(smem_raw);
  float2* xch = stage + F * W;
  uint64_t* bar = reinterpret_cast<uint64_t*>(xch + W * R);
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
    fft_fwd_I2O_half<F>(v, t, xch + c * R, a.tw, BlockSync{});
#pragma unroll
    for (int sl = 0; sl < N2; ++sl) acc[sl] = fmaf(v[sl].x, v[sl].x, fmaf(v[sl].y, v[sl].y, acc[sl]));
  }
  if (!ok) {                                   // give a lost copy a bounded chance to land, then stop
    if (threadIdx.x == 0) mbar_wait_bounded(bar, phase, a.status);
    return;
  }
  const float inv = 1.0f / (float)F;
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

template <int F>
__global__ void __launch_bounds__(ColCfg<F>::threads, 2)
k_col_adj_tma2(const __grid_constant__ CUtensorMap map, float2* __restrict__ S, KArgs a, AdjArgs aa) {
  pdl_wait();
  pdl_trigger();
  constexpr int N1 = FftShape<F>::N1, N2 = FftShape<F>::N2, W = ColCfg<F>::W, R = XchHalf<F>::region_cols;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float2* stage = align_tma_stage(smem_raw);
  float2* xch = stage + F * W;
  uint64_t* bar = reinterpret_cast<uint64_t*>(xch + W * R);
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
  // this thread's column of the dL/dI factors (DC-centred storage), read per mode through L1/L2
  const float* Gc = (aa.remap ? aa.Gt : aa.D) + (long long)b * F * F + ((col + F / 2) & (F - 1));
  const float scale = 2.0f / (float)F;
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
    fft_fwd_I2O_half<F>(v, t, xch + c * R, a.tw, BlockSync{});
#pragma unroll
    for (int sl = 0; sl < N2; ++sl) {
      const float gk = __ldg(Gc + (long long)((idxO<F>(t, sl) + F / 2) & (F - 1)) * F) * scale;
      v[sl] = cscale(cscale(v[sl], inv), gk);
    }
    fft_inv_O2I_half<F>(v, t, xch + c * R, a.tw, BlockSync{});
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
__device__ __forceinline__ void row_adj_body(const float2* __restrict__ O, const float2* __restrict__ P, float2* __restrict__ S,
          float2* __restrict__ gP, float2* __restrict__ gO, const KArgs& a, const uint3 bid) {
  constexpr int N1 = FftShape<F>::N1, N2 = FftShape<F>::N2, T = RowAdjCfg<F>::T, RPB = RowAdjCfg<F>::RPB;
  extern __shared__ float2 smem[];
  __shared__ int2 spos[kMaxB];
  __shared__ float ssig[kMaxB];
  const int vec = threadIdx.x / T, t = threadIdx.x % T;
  const int slot = vec / RPB, rr = vec % RPB;
  const int r = bid.x * RPB + rr;
  const int cm = bid.y;
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

template <int F, bool ATOMIC>
__global__ void __launch_bounds__(RowAdjCfg<F>::threads, (F <= 256 ? 2 : 1))
k_row_adj(const float2* __restrict__ O, const float2* __restrict__ P, float2* __restrict__ S,
          float2* __restrict__ gP, float2* __restrict__ gO, KArgs a) {
  pdl_wait();
  pdl_trigger();
  row_adj_body<F, ATOMIC>(O, P, S, gP, gO, a, blockIdx);
}

// ---------------------------------------------------------------------------------------
// object gradient: one block per 32x32 tile of grad O_l inside the batch's bounding box; it
// adds, in a fixed order, every overlapping patch contribution of the chunk's modes.
// grid (tiles of the largest box, L)
// ---------------------------------------------------------------------------------------
template <int F>
__device__ __forceinline__ void obj_grad_body(const float2* __restrict__ S, float2* __restrict__ gO, const KArgs& a, const uint3 bid) {
  __shared__ int2 spos[kMaxB];
  __shared__ float ssig[kMaxB];
  const int l = bid.y;
  const int mlo = max(a.chunk_base, l * a.M), mhi = min(a.chunk_base + a.chunk_len, (l + 1) * a.M);
  if (mlo >= mhi) return;                             // uniform over the block
  const int by0 = a.box[l][0], bx0 = a.box[l][1];
  const int ntx = (a.box[l][3] - bx0 + kTile - 1) / kTile;
  const int nty = (a.box[l][2] - by0 + kTile - 1) / kTile;
  if ((int)bid.x >= ntx * nty) return;          // uniform over the block
  stage_batch(a, l, spos, ssig);
  const int oy0 = by0 + ((int)bid.x / ntx) * kTile, ox0 = bx0 + ((int)bid.x % ntx) * kTile;
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

template <int F>
__global__ void __launch_bounds__(256)
k_obj_grad(const float2* __restrict__ S, float2* __restrict__ gO, KArgs a) {
  pdl_wait();
  pdl_trigger();
  obj_grad_body<F>(S, gO, a, blockIdx);
}

// ---------------------------------------------------------------------------------------
// adjoint row pass over all modes of one wavelength (one mode chunk holds every mode).
// Vector v = rr*M + m of a block takes row r = blockIdx.x*rpb + rr of probe mode (l, m).
// Per scan position of the block's split: chi = dL/dpsi by the inverse row DFT; the probe
// gradient of (l, m, r) is summed in registers over the split's positions; the object-gradient
// row sum_m conj(sigma P_lm) chi is formed in shared memory (modes added in order) and written
// to the slot of mode (l, 0), which is then the only slot the object-gradient kernel reads.
// The probe row sits in shared memory for the whole batch and the object row is read once per
// position.  Probe-gradient sums go to buffer gPs + split*gp_stride (read-modify-write).
// grid (F/rpb, L, nsplit), block T*M*rpb <= 256, dynamic smem row_adj_l_smem<F>(M, rpb)
// ---------------------------------------------------------------------------------------
constexpr int kRowAdjLSmemMax = 200 * 1024;       // dynamic shared memory cap of k_row_adj_l / k_row_fwd_l
template <int F>
__host__ __device__ constexpr int row_adj_l_smem(int M, int rpb, bool probe_l2 = false) {
  return ((probe_l2 ? 0 : M * rpb * F) + 2 * M * rpb * Xch<F>::region_rows + 2 * rpb * F) * (int)sizeof(float2);
}
// Variant of k_row_adj_l whose probe rows are read through L1/L2 instead of being held in
// shared memory: at F = 512 with 10 modes that frees 40 KB per block, and the block (at most
// kRowAdjL2Threads threads) is compiled for two blocks per SM instead of one.
constexpr int kRowAdjL2Threads = 160;

// Next position of this split after b whose index is valid, or -1 (uniform over the block).
__device__ __forceinline__ int next_pos(const int2* spos, int b, int nb, int nsplit) {
  for (int bb = b + nsplit; bb < nb; bb += nsplit)
    if (spos[bb].x >= 0) return bb;
  return -1;
}

// Copies of the rpb object rows of position (y, x) (8-byte pieces: x may be odd).
template <int F>
__device__ __forceinline__ void prefetch_orows(const float2* __restrict__ Ol, int Wl, int2 yx, int row0, int rpb,
                                               float2* dst) {
  for (int e = threadIdx.x; e < rpb * F; e += blockDim.x) {
    const int rr = e / F, c = e % F;
    cp_async8(dst + e, Ol + (long long)(yx.x + row0 + rr) * Wl + yx.y + c);
  }
}

template <int F, bool PL2>
__device__ __forceinline__ void row_adj_l_body(const float2* __restrict__ O, const float2* __restrict__ P,
                                               float2* __restrict__ S, float2* __restrict__ gPs, long long gp_stride,
                                               const KArgs& a, int rpb, int nsplit, const uint3 bid) {
  constexpr int N1 = FftShape<F>::N1, N2 = FftShape<F>::N2, T = N1, RR = Xch<F>::region_rows;
  extern __shared__ __align__(16) float2 smem[];
  __shared__ int2 spos[kMaxB];
  __shared__ float ssig[kMaxB];
  const int M = a.M, V = M * rpb;
  float2* Psm = smem;                                 // [V][F]    probe rows (not with PL2)
  float2* Sst = Psm + (PL2 ? 0 : V * F);              // [2][V][RR] scratch rows; the current buffer
                                                      //   is also the FFT exchange and the mode-sum area
  float2* Ost = Sst + 2 * V * RR;                     // [2][rpb][F] object rows
  const int vec = threadIdx.x / T, t = threadIdx.x % T;
  const int rr = vec / M, m = vec % M;
  const int row0 = bid.x * rpb, r = row0 + rr;
  const int l = bid.y, split = bid.z;
  const int cm = l * M + m - a.chunk_base;
  const int slot0 = l * M - a.chunk_base;             // slot of the mode sum
  stage_batch(a, l, spos, ssig);
  const float2* Prow = P + ((long long)(l * M + m) * F + r) * F;
  if constexpr (!PL2) {
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) Psm[vec * F + t + N1 * n2] = __ldg(Prow + t + N1 * n2);
  }
  const float2* Ol = O + a.obj_off[l];
  const int Wl = a.obj_w[l];
  // position b's scratch row of this vector (2 KB contiguous, 16-byte pieces by its T threads)
  // and the block's object rows, into buffer buf
  auto prefetch = [&](int b, int buf) {
    const float2* row = S + (((long long)b * a.C + cm) * F + r) * F;
    float2* dst = Sst + (buf * V + vec) * RR;
#pragma unroll
    for (int k = 0; k < F / (2 * T); ++k) cp_async16(dst + 2 * (t + T * k), row + 2 * (t + T * k));
    if (a.patch)
      prefetch_orows<F>(a.patch + ((long long)b * a.L + l) * F * F, F, make_int2(0, 0), row0, rpb, Ost + buf * rpb * F);
    else
      prefetch_orows<F>(Ol, Wl, spos[b], row0, rpb, Ost + buf * rpb * F);
    cp_async_commit();
  };
  float2 acc[N2];
#pragma unroll
  for (int n2 = 0; n2 < N2; ++n2) acc[n2] = make_float2(0.f, 0.f);
  int b = next_pos(spos, split - nsplit, a.nb, nsplit);
  if (b >= 0) prefetch(b, 0);
  for (int buf = 0; b >= 0; buf ^= 1) {
    cp_async_wait<0>();
    __syncthreads();                                  // position b has landed; buffer buf^1 is free
    const int bn = next_pos(spos, b, a.nb, nsplit);
    if (bn >= 0) prefetch(bn, buf ^ 1);
    const float s = ssig[b];
    float2* reg = Sst + (buf * V + vec) * RR;         // this vector's row, then its exchange/mode-sum area
    const float2* orow = Ost + (buf * rpb + rr) * F;
    float2 v[N2];
#pragma unroll
    for (int sl = 0; sl < N2; ++sl) v[sl] = reg[idxO<F>(t, sl)];
    __syncwarp();                                     // the row is in registers before the exchange reuses it
    fft_inv_O2I<F>(v, t, reg, a.tw, WarpSync{});
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) {
      const int c = t + N1 * n2;
      const float2 gp = cconjmul(orow[c], v[n2]);                       // conj(p) chi
      acc[n2].x = fmaf(s, gp.x, acc[n2].x);
      acc[n2].y = fmaf(s, gp.y, acc[n2].y);
      const float2 pv = PL2 ? __ldg(Prow + c) : Psm[vec * F + c];
      reg[c] = cscale(cconjmul(pv, v[n2]), s);                          // conj(sigma P) chi
    }
    __syncthreads();
    float2* dst = S + (((long long)b * a.C + slot0) * F + row0) * F;      // the block's rpb rows, contiguous
    for (int e = threadIdx.x; e < rpb * F; e += blockDim.x) {           // modes added in order
      const int rr2 = e / F, c = e % F;
      const float2* red = Sst + (buf * V + rr2 * M) * RR + c;
      float2 sum = red[0];
      switch (M) {                                    // small mode counts unrolled, same order
        case 1: break;
        case 2: sum = cadd(sum, red[RR]); break;
        case 3: sum = cadd(cadd(sum, red[RR]), red[2 * RR]); break;
        case 4: sum = cadd(cadd(cadd(sum, red[RR]), red[2 * RR]), red[3 * RR]); break;
        default:
          for (int mm = 1; mm < M; ++mm) sum = cadd(sum, red[mm * RR]);
      }
      dst[e] = sum;
    }
    b = bn;
  }
  float2* g = gPs + (long long)split * gp_stride + ((long long)(l * M + m) * F + r) * F;
#pragma unroll
  for (int n2 = 0; n2 < N2; ++n2) {
    const int c = t + N1 * n2;
    g[c] = cadd(g[c], acc[n2]);
  }
}

template <int F, bool PL2>
__global__ void __launch_bounds__(PL2 ? kRowAdjL2Threads : 256, (F <= 256 || PL2 ? 2 : 1))
k_row_adj_l(const float2* __restrict__ O, const float2* __restrict__ P, float2* __restrict__ S,
            float2* __restrict__ gPs, long long gp_stride, KArgs a, int rpb, int nsplit) {
  pdl_wait();
  pdl_trigger();
  row_adj_l_body<F, PL2>(O, P, S, gPs, gp_stride, a, rpb, nsplit, blockIdx);
}

// Same pass at F = 512 with one warp per row (fft512_inv_warp: 16 values per lane instead of 32
// per thread of a 16-thread vector), probe rows through L1/L2: the row and its probe-gradient
// sums take half the registers, so twice as many warps fit on an SM.  Vector v (warp v) takes
// row blockIdx.x*rpb + v/M of mode v%M; element n of the row is value n/32 of lane n%32.
// grid (512/rpb, L, nsplit), block 32*M*rpb <= kRowAdjWThreads, dynamic smem row_adj_w_smem(M, rpb)
constexpr int kRowAdjWThreads = 320;
constexpr int kRowAdjWRegion = kFft512WarpXch;      // per-vector row / exchange / mode-sum area (>= 512)
__host__ __device__ constexpr int row_adj_w_smem(int M, int rpb) {
  return (2 * M * rpb * kRowAdjWRegion + 2 * rpb * 512) * (int)sizeof(float2);
}

template <int F>
__device__ __forceinline__ void row_adj_w_body(const float2* __restrict__ O, const float2* __restrict__ P,
                                               float2* __restrict__ S, float2* __restrict__ gPs, long long gp_stride,
                                               const KArgs& a, int rpb, int nsplit, const uint3 bid) {
  static_assert(F == 512, "one warp per row is the 512-point layout");
  constexpr int RR = kRowAdjWRegion;
  extern __shared__ __align__(16) float2 smem[];
  __shared__ int2 spos[kMaxB];
  __shared__ float ssig[kMaxB];
  const int M = a.M, V = M * rpb;
  float2* Sst = smem;                                 // [2][V][RR] scratch rows / exchange / mode sums
  float2* Ost = Sst + 2 * V * RR;                     // [2][rpb][F] object rows
  const int vec = threadIdx.x >> 5, t = threadIdx.x & 31;
  const int rr = vec / M, m = vec % M;
  const int row0 = bid.x * rpb, r = row0 + rr;
  const int l = bid.y, split = bid.z;
  const int cm = l * M + m - a.chunk_base;
  const int slot0 = l * M - a.chunk_base;
  stage_batch(a, l, spos, ssig);
  const float2* Prow = P + ((long long)(l * M + m) * F + r) * F;
  const float2* Ol = O + a.obj_off[l];
  const int Wl = a.obj_w[l];
  auto prefetch = [&](int b, int buf) {
    const float2* row = S + (((long long)b * a.C + cm) * F + r) * F;
    float2* dst = Sst + (buf * V + vec) * RR;
#pragma unroll
    for (int k = 0; k < F / 64; ++k) cp_async16(dst + 2 * (t + 32 * k), row + 2 * (t + 32 * k));
    if (a.patch)
      prefetch_orows<F>(a.patch + ((long long)b * a.L + l) * F * F, F, make_int2(0, 0), row0, rpb, Ost + buf * rpb * F);
    else
      prefetch_orows<F>(Ol, Wl, spos[b], row0, rpb, Ost + buf * rpb * F);
    cp_async_commit();
  };
  float2 acc[16];
#pragma unroll
  for (int n2 = 0; n2 < 16; ++n2) acc[n2] = make_float2(0.f, 0.f);
  int b = next_pos(spos, split - nsplit, a.nb, nsplit);
  if (b >= 0) prefetch(b, 0);
  for (int buf = 0; b >= 0; buf ^= 1) {
    cp_async_wait<0>();
    __syncthreads();                                  // position b has landed; buffer buf^1 is free
    const int bn = next_pos(spos, b, a.nb, nsplit);
    if (bn >= 0) prefetch(bn, buf ^ 1);
    const float s = ssig[b];
    float2* reg = Sst + (buf * V + vec) * RR;
    const float2* orow = Ost + (buf * rpb + rr) * F;
    float2 v[16];
    fft512_inv_warp(reg, v, t, reg, a.tw);
#pragma unroll
    for (int n2 = 0; n2 < 16; ++n2) {
      const int c = t + 32 * n2;
      const float2 gp = cconjmul(orow[c], v[n2]);                       // conj(p) chi
      acc[n2].x = fmaf(s, gp.x, acc[n2].x);
      acc[n2].y = fmaf(s, gp.y, acc[n2].y);
      reg[c] = cscale(cconjmul(__ldg(Prow + c), v[n2]), s);             // conj(sigma P) chi
    }
    __syncthreads();
    float2* dst = S + (((long long)b * a.C + slot0) * F + row0) * F;
    for (int e = threadIdx.x; e < rpb * F; e += blockDim.x) {           // modes added in order
      const int rr2 = e / F, c = e % F;
      const float2* red = Sst + (buf * V + rr2 * M) * RR + c;
      float2 sum = red[0];
      for (int mm = 1; mm < M; ++mm) sum = cadd(sum, red[mm * RR]);
      dst[e] = sum;
    }
    b = bn;
  }
  float2* g = gPs + (long long)split * gp_stride + ((long long)(l * M + m) * F + r) * F;
#pragma unroll
  for (int n2 = 0; n2 < 16; ++n2) {
    const int c = t + 32 * n2;
    g[c] = cadd(g[c], acc[n2]);
  }
}

template <int F>
__global__ void __launch_bounds__(kRowAdjWThreads, 2)
k_row_adj_w(const float2* __restrict__ O, const float2* __restrict__ P, float2* __restrict__ S,
            float2* __restrict__ gPs, long long gp_stride, KArgs a, int rpb, int nsplit) {
  pdl_wait();
  pdl_trigger();
  row_adj_w_body<F>(O, P, S, gPs, gp_stride, a, rpb, nsplit, blockIdx);
}

// ---------------------------------------------------------------------------------------
// forward row pass over all modes of one wavelength (one mode chunk holds every mode).
// Vector v = rr*M + m takes row r = blockIdx.x*rpb + rr of probe mode (l, m); its probe row
// stays in registers while the block runs over the positions of its split; the object rows
// of the next position are copied into shared memory (cp.async) during the current one.
// grid (F/rpb, L, nsplit), block T*M*rpb <= 256, dynamic smem row_fwd_l_smem<F>(M, rpb)
// ---------------------------------------------------------------------------------------
template <int F>
__host__ __device__ constexpr int row_fwd_l_smem(int M, int rpb) {
  return (M * rpb * Xch<F>::region_rows + 2 * rpb * F) * (int)sizeof(float2);
}

template <int F>
__global__ void __launch_bounds__(256, (F <= 256 ? 2 : 1))
k_row_fwd_l(const float2* __restrict__ O, const float2* __restrict__ P, float2* __restrict__ S, KArgs a, int rpb,
            int nsplit) {
  pdl_wait();
  pdl_trigger();
  constexpr int N1 = FftShape<F>::N1, N2 = FftShape<F>::N2, T = N1, RR = Xch<F>::region_rows;
  extern __shared__ __align__(16) float2 smem[];
  __shared__ int2 spos[kMaxB];
  __shared__ float ssig[kMaxB];
  const int M = a.M, V = M * rpb;
  float2* xch = smem;                                 // [V][RR]
  float2* Ost = xch + V * RR;                         // [2][rpb][F]
  const int vec = threadIdx.x / T, t = threadIdx.x % T;
  const int rr = vec / M, m = vec % M;
  const int row0 = blockIdx.x * rpb, r = row0 + rr;
  const int l = blockIdx.y, split = blockIdx.z;
  const int cm = l * M + m - a.chunk_base;
  stage_batch(a, l, spos, ssig);
  float2 pr[N2];
  {
    const float2* Prow = P + ((long long)(l * M + m) * F + r) * F;
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) pr[n2] = __ldg(Prow + t + N1 * n2);
  }
  const float2* Ol = O + a.obj_off[l];
  const int Wl = a.obj_w[l];
  int b = next_pos(spos, split - nsplit, a.nb, nsplit);
  if (b >= 0) {
    prefetch_orows<F>(Ol, Wl, spos[b], row0, rpb, Ost);
    cp_async_commit();
  }
  for (int buf = 0; b >= 0; buf ^= 1) {
    cp_async_wait<0>();
    __syncthreads();                                  // position b's rows have landed; buf^1 is free
    const int bn = next_pos(spos, b, a.nb, nsplit);
    if (bn >= 0) {
      prefetch_orows<F>(Ol, Wl, spos[bn], row0, rpb, Ost + (buf ^ 1) * rpb * F);
      cp_async_commit();
    }
    const float s = ssig[b];
    const float2* orow = Ost + (buf * rpb + rr) * F;
    float2 v[N2];
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) v[n2] = cmul(pr[n2], cscale(orow[t + N1 * n2], s));
    fft_fwd_I2O<F>(v, t, xch + vec * RR, a.tw, WarpSync{});
    float2* out = S + (((long long)b * a.C + cm) * F + r) * F;
#pragma unroll
    for (int sl = 0; sl < N2; ++sl) out[idxO<F>(t, sl)] = v[sl];
    b = bn;
  }
}

// Same pass at F = 512 with one warp per row (fft512_fwd_warp): the probe row takes 16 values per
// lane in registers instead of 32, so two blocks of up to 10 warps fit on an SM.
// grid (512/rpb, L, nsplit), block 32*M*rpb <= kRowAdjWThreads, dynamic smem row_fwd_w_smem(M, rpb)
__host__ __device__ constexpr int row_fwd_w_smem(int M, int rpb) {
  return (M * rpb * kFft512WarpXchF + 2 * rpb * 512) * (int)sizeof(float2);
}

template <int F>
__global__ void __launch_bounds__(kRowAdjWThreads, 2)
k_row_fwd_w(const float2* __restrict__ O, const float2* __restrict__ P, float2* __restrict__ S, KArgs a, int rpb,
            int nsplit) {
  static_assert(F == 512, "one warp per row is the 512-point layout");
  pdl_wait();
  pdl_trigger();
  constexpr int RR = kFft512WarpXchF;
  extern __shared__ __align__(16) float2 smem[];
  __shared__ int2 spos[kMaxB];
  __shared__ float ssig[kMaxB];
  const int M = a.M, V = M * rpb;
  float2* xch = smem;                                 // [V][RR]
  float2* Ost = xch + V * RR;                         // [2][rpb][F]
  const int vec = threadIdx.x >> 5, t = threadIdx.x & 31;
  const int rr = vec / M, m = vec % M;
  const int row0 = blockIdx.x * rpb, r = row0 + rr;
  const int l = blockIdx.y, split = blockIdx.z;
  const int cm = l * M + m - a.chunk_base;
  stage_batch(a, l, spos, ssig);
  float2 pr[16];
  {
    const float2* Prow = P + ((long long)(l * M + m) * F + r) * F;
#pragma unroll
    for (int n2 = 0; n2 < 16; ++n2) pr[n2] = __ldg(Prow + t + 32 * n2);
  }
  const float2* Ol = O + a.obj_off[l];
  const int Wl = a.obj_w[l];
  const int oc = (t & 15) + 256 * (t >> 4);           // output column of x[0] (then + 16 j)
  int b = next_pos(spos, split - nsplit, a.nb, nsplit);
  if (b >= 0) {
    prefetch_orows<F>(Ol, Wl, spos[b], row0, rpb, Ost);
    cp_async_commit();
  }
  for (int buf = 0; b >= 0; buf ^= 1) {
    cp_async_wait<0>();
    __syncthreads();                                  // position b's rows have landed; buf^1 is free
    const int bn = next_pos(spos, b, a.nb, nsplit);
    if (bn >= 0) {
      prefetch_orows<F>(Ol, Wl, spos[bn], row0, rpb, Ost + (buf ^ 1) * rpb * F);
      cp_async_commit();
    }
    const float s = ssig[b];
    const float2* orow = Ost + (buf * rpb + rr) * F;
    float2 v[16];
#pragma unroll
    for (int n2 = 0; n2 < 16; ++n2) v[n2] = cmul(pr[n2], cscale(orow[t + 32 * n2], s));
    fft512_fwd_warp(v, t, xch + vec * RR, a.tw);
    float2* out = S + (((long long)b * a.C + cm) * F + r) * F + oc;
#pragma unroll
    for (int j = 0; j < 16; ++j) out[16 * j] = v[j];
    b = bn;
  }
}

// Fixed-order sum of the per-split probe-gradient buffers: out[i] = sum_s part[s][i].
__global__ void k_sum_splits(const float2* __restrict__ part, int nsplit, long long n, float2* __restrict__ out);

// ---------------------------------------------------------------------------------------
// object gradient from one mode-summed slot per (position, wavelength) (after k_row_adj_l):
// one block per 32x32 tile of grad O_l inside the batch's bounding box.  The positions whose
// patches overlap the tile are listed first (ascending), then added four at a time with
// their loads issued together.   grid (tiles of the largest box, L)
// ---------------------------------------------------------------------------------------
template <int F>
__device__ __forceinline__ void obj_grad_l_body(const float2* __restrict__ S, float2* __restrict__ gO, const KArgs& a,
                                                const uint3 bid) {
  __shared__ int2 spos[kMaxB];
  __shared__ float ssig[kMaxB];
  __shared__ int list[kMaxB];
  __shared__ int nlist;
  const int l = bid.y;
  const int by0 = a.box[l][0], bx0 = a.box[l][1];
  const int ntx = (a.box[l][3] - bx0 + kTile - 1) / kTile;
  const int nty = (a.box[l][2] - by0 + kTile - 1) / kTile;
  if ((int)bid.x >= ntx * nty) return;          // uniform over the block
  stage_batch(a, l, spos, ssig);
  const int oy0 = by0 + ((int)bid.x / ntx) * kTile, ox0 = bx0 + ((int)bid.x % ntx) * kTile;
  if (threadIdx.x < 32) {                             // ordered compaction by warp 0
    int n = 0;
    for (int b0 = 0; b0 < a.nb; b0 += 32) {
      const int b = b0 + (int)threadIdx.x;
      bool hit = false;
      if (b < a.nb) {
        const int y = spos[b].x, x = spos[b].y;
        hit = !(y < 0 || y >= oy0 + kTile || y + F <= oy0 || x >= ox0 + kTile || x + F <= ox0);
      }
      const unsigned mask = __ballot_sync(0xffffffffu, hit);
      if (hit) list[n + __popc(mask & ((1u << threadIdx.x) - 1u))] = b;
      n += __popc(mask);
    }
    if (threadIdx.x == 0) nlist = n;
  }
  __syncthreads();
  const int n = nlist;
  const int H = a.obj_h[l], Wd = a.obj_w[l];
  const int tx = threadIdx.x % kTile, ty0 = threadIdx.x / kTile;   // 8 row slots
  const int ox = ox0 + tx;
  const int slot0 = l * a.M - a.chunk_base;
  float2 acc[kTile / 8];
#pragma unroll
  for (int k = 0; k < kTile / 8; ++k) acc[k] = make_float2(0.f, 0.f);
  constexpr int PG = 4;                               // patches per group of loads
  for (int i0 = 0; i0 < n; i0 += PG) {
    float2 v[PG][kTile / 8];
#pragma unroll
    for (int pp = 0; pp < PG; ++pp) {
      const int b = i0 + pp < n ? list[i0 + pp] : -1;
      const int y = b >= 0 ? spos[b].x : 0, x = b >= 0 ? spos[b].y : 0;
      const bool in_x = b >= 0 && ox >= x && ox < x + F;
      const float2* src = S + ((long long)(b >= 0 ? b : 0) * a.C + slot0) * F * F + (ox - x);
#pragma unroll
      for (int k = 0; k < kTile / 8; ++k) {
        const int oy = oy0 + ty0 + 8 * k;
        const bool ok = in_x && oy >= y && oy < y + F;
        v[pp][k] = ok ? src[(long long)(oy - y) * F] : make_float2(0.f, 0.f);
      }
    }
#pragma unroll
    for (int pp = 0; pp < PG; ++pp)
#pragma unroll
      for (int k = 0; k < kTile / 8; ++k) acc[k] = cadd(acc[k], v[pp][k]);
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

template <int F>
__global__ void __launch_bounds__(256)
k_obj_grad_l(const float2* __restrict__ S, float2* __restrict__ gO, KArgs a) {
  pdl_wait();
  pdl_trigger();
  obj_grad_l_body<F>(S, gO, a, blockIdx);
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
