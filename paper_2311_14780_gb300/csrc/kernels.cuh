// Kernels of the batched multi-wavelength, multi-mode ptychography forward model and its
// adjoint (Eq. 1 written as f5(f4(f3(f1(sigma_j), f2(s_j)))) of Eq. 2).
//
// Work is organised per *position batch* (B scan positions) and per *mode chunk* (a run of
// the L*M (wavelength, probe-mode) pairs, index mode = l*M + m).  For a batch the 2D DFT of
// every exit wave goes through a scratch buffer S[B][C][F][F] (complex64) sized to stay in
// the GPU's L2 cache:
//
//   k_row_fwd   psi = sigma_j P_lm * O_l(r - s_j) for one row; 1D FFT along the row -> S
//   k_col_fwd   1D FFT along columns of S -> Psi (scaled by 1/F); accumulate |Psi|^2 over
//               the modes of a group into Ipart; optionally keep Psi in S for the adjoint
//   k_loss      I = sum of groups (+ background) on the model grid; tilted-plane remap to the
//               camera grid; mask; loss terms (FP64 block partials) and D = mask dL/dI
//   k_col_adj   G = R^T D on the model grid; Psi (kept, or recomputed from S);
//               (2/F) G Psi; inverse 1D FFT along columns -> S
//   k_row_adj   inverse 1D FFT along rows -> chi = dL/dpsi; grad P_lm += conj(sigma p) chi
//               summed over the batch in registers; S <- conj(sigma P_lm) chi
//   k_obj_grad  grad O_l tile += sum over the batch's overlapping patches and the chunk's
//               modes of S (each object tile is owned by one thread block: deterministic)
//   k_loss_reduce  fixed-order FP64 sum of the per-block loss partials
//   k_adam      Adam on the real and imaginary parts of O and P
#pragma once
#include "fft_regs.cuh"

namespace ptycho {

constexpr int kMaxL = 16;
constexpr int kLossThreads = 256;
constexpr int kTile = 32;        // object-gradient tile side

struct KArgs {
  int L, M, F, J;
  const int32_t* pos;            // [L][J][2] (row, col) of the patch corner, device
  long long obj_off[kMaxL];      // complex offset of O_l in the packed object buffer
  int obj_h[kMaxL], obj_w[kMaxL];
  const int32_t* bidx;           // positions of this call, in processing order
  int nbatch;                    // number of entries in bidx
  int batch_off;                 // first entry of the current position batch
  int nb;                        // positions in the current batch (<= B)
  const float* sigma;            // [J] power coefficients or null
  const float2* tw;              // W_F^(t*k2) table
  int C;                         // stride (modes) of the scratch buffer
  int chunk_base, chunk_len;     // global modes [chunk_base, chunk_base + chunk_len)
  int MG;                        // modes per column-kernel group
  int G;                         // groups per chunk (Ipart has G slices per position)
  int* status;                   // device status word (bit 0: a position index was out of range)
};

// Position index of batch entry i, or -1 (and the status bit set) if out of range.
__device__ __forceinline__ int batch_pos(const KArgs& a, int i) {
  const int j = a.bidx[i];
  if (j < 0 || j >= a.J) {
    atomicOr(a.status, 1);
    return -1;
  }
  return j;
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
// forward row pass: exit wave (f1, f2, f3) and the row DFT (first half of f4)
// grid (F/RPB, chunk_len, nb)
// ---------------------------------------------------------------------------------------
template <int F>
__global__ void __launch_bounds__(RowCfg<F>::threads)
k_row_fwd(const float2* __restrict__ O, const float2* __restrict__ P, float2* __restrict__ S, KArgs a) {
  constexpr int N1 = FftShape<F>::N1, N2 = FftShape<F>::N2, T = RowCfg<F>::T;
  extern __shared__ float2 smem[];
  const int vec = threadIdx.x / T, t = threadIdx.x % T;
  const int r = blockIdx.x * RowCfg<F>::RPB + vec;
  const int cm = blockIdx.y, b = blockIdx.z;
  const int mode = a.chunk_base + cm;
  const int l = mode / a.M;
  const int j = batch_pos(a, a.batch_off + b);
  if (j < 0) return;                                  // uniform over the block
  const int y = a.pos[(l * a.J + j) * 2], x = a.pos[(l * a.J + j) * 2 + 1];
  const float s = sigma_of(a, j);
  const float2* Orow = O + a.obj_off[l] + (long long)(y + r) * a.obj_w[l] + x;
  const float2* Prow = P + ((long long)mode * F + r) * F;
  float2 v[N2];
#pragma unroll
  for (int n2 = 0; n2 < N2; ++n2) {
    const int c = t + N1 * n2;
    v[n2] = cscale(cmul(__ldg(Prow + c), __ldg(Orow + c)), s);
  }
  fft_fwd_I2O<F>(v, t, smem + vec * Xch<F>::region_rows, a.tw, WarpSync{});
  float2* out = S + (((long long)b * a.C + cm) * F + r) * F;
#pragma unroll
  for (int sl = 0; sl < N2; ++sl) out[idxO<F>(t, sl)] = v[sl];
}

// ---------------------------------------------------------------------------------------
// forward column pass: column DFT (second half of f4), |Psi|^2 summed over a mode group
// grid (F/W, G, nb)
// ---------------------------------------------------------------------------------------
template <int F, bool STORE>
__global__ void __launch_bounds__(ColCfg<F>::threads)
k_col_fwd(float2* __restrict__ S, float* __restrict__ Ipart, KArgs a, int first_chunk) {
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
// measurement (f5) and loss: camera-grid prediction, masked loss partials, D = mask dL/dI
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
  constexpr int FF = F * F;
  __shared__ double red[kLossThreads / 32];
  const int b = blockIdx.y;
  const int i = a.batch_off + b;
  const int j = batch_pos(a, i);
  if (j < 0) {                                        // uniform over the block
    if (la.loss_part && threadIdx.x == 0) la.loss_part[(long long)i * (FF / kLossThreads) + blockIdx.x] = 0.0;
    if (la.D) la.D[(long long)b * FF + blockIdx.x * kLossThreads + threadIdx.x] = 0.f;
    return;
  }
  const int q = blockIdx.x * kLossThreads + threadIdx.x;
  const float* Ip = la.Ipart + (long long)b * a.G * FF;
  float Ic = 0.f;
  bool valid = true;
  if (la.remap) {
    const int u = la.tap_base[q];
    if (u < 0) {
      valid = false;
    } else {
      const float2 w = la.tap_w[q];
      const float i00 = model_I(Ip, la.bg, a.G, FF, u), i01 = model_I(Ip, la.bg, a.G, FF, u + 1);
      const float i10 = model_I(Ip, la.bg, a.G, FF, u + F), i11 = model_I(Ip, la.bg, a.G, FF, u + F + 1);
      Ic = (1.f - w.x) * ((1.f - w.y) * i00 + w.y * i01) + w.x * ((1.f - w.y) * i10 + w.y * i11);
    }
  } else {
    Ic = model_I(Ip, la.bg, a.G, FF, q);
  }
  if (la.I_pred) la.I_pred[(long long)j * FF + q] = valid ? Ic : 0.f;
  double term = 0.0;
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
  }
  if (la.loss_part) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) term += __shfl_down_sync(0xffffffffu, term, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = term;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int w = 0; w < kLossThreads / 32; ++w) s += red[w];
      la.loss_part[(long long)i * (FF / kLossThreads) + blockIdx.x] = s;
    }
  }
}

// ---------------------------------------------------------------------------------------
// adjoint column pass: G = R^T D, (2/F) G Psi, inverse column DFT
// grid (F/W, G, nb)
// ---------------------------------------------------------------------------------------
struct AdjArgs {
  const float* D;                // [B][F][F] camera grid
  const int32_t* rt_ptr;         // [F*F+1] CSR of R^T over centred model pixels (remap only)
  const int32_t* rt_idx;         // camera pixel of each entry
  const float* rt_w;             // weight of each entry
  int remap;
};

template <int F, bool STORE>
__global__ void __launch_bounds__(ColCfg<F>::threads)
k_col_adj(float2* __restrict__ S, KArgs a, AdjArgs aa) {
  constexpr int N1 = FftShape<F>::N1, N2 = FftShape<F>::N2, W = ColCfg<F>::W;
  extern __shared__ float2 smem[];
  float* gt = reinterpret_cast<float*>(smem + W * Xch<F>::region_cols);   // [F][W]
  const int c = threadIdx.x % W, t = threadIdx.x / W;
  const int col0 = blockIdx.x * W;
  const int g = blockIdx.y, b = blockIdx.z;
  const float* Db = aa.D + (long long)b * F * F;
  const float scale = 2.0f / (float)F;
  for (int e = threadIdx.x; e < F * W; e += blockDim.x) {
    const int k = e / W, ce = e % W;
    const int u = ((k + F / 2) & (F - 1)) * F + ((col0 + ce + F / 2) & (F - 1));
    float gv;
    if (aa.remap) {
      gv = 0.f;
      const int e1 = __ldg(aa.rt_ptr + u + 1);
      for (int q = __ldg(aa.rt_ptr + u); q < e1; ++q) gv = fmaf(__ldg(aa.rt_w + q), Db[__ldg(aa.rt_idx + q)], gv);
    } else {
      gv = Db[u];
    }
    gt[k * W + ce] = gv * scale;
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

// ---------------------------------------------------------------------------------------
// adjoint row pass: chi = dL/dpsi; probe gradient summed over the batch; object-gradient
// contributions conj(sigma P) chi left in S.   grid (F/RPB, chunk_len)
// ---------------------------------------------------------------------------------------
template <int F>
__global__ void __launch_bounds__(RowCfg<F>::threads)
k_row_adj(const float2* __restrict__ O, const float2* __restrict__ P, float2* __restrict__ S,
          float2* __restrict__ gP, KArgs a) {
  constexpr int N1 = FftShape<F>::N1, N2 = FftShape<F>::N2, T = RowCfg<F>::T;
  extern __shared__ float2 smem[];
  const int vec = threadIdx.x / T, t = threadIdx.x % T;
  const int r = blockIdx.x * RowCfg<F>::RPB + vec;
  const int cm = blockIdx.y;
  const int mode = a.chunk_base + cm;
  const int l = mode / a.M;
  const float2* Prow = P + ((long long)mode * F + r) * F;
  float2 acc[N2];
#pragma unroll
  for (int n2 = 0; n2 < N2; ++n2) acc[n2] = make_float2(0.f, 0.f);
  for (int b = 0; b < a.nb; ++b) {
    const int j = batch_pos(a, a.batch_off + b);
    if (j < 0) continue;                              // uniform over the block
    const int y = a.pos[(l * a.J + j) * 2], x = a.pos[(l * a.J + j) * 2 + 1];
    const float s = sigma_of(a, j);
    float2* row = S + (((long long)b * a.C + cm) * F + r) * F;
    float2 v[N2];
#pragma unroll
    for (int sl = 0; sl < N2; ++sl) v[sl] = row[idxO<F>(t, sl)];
    fft_inv_O2I<F>(v, t, smem + vec * Xch<F>::region_rows, a.tw, WarpSync{});
    const float2* Orow = O + a.obj_off[l] + (long long)(y + r) * a.obj_w[l] + x;
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) {
      const int c = t + N1 * n2;
      const float2 p = __ldg(Orow + c);
      const float2 pr = __ldg(Prow + c);
      const float2 gp = cconjmul(p, v[n2]);        // conj(p) chi
      acc[n2].x = fmaf(s, gp.x, acc[n2].x);
      acc[n2].y = fmaf(s, gp.y, acc[n2].y);
      row[c] = cscale(cconjmul(pr, v[n2]), s);     // conj(sigma P) chi
    }
  }
  float2* g = gP + ((long long)mode * F + r) * F;
#pragma unroll
  for (int n2 = 0; n2 < N2; ++n2) {
    const int c = t + N1 * n2;
    g[c] = cadd(g[c], acc[n2]);
  }
}

// ---------------------------------------------------------------------------------------
// object gradient: each block owns 32x32 tiles of grad O_l inside the batch's bounding box
// and adds, in a fixed order, every overlapping patch contribution of the chunk's modes.
// grid (nblocks, L)
// ---------------------------------------------------------------------------------------
template <int F>
__global__ void __launch_bounds__(256)
k_obj_grad(const float2* __restrict__ S, float2* __restrict__ gO, KArgs a) {
  const int l = blockIdx.y;
  const int mlo = max(a.chunk_base, l * a.M), mhi = min(a.chunk_base + a.chunk_len, (l + 1) * a.M);
  if (mlo >= mhi) return;
  __shared__ int box[4];
  if (threadIdx.x == 0) {
    int y0 = 1 << 30, x0 = 1 << 30, y1 = -1, x1 = -1;
    for (int b = 0; b < a.nb; ++b) {
      const int j = batch_pos(a, a.batch_off + b);
      if (j < 0) continue;
      const int y = a.pos[(l * a.J + j) * 2], x = a.pos[(l * a.J + j) * 2 + 1];
      y0 = min(y0, y); x0 = min(x0, x); y1 = max(y1, y + F); x1 = max(x1, x + F);
    }
    if (y1 < 0) { y0 = 0; x0 = 0; y1 = 0; x1 = 0; }   // no valid position: empty box
    box[0] = y0; box[1] = x0; box[2] = y1; box[3] = x1;
  }
  __syncthreads();
  const int by0 = box[0], bx0 = box[1];
  const int nty = (box[2] - by0 + kTile - 1) / kTile, ntx = (box[3] - bx0 + kTile - 1) / kTile;
  const int H = a.obj_h[l], Wd = a.obj_w[l];
  float2* g = gO + a.obj_off[l];
  const int tx = threadIdx.x % kTile, ty0 = threadIdx.x / kTile;   // 8 row slots
  for (int tile = blockIdx.x; tile < nty * ntx; tile += gridDim.x) {
    const int oy0 = by0 + (tile / ntx) * kTile, ox0 = bx0 + (tile % ntx) * kTile;
    const int ox = ox0 + tx;
    float2 acc[kTile / 8];
#pragma unroll
    for (int k = 0; k < kTile / 8; ++k) acc[k] = make_float2(0.f, 0.f);
    for (int b = 0; b < a.nb; ++b) {
      const int j = a.bidx[a.batch_off + b];
      if (j < 0 || j >= a.J) continue;
      const int y = a.pos[(l * a.J + j) * 2], x = a.pos[(l * a.J + j) * 2 + 1];
      if (y >= oy0 + kTile || y + F <= oy0 || x >= ox0 + kTile || x + F <= ox0) continue;
      const bool in_x = ox >= x && ox < x + F;
      for (int mode = mlo; mode < mhi; ++mode) {
        const float2* src = S + ((long long)b * a.C + (mode - a.chunk_base)) * F * F;
#pragma unroll
        for (int k = 0; k < kTile / 8; ++k) {
          const int oy = oy0 + ty0 + 8 * k;
          if (in_x && oy >= y && oy < y + F) acc[k] = cadd(acc[k], src[(long long)(oy - y) * F + (ox - x)]);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < kTile / 8; ++k) {
      const int oy = oy0 + ty0 + 8 * k;
      if (oy < H && ox < Wd) {
        float2* p = g + (long long)oy * Wd + ox;
        *p = cadd(*p, acc[k]);
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// loss reduction and Adam
// ---------------------------------------------------------------------------------------
__global__ void k_loss_reduce(const double* __restrict__ part, long long n, double* out);
__global__ void k_adam(float* __restrict__ theta, const float* __restrict__ grad, float* __restrict__ m,
                       float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1,
                       float c2);

}  // namespace ptycho
