// Fractional scan offsets (f2 of Eq. 2 by the Fourier shift theorem) and the gradient with
// respect to them.
//
// With offsets delta[l][j] (rows, columns; pixels) the object patch of position j at
// wavelength l is the F x F window at the integer position resampled at r + delta:
//   p_delta = F2^-1[ ramp * F2 p ],   ramp(k) = exp(2 pi i (f(k_y) d_y + f(k_x) d_x)),
// with f(k) = k/F for k < F/2 and (k - F)/F otherwise, the window taken as one period.
// Per position batch, before the forward row pass:
//   k_shift_rows (window rows from O -> row DFT -> T)
//   k_shift_cols (column DFT, * ramp, keep Q = ramp * DFT2(p) for the adjoint, inverse column DFT)
//   k_shift_rows (inverse row DFT, / F^2 -> the batch's patch buffer, read by the row passes)
// and after the adjoint row pass, on the mode-summed object-gradient patch g (the gradient
// with respect to p_delta) in scratch slot (b, l*M):
//   k_shift_rows (row DFT -> T)
//   k_shift_cols (column DFT -> Ghat; position-gradient partials
//                 dL/d delta_a = (1/F^2) Re sum_k conj(Ghat) (2 pi i f_a) Q, by Parseval's theorem;
//                 * conj(ramp); inverse column DFT)
//   k_shift_rows (inverse row DFT, / F^2 -> back into the slot: the adjoint-shifted patch
//                 gradient that the object-gradient kernel adds into grad O)
// All transforms are the unscaled two-stage register FFTs of fft_regs.cuh.
#pragma once
#include "kernels.cuh"

namespace ptycho {

// Frequency of DFT index k in cycles per pixel (numpy's fftfreq order).
template <int F>
__device__ __forceinline__ float dft_freq(int k) {
  return (float)(k < F / 2 ? k : k - F) * (1.0f / (float)F);
}

struct ShiftArgs {
  const float2* src;             // rows to transform (see k_shift_rows)
  long long src_b, src_l;        // element strides of the source between positions and wavelengths
  float2* dst;
  long long dst_b, dst_l;
  float scale;                   // applied to the output (1 or 1/F^2)
  const float* delta;            // [L][J][2] fractional offsets (device)
  float2* T;                     // [B][L][F][F] transform workspace of the batch
  float2* Q;                     // [B][L][F][F] ramp * DFT2(window) of the batch
  double* dpart;                 // [nbatch][L][F/W][2] position-gradient partials, or null
};

// Row DFT of the F x F patches of the batch, one row per T threads.
// INV = false: source rows in natural order -> forward DFT -> destination in natural order;
// INV = true: the inverse.  FROM_O: the source rows are the object window at the integer
// position (src/src_b/src_l unused).   grid (F/RPB, L, nb)
template <int F, bool INV, bool FROM_O>
__global__ void __launch_bounds__(RowCfg<F>::threads)
k_shift_rows(const float2* __restrict__ O, KArgs a, ShiftArgs sa) {
  pdl_wait();
  pdl_trigger();
  constexpr int N1 = FftShape<F>::N1, N2 = FftShape<F>::N2, T = RowCfg<F>::T;
  extern __shared__ float2 smem[];
  const int vec = threadIdx.x / T, t = threadIdx.x % T;
  const int r = blockIdx.x * RowCfg<F>::RPB + vec;
  const int l = blockIdx.y, b = blockIdx.z;
  const int j = batch_pos(a, a.batch_off + b);
  if (j < 0) return;                                  // uniform over the block
  const float2* src = FROM_O ? O + a.obj_off[l] + (long long)(a.pos[(l * a.J + j) * 2] + r) * a.obj_w[l] +
                                   a.pos[(l * a.J + j) * 2 + 1]
                             : sa.src + b * sa.src_b + l * sa.src_l + (long long)r * F;
  float2* dst = sa.dst + b * sa.dst_b + l * sa.dst_l + (long long)r * F;
  float2* xc = smem + vec * Xch<F>::region_rows;
  float2 v[N2];
  if (!INV) {
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) v[n2] = src[t + N1 * n2];
    fft_fwd_I2O<F>(v, t, xc, a.tw, WarpSync{});
#pragma unroll
    for (int sl = 0; sl < N2; ++sl) dst[idxO<F>(t, sl)] = cscale(v[sl], sa.scale);
  } else {
#pragma unroll
    for (int sl = 0; sl < N2; ++sl) v[sl] = src[idxO<F>(t, sl)];
    fft_inv_O2I<F>(v, t, xc, a.tw, WarpSync{});
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) dst[t + N1 * n2] = cscale(v[n2], sa.scale);
  }
}

// Column pass of the shift on T (rows already transformed): column DFT, phase ramp
// (ADJ: its conjugate, after the position-gradient partials), inverse column DFT, back to T.
// Forward: Q <- ramp * spectrum.   grid (F/W, L, nb)
template <int F, bool ADJ>
__global__ void __launch_bounds__(ColCfg<F>::threads)
k_shift_cols(KArgs a, ShiftArgs sa) {
  pdl_wait();
  pdl_trigger();
  constexpr int N1 = FftShape<F>::N1, N2 = FftShape<F>::N2, W = ColCfg<F>::W;
  extern __shared__ float2 smem[];
  __shared__ float red[4][ColCfg<F>::threads / 32];
  const int c = threadIdx.x % W, t = threadIdx.x / W;
  const int col = blockIdx.x * W + c;
  const int l = blockIdx.y, b = blockIdx.z;
  const int j = batch_pos(a, a.batch_off + b);
  if (j < 0) {
    if (ADJ && sa.dpart && threadIdx.x < 2)
      sa.dpart[(((long long)(a.batch_off + b) * a.L + l) * gridDim.x + blockIdx.x) * 2 + threadIdx.x] = 0.0;
    return;                                           // uniform over the block
  }
  const float dy = __ldg(sa.delta + (l * a.J + j) * 2), dx = __ldg(sa.delta + (l * a.J + j) * 2 + 1);
  float2* base = sa.T + ((long long)b * a.L + l) * F * F + col;
  float2* qb = sa.Q + ((long long)b * a.L + l) * F * F + col;
  float2 v[N2];
#pragma unroll
  for (int n2 = 0; n2 < N2; ++n2) v[n2] = base[(long long)(t + N1 * n2) * F];
  fft_fwd_I2O<F>(v, t, smem + c * Xch<F>::region_cols, a.tw, BlockSync{});
  const float fx = dft_freq<F>(col);
  float gyh = 0.f, gyl = 0.f, gxh = 0.f, gxl = 0.f;    // double-float sums of the gradient terms
#pragma unroll
  for (int sl = 0; sl < N2; ++sl) {
    const int k = idxO<F>(t, sl);
    const float fy = dft_freq<F>(k);
    float sn, cs;
    sincospif(2.0f * (fy * dy + fx * dx), &sn, &cs);  // ramp = exp(2 pi i (fy dy + fx dx))
    const float2 ramp = make_float2(cs, sn);
    if (!ADJ) {
      v[sl] = cmul(v[sl], ramp);
      qb[(long long)k * F] = v[sl];
    } else {
      // Re(conj(G) (2 pi i f) Q) = -2 pi f Im(conj(G) Q)
      const float2 q = qb[(long long)k * F];
      const float im = fmaf(v[sl].x, q.y, -v[sl].y * q.x);
      df_add(gyh, gyl, -6.283185307179586f * fy * im);
      df_add(gxh, gxl, -6.283185307179586f * fx * im);
      v[sl] = cmulc(v[sl], ramp);
    }
  }
  if (ADJ && sa.dpart) {
    df_warp_sum(gyh, gyl);
    df_warp_sum(gxh, gxl);
    if ((threadIdx.x & 31) == 0) {
      red[0][threadIdx.x >> 5] = gyh;
      red[1][threadIdx.x >> 5] = gyl;
      red[2][threadIdx.x >> 5] = gxh;
      red[3][threadIdx.x >> 5] = gxl;
    }
  }
  fft_inv_O2I<F>(v, t, smem + c * Xch<F>::region_cols, a.tw, BlockSync{});   // its barriers publish red
#pragma unroll
  for (int n2 = 0; n2 < N2; ++n2) base[(long long)(t + N1 * n2) * F] = v[n2];
  if (ADJ && sa.dpart && threadIdx.x < 2) {
    double s = 0.0;
    for (int w = 0; w < ColCfg<F>::threads / 32; ++w)
      s += (double)red[2 * threadIdx.x][w] + (double)red[2 * threadIdx.x + 1][w];
    const double inv = 1.0 / ((double)F * (double)F);
    sa.dpart[(((long long)(a.batch_off + b) * a.L + l) * gridDim.x + blockIdx.x) * 2 + threadIdx.x] = s * inv;
  }
}

// Position gradient: g_delta[l][j][a] = sum, in call-entry order, of the partials of every
// entry i with bidx[i] = j; 0 for positions outside the call.   grid (ceil(L*J/256))
__global__ void k_delta_grad(const int32_t* __restrict__ bidx, int nbatch, int L, int J, const double* __restrict__ dpart,
                             int nstrips, float* __restrict__ g_delta);

}  // namespace ptycho
