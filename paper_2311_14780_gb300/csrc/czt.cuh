// Chirp-z (zoom DFT) propagator: the paper's propagator for wavelength multiplexing (Section
// "Benchmarking ..."), which samples every wavelength's far field on the detector pixels from
// one common object grid.
//
// Along one axis, with centred indices n', k' in [-F/2, F/2) (array index = index + F/2):
//   Z_l[k'][n'] = exp(-2 pi i zeta_l n' k' / F),     zeta_l = lambda_ref / lambda_l,
// and the propagator is Psi = (1/F) Z_l psi Z_l^T (rows, then columns; output centred).
// Bluestein's identity n'k' = (n'^2 + k'^2 - (k'-n')^2) / 2 turns Z into a chirp, a circular
// convolution of length N = 2F with the chirp kernel h(m) = exp(+i pi zeta m^2 / F), |m| < F,
// and a chirp:  (Z x)(k') = w(k') sum_n [x(n) w(n')] h(k - n),  w(m) = exp(-i pi zeta m^2 / F).
// The convolution runs as an N-point FFT, a product with the kernel's spectrum Hhat (one per
// wavelength, built in FP64 on the host) and an inverse FFT.  Z^H uses the conjugate chirps.
//
// A vector of F values sits with T = N1 = F/16 threads (layout I: thread t holds n = t + N1*n2,
// 16 values); the N-point transform uses the same threads with 2F/N1 = 32 values each, the data
// in the first half and zeros in the second.  At F = 64, 128 and 256 N1 is the register FFT's
// (4, 8, 16); at F = 512 a vector takes a whole warp (N1 = 32, where the register FFT's 512-point
// rows use 16 threads of 32 values), so that the 1024-point transform is 32 x 32 and still fits
// 32 values per thread.
#pragma once
#include "kernels.cuh"

namespace ptycho {

constexpr int kCztV = 32;                             // values per thread of the N = 2F transform

struct CztArgs {
  const float2* chirp;           // [L][F] w(n') = exp(-i pi zeta n'^2 / F)
  const float2* hf;              // [L][2F] spectrum of the kernel of Z
  const float2* ha;              // [L][2F] spectrum of the kernel of Z^H
  const float2* tw2;             // [2F] twiddles W_2F^(t*k2) at tw2[k2*N1 + t]
};

// Two-stage FFT of length N1*N2 held by N1 threads with N2 values each (as fft_fwd_I2O /
// fft_inv_O2I of fft_regs.cuh, for any N1 <= N2 with N1 | N2).  xc: N2*(N1+1) elements.
template <int N1, int N2, class Sync>
__device__ __forceinline__ void fftn_fwd_I2O(float2 (&x)[N2], int t, float2* xc, const float2* __restrict__ tw,
                                             Sync sync) {
  Dft<N2, 1, false>::run(x);
#pragma unroll
  for (int k2 = 1; k2 < N2; ++k2) x[k2] = cmul(x[k2], __ldg(tw + k2 * N1 + t));
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) xc[k2 * (N1 + 1) + t] = x[k2];
  sync();
#pragma unroll
  for (int q = 0; q < N2 / N1; ++q)
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) x[q * N1 + n1] = xc[(t + N1 * q) * (N1 + 1) + n1];
  sync();
#pragma unroll
  for (int q = 0; q < N2 / N1; ++q) Dft<N1, 1, false>::run(x + q * N1);
}

template <int N1, int N2, class Sync>
__device__ __forceinline__ void fftn_inv_O2I(float2 (&x)[N2], int t, float2* xc, const float2* __restrict__ tw,
                                             Sync sync) {
#pragma unroll
  for (int q = 0; q < N2 / N1; ++q) Dft<N1, 1, true>::run(x + q * N1);
#pragma unroll
  for (int q = 0; q < N2 / N1; ++q)
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) xc[(t + N1 * q) * (N1 + 1) + n1] = x[q * N1 + n1];
  sync();
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) x[k2] = xc[k2 * (N1 + 1) + t];
  sync();
#pragma unroll
  for (int k2 = 1; k2 < N2; ++k2) x[k2] = cmulc(x[k2], __ldg(tw + k2 * N1 + t));
  Dft<N2, 1, true>::run(x);
}

template <int F> struct CztShape {
  static constexpr int N1 = F / 16;                   // threads per vector (FftShape<F>::N1 up to 256)
  static constexpr int NF = F / N1;                   // values per thread of an F-vector (16)
  static_assert(2 * NF == kCztV, "the chirp-z transform needs F/N1 = 16");
  static constexpr int xch = kCztV * (N1 + 1);        // exchange elements per vector
};

// In place on y (first NF slots: the F-vector in layout I; the rest is overwritten):
// ADJ = false computes Z_l x, ADJ = true computes Z_l^H x; the result is in layout I.
template <int F, bool ADJ, class Sync>
__device__ __forceinline__ void czt_vec(float2 (&y)[kCztV], int t, float2* xc, const CztArgs& ct, int l, Sync sync) {
  constexpr int N1 = CztShape<F>::N1, NF = CztShape<F>::NF;
  const float2* w = ct.chirp + (long long)l * F;
  const float2* H = (ADJ ? ct.ha : ct.hf) + (long long)l * 2 * F;
#pragma unroll
  for (int n2 = 0; n2 < NF; ++n2) {
    const float2 c = __ldg(w + t + N1 * n2);
    y[n2] = ADJ ? cmulc(y[n2], c) : cmul(y[n2], c);
  }
#pragma unroll
  for (int n2 = NF; n2 < kCztV; ++n2) y[n2] = make_float2(0.f, 0.f);
  fftn_fwd_I2O<N1, kCztV>(y, t, xc, ct.tw2, sync);
#pragma unroll
  for (int sl = 0; sl < kCztV; ++sl) y[sl] = cmul(y[sl], __ldg(H + kCztV * (sl % N1) + t + N1 * (sl / N1)));
  fftn_inv_O2I<N1, kCztV>(y, t, xc, ct.tw2, sync);
  const float inv = 1.0f / (float)(2 * F);
#pragma unroll
  for (int n2 = 0; n2 < NF; ++n2) {
    const float2 c = __ldg(w + t + N1 * n2);
    y[n2] = cscale(ADJ ? cmulc(y[n2], c) : cmul(y[n2], c), inv);
  }
}


// ---------------------------------------------------------------------------------------
// Passes of the pipeline with the chirp-z propagator (as k_row_fwd, k_col_fwd with the
// column DFT recomputed in the adjoint, k_col_adj and k_row_adj, with Z_l in place of the
// DFT; every layout is natural: the zoom transforms are centred, so no fftshift).
// ---------------------------------------------------------------------------------------
template <int F> struct CztRowCfg {
  static constexpr int T = CztShape<F>::N1;
  static constexpr int RPB = 256 / T;
  static constexpr int threads = RPB * T;
  static constexpr int smem = RPB * CztShape<F>::xch * (int)sizeof(float2);
};
template <int F> struct CztColCfg {
  static constexpr int T = CztShape<F>::N1;
  static constexpr int W = 256 / T;
  static constexpr int threads = W * T;
  static constexpr int R = CztShape<F>::xch | 1;      // odd stride between the columns' regions
  static constexpr int smem_fwd = W * R * (int)sizeof(float2);
  static constexpr int smem_adj = smem_fwd + F * W * (int)sizeof(float);
};
template <int F> struct CztRowAdjCfg {
  static constexpr int T = CztShape<F>::N1;
  static constexpr int RPB = 256 / (T * kAdjSlots);
  static constexpr int threads = RPB * T * kAdjSlots;
  static constexpr int vecs = RPB * kAdjSlots;
  static constexpr int smem_xch = vecs * CztShape<F>::xch * (int)sizeof(float2);
  static constexpr int smem_red = (kAdjSlots - 1) * RPB * F * (int)sizeof(float2);
  static constexpr int smem = smem_xch > smem_red ? smem_xch : smem_red;
};

// exit waves and the row transform.   grid (nb, F/RPB, L): positions vary fastest, so that the
// blocks running at the same time share probe rows in L2
template <int F>
__global__ void __launch_bounds__(CztRowCfg<F>::threads)
k_czt_row_fwd(const float2* __restrict__ O, const float2* __restrict__ P, float2* __restrict__ S, KArgs a,
              CztArgs ct) {
  pdl_wait();
  pdl_trigger();
  constexpr int N1 = CztShape<F>::N1, NF = CztShape<F>::NF, T = CztRowCfg<F>::T;
  extern __shared__ float2 smem[];
  const int vec = threadIdx.x / T, t = threadIdx.x % T;
  const int r = blockIdx.y * CztRowCfg<F>::RPB + vec;
  const int l = blockIdx.z, b = blockIdx.x;
  const int mlo = max(a.chunk_base, l * a.M), mhi = min(a.chunk_base + a.chunk_len, (l + 1) * a.M);
  if (mlo >= mhi) return;                             // uniform over the block
  const int j = batch_pos(a, a.batch_off + b);
  if (j < 0) return;                                  // uniform over the block
  const int y = a.pos[(l * a.J + j) * 2], x = a.pos[(l * a.J + j) * 2 + 1];
  const float s = sigma_of(a, j);
  const float2* Orow = O + a.obj_off[l] + (long long)(y + r) * a.obj_w[l] + x;
  float2 p[NF];
#pragma unroll
  for (int n2 = 0; n2 < NF; ++n2) p[n2] = cscale(__ldg(Orow + t + N1 * n2), s);
  float2* xc = smem + vec * CztShape<F>::xch;
  for (int mode = mlo; mode < mhi; ++mode) {
    const float2* Prow = P + ((long long)mode * F + r) * F;
    float2 v[kCztV];
#pragma unroll
    for (int n2 = 0; n2 < NF; ++n2) v[n2] = cmul(__ldg(Prow + t + N1 * n2), p[n2]);
    czt_vec<F, false>(v, t, xc, ct, l, WarpSync{});
    float2* out = S + (((long long)b * a.C + (mode - a.chunk_base)) * F + r) * F;
#pragma unroll
    for (int n2 = 0; n2 < NF; ++n2) out[t + N1 * n2] = v[n2];
  }
}

// column transform, (1/F) scaling and |Psi|^2 summed over a mode group.   grid (F/W, G, nb)
template <int F>
__global__ void __launch_bounds__(CztColCfg<F>::threads)
k_czt_col_fwd(const float2* __restrict__ S, float* __restrict__ Ipart, KArgs a, CztArgs ct) {
  pdl_wait();
  pdl_trigger();
  constexpr int N1 = CztShape<F>::N1, NF = CztShape<F>::NF, W = CztColCfg<F>::W;
  extern __shared__ float2 smem[];
  const int c = threadIdx.x % W, t = threadIdx.x / W;
  const int col = blockIdx.x * W + c;
  const int g = blockIdx.y, b = blockIdx.z;
  const int m0 = g * a.MG, m1 = min(a.chunk_len, m0 + a.MG);
  float acc[NF];
#pragma unroll
  for (int i = 0; i < NF; ++i) acc[i] = 0.f;
  for (int cm = m0; cm < m1; ++cm) {
    const int l = (a.chunk_base + cm) / a.M;
    const float2* base = S + ((long long)b * a.C + cm) * F * F + col;
    float2 v[kCztV];
#pragma unroll
    for (int n2 = 0; n2 < NF; ++n2) v[n2] = base[(long long)(t + N1 * n2) * F];
    czt_vec<F, false>(v, t, smem + c * CztColCfg<F>::R, ct, l, BlockSync{});
#pragma unroll
    for (int n2 = 0; n2 < NF; ++n2) acc[n2] = fmaf(v[n2].x, v[n2].x, fmaf(v[n2].y, v[n2].y, acc[n2]));
  }
  float* dst = Ipart + ((long long)b * a.G + g) * F * F;
  const float s2 = 1.0f / ((float)F * (float)F);
#pragma unroll
  for (int n2 = 0; n2 < NF; ++n2) dst[(t + N1 * n2) * F + col] = acc[n2] * s2;
}

// adjoint columns: recompute Z_c S, times (2/F) G, Z_c^H, times 1/F.   grid (F/W, G, nb)
template <int F>
__global__ void __launch_bounds__(CztColCfg<F>::threads)
k_czt_col_adj(float2* __restrict__ S, KArgs a, AdjArgs aa, CztArgs ct) {
  pdl_wait();
  pdl_trigger();
  constexpr int N1 = CztShape<F>::N1, NF = CztShape<F>::NF, W = CztColCfg<F>::W;
  extern __shared__ float2 smem[];
  float* gt = reinterpret_cast<float*>(smem + W * CztColCfg<F>::R);   // [F][W]
  const int c = threadIdx.x % W, t = threadIdx.x / W;
  const int col0 = blockIdx.x * W, col = col0 + c;
  const int g = blockIdx.y, b = blockIdx.z;
  const float* Gb = (aa.remap ? aa.Gt : aa.D) + (long long)b * F * F;
  const float scale = 2.0f / (float)F;
  for (int e = threadIdx.x; e < F * W; e += blockDim.x) {
    const int k = e / W, ce = e % W;
    gt[k * W + ce] = Gb[k * F + col0 + ce] * scale;
  }
  __syncthreads();
  const int m0 = g * a.MG, m1 = min(a.chunk_len, m0 + a.MG);
  const float inv = 1.0f / (float)F;
  for (int cm = m0; cm < m1; ++cm) {
    const int l = (a.chunk_base + cm) / a.M;
    float2* base = S + ((long long)b * a.C + cm) * F * F + col;
    float2 v[kCztV];
#pragma unroll
    for (int n2 = 0; n2 < NF; ++n2) v[n2] = base[(long long)(t + N1 * n2) * F];
    czt_vec<F, false>(v, t, smem + c * CztColCfg<F>::R, ct, l, BlockSync{});
#pragma unroll
    for (int n2 = 0; n2 < NF; ++n2) v[n2] = cscale(v[n2], gt[(t + N1 * n2) * W + c]);
    czt_vec<F, true>(v, t, smem + c * CztColCfg<F>::R, ct, l, BlockSync{});
#pragma unroll
    for (int n2 = 0; n2 < NF; ++n2) base[(long long)(t + N1 * n2) * F] = cscale(v[n2], inv);
  }
}

// adjoint rows: chi = Z_r^H row; probe gradient over the batch (kAdjSlots slots added in slot
// order); S <- conj(sigma P) chi per mode for the object-gradient kernel.   grid (F/RPB, chunk_len)
template <int F>
__global__ void __launch_bounds__(CztRowAdjCfg<F>::threads, 1)
k_czt_row_adj(const float2* __restrict__ O, const float2* __restrict__ P, float2* __restrict__ S,
              float2* __restrict__ gP, KArgs a, CztArgs ct) {
  pdl_wait();
  pdl_trigger();
  constexpr int N1 = CztShape<F>::N1, NF = CztShape<F>::NF, T = CztRowAdjCfg<F>::T, RPB = CztRowAdjCfg<F>::RPB;
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
  float2 acc[NF];
#pragma unroll
  for (int n2 = 0; n2 < NF; ++n2) acc[n2] = make_float2(0.f, 0.f);
  float2* xc = smem + vec * CztShape<F>::xch;
  for (int b = slot; b < a.nb; b += kAdjSlots) {
    const int2 yx = spos[b];
    if (yx.x < 0) continue;                           // uniform over the slot's warps
    const float s = ssig[b];
    float2* row = S + (((long long)b * a.C + cm) * F + r) * F;
    const float2* Orow = Ol + (long long)(yx.x + r) * Wl + yx.y;
    float2 v[kCztV];
#pragma unroll
    for (int n2 = 0; n2 < NF; ++n2) v[n2] = row[t + N1 * n2];
    czt_vec<F, true>(v, t, xc, ct, l, WarpSync{});
#pragma unroll
    for (int n2 = 0; n2 < NF; ++n2) {
      const float2 p = __ldg(Orow + t + N1 * n2);
      const float2 gp = cconjmul(p, v[n2]);
      acc[n2].x = fmaf(s, gp.x, acc[n2].x);
      acc[n2].y = fmaf(s, gp.y, acc[n2].y);
      row[t + N1 * n2] = cscale(cconjmul(__ldg(Prow + t + N1 * n2), v[n2]), s);
    }
  }
  __syncthreads();
  float2* red = smem;                                 // [kAdjSlots-1][RPB][F]
  if (slot > 0) {
#pragma unroll
    for (int n2 = 0; n2 < NF; ++n2) red[((slot - 1) * RPB + rr) * F + t + N1 * n2] = acc[n2];
  }
  __syncthreads();
  if (slot == 0) {
    float2* gdst = gP + ((long long)mode * F + r) * F;
#pragma unroll
    for (int n2 = 0; n2 < NF; ++n2) {
      const int cidx = t + N1 * n2;
      float2 sum = acc[n2];
      for (int s2 = 1; s2 < kAdjSlots; ++s2) sum = cadd(sum, red[((s2 - 1) * RPB + rr) * F + cidx]);
      gdst[cidx] = cadd(gdst[cidx], sum);
    }
  }
}

}  // namespace ptycho
