// Frame-resident forward and adjoint passes for F <= 128 (propagation f4 of Eq. 2 and its
// adjoint, Fig. 1B): one thread block holds a whole F x F field in shared memory, so neither
// the exit wave psi = sigma P p nor its spectrum Psi nor the back-propagated chi ever leaves the
// SM.  A 64^2 complex64 frame is 32 KB and a 128^2 frame 128 KB, both inside one SM's 227 KB.
//
// The 2D DFT is the row/column factorisation of the register FFT (fft_regs.cuh): 64 vectors of
// N1 threads at a time (256 threads at F = 64, 512 at F = 128), each vector one row or one column
// of the frame.  Rows and columns move between registers and the frame; the two-stage exchange
// of each 1D FFT goes through a separate per-vector area (warp-synchronous: the N1 threads of a
// vector share a warp in both passes).  The frame rows have a pitch of F + 4 complex values so
// that the 8-byte accesses of both passes (four or eight rows of a warp at once) spread over the
// 32 banks.
//
// Selected by PTYCHO_FLAG_RESIDENT_FRAMES.  Measured on a GB300 at 0.5-0.9x the speed of the
// default scratch passes: both forms are bound by the shared-memory / L1 pipe of the 1D FFTs
// (the scratch passes already overlap their HBM traffic across three streams), a 128^2 frame
// leaves room for one 16-warp block per SM, and the adjoint recomputes Psi (three 2D DFTs per
// evaluation instead of two).
//
//   k_res_fwd   grid (nb, G): position b, mode group g.  For each mode of the group: psi row by
//               row -> row DFT -> frame; column DFT -> |Psi|^2 summed in registers over the
//               group's modes; the sum (times 1/F^2) goes to Ipart[b][g], the same slice layout
//               the scratch pipeline's column pass leaves for the loss kernel.
//   k_res_adj   grid (L*M, nsplit): probe mode (l, m), a contiguous split of the batch's
//               positions.  Per position: psi -> row DFT -> column DFT (Psi recomputed on chip)
//               -> times (2/F^2) G -> inverse column DFT -> inverse row DFT = chi; the probe
//               gradient conj(sigma p) chi is summed over the split's positions (registers at
//               F = 64; the split's own buffer at F = 128, where the registers are taken by the
//               transform) and the mode's object-gradient patch conj(sigma P) chi goes to the
//               scratch slot S[b][l*M + m] that the object-gradient kernel reads.  chi goes back
//               to the frame first, so that these products run element by element with
//               consecutive threads on consecutive columns.
#pragma once
#include "kernels.cuh"

namespace ptycho {

template <int F> struct ResCfg {
  static constexpr int N1 = FftShape<F>::N1, N2 = FftShape<F>::N2;
  static constexpr int VPR = 64;                                   // vectors per round
  static constexpr int threads = VPR * N1;                         // 256 (F = 64), 512 (F = 128)
  static constexpr int rounds = F / VPR;                           // rows (columns) per vector
  static constexpr int pitch = F + 4;                              // complex values per frame row
  static constexpr int frame = F * pitch;                          // complex values
  static constexpr int xch = VPR * Xch<F>::region_rows;            // complex values
  static constexpr int smem = (frame + xch) * (int)sizeof(float2);
  static constexpr int min_blocks = F <= 64 ? 2 : 1;
  static constexpr int per_thread = F * F / threads;               // frame elements per thread
};

template <int F> struct ResSupported { static constexpr bool value = F <= 128; };

// Row DFTs of psi = s * P_mode * O-patch (rows v + 64*rho of the frame), written to the frame in
// natural frequency order (slot sl of thread t holds frequency idxO(t, sl)).
template <int F>
__device__ __forceinline__ void res_rows_fwd(const float2* __restrict__ Pm, const float2* __restrict__ Op, int Wo,
                                             float s, float2* fr, float2* xc, const float2* __restrict__ tw, int v,
                                             int t) {
  using C = ResCfg<F>;
  constexpr int N1 = C::N1, N2 = C::N2;
#pragma unroll
  for (int rho = 0; rho < C::rounds; ++rho) {
    const int r = v + C::VPR * rho;
    const float2* Prow = Pm + (long long)r * F;
    const float2* Orow = Op + (long long)r * Wo;
    float2 z[N2];
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) z[n2] = cmul(__ldg(Prow + t + N1 * n2), cscale(__ldg(Orow + t + N1 * n2), s));
    fft_fwd_I2O<F>(z, t, xc, tw, WarpSync{});
#pragma unroll
    for (int sl = 0; sl < N2; ++sl) fr[r * C::pitch + idxO<F>(t, sl)] = z[sl];
  }
}

// grid (nb, G), block ResCfg<F>::threads, dynamic smem ResCfg<F>::smem
template <int F>
__global__ void __launch_bounds__(ResCfg<F>::threads, ResCfg<F>::min_blocks)
k_res_fwd(const float2* __restrict__ O, const float2* __restrict__ P, float* __restrict__ Ipart, KArgs a) {
  pdl_wait();
  pdl_trigger();
  using C = ResCfg<F>;
  constexpr int N1 = C::N1, N2 = C::N2, R = C::rounds;
  extern __shared__ float2 smem[];
  float2* fr = smem;
  const int v = threadIdx.x / N1, t = threadIdx.x % N1;
  float2* xc = smem + C::frame + v * Xch<F>::region_rows;
  const int b = blockIdx.x, g = blockIdx.y;
  const int m0 = g * a.MG, m1 = min(a.chunk_len, m0 + a.MG);
  const int j = batch_pos(a, a.batch_off + b);       // uniform over the block
  float acc[R][N2];
#pragma unroll
  for (int rho = 0; rho < R; ++rho)
#pragma unroll
    for (int sl = 0; sl < N2; ++sl) acc[rho][sl] = 0.f;
  if (j >= 0) {
    const float s = sigma_of(a, j);
    for (int cm = m0; cm < m1; ++cm) {
      const int mode = a.chunk_base + cm, l = mode / a.M;
      const int y = a.pos[(l * a.J + j) * 2], x = a.pos[(l * a.J + j) * 2 + 1];
      res_rows_fwd<F>(P + (long long)mode * F * F, O + a.obj_off[l] + (long long)y * a.obj_w[l] + x, a.obj_w[l], s,
                      fr, xc, a.tw, v, t);
      __syncthreads();
#pragma unroll
      for (int rho = 0; rho < R; ++rho) {
        const int c = v + C::VPR * rho;
        float2 z[N2];
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) z[n2] = fr[(t + N1 * n2) * C::pitch + c];
        fft_fwd_I2O<F>(z, t, xc, a.tw, WarpSync{});
#pragma unroll
        for (int sl = 0; sl < N2; ++sl) acc[rho][sl] = fmaf(z[sl].x, z[sl].x, fmaf(z[sl].y, z[sl].y, acc[rho][sl]));
      }
      __syncthreads();                                // the frame is rewritten by the next mode
    }
  }
  float* dst = Ipart + ((long long)b * a.G + g) * F * F;
  constexpr float inv2 = 1.0f / (float)(F * F);
#pragma unroll
  for (int rho = 0; rho < R; ++rho) {
    const int cc = (v + C::VPR * rho + F / 2) & (F - 1);
#pragma unroll
    for (int sl = 0; sl < N2; ++sl) dst[((idxO<F>(t, sl) + F / 2) & (F - 1)) * F + cc] = acc[rho][sl] * inv2;
  }
}

// grid (chunk_len, nsplit), block ResCfg<F>::threads, dynamic smem ResCfg<F>::smem.
// gPs + split * gp_stride is the split's probe-gradient buffer ([L*M][F][F], read-modify-write).
template <int F>
__global__ void __launch_bounds__(ResCfg<F>::threads, ResCfg<F>::min_blocks)
k_res_adj(const float2* __restrict__ O, const float2* __restrict__ P, float2* __restrict__ S, float2* __restrict__ gPs,
          long long gp_stride, KArgs a, AdjArgs aa, int nsplit) {
  pdl_wait();
  pdl_trigger();
  using C = ResCfg<F>;
  constexpr int N1 = C::N1, N2 = C::N2, R = C::rounds;
  constexpr bool kRegAcc = F <= 64;                   // probe-gradient sums in registers
  extern __shared__ float2 smem[];
  __shared__ int2 spos[kMaxB];
  __shared__ float ssig[kMaxB];
  float2* fr = smem;
  const int v = threadIdx.x / N1, t = threadIdx.x % N1;
  float2* xc = smem + C::frame + v * Xch<F>::region_rows;
  const int cm = blockIdx.x, split = blockIdx.y;
  const int mode = a.chunk_base + cm, l = mode / a.M;
  stage_batch(a, l, spos, ssig);
  const int b0 = (int)(((long long)split * a.nb) / nsplit), b1 = (int)(((long long)(split + 1) * a.nb) / nsplit);
  const float2* Pm = P + (long long)mode * F * F;
  const float2* Ol = O + a.obj_off[l];
  const int Wl = a.obj_w[l];
  const float* Gall = aa.remap ? aa.Gt : aa.D;
  float2* gP = gPs + split * gp_stride + (long long)mode * F * F;
  constexpr float gscale = 2.0f / (float)(F * F);     // 2/F for the gradient, 1/F for the recomputed Psi
  float2 gacc[kRegAcc ? C::per_thread : 1];
  if constexpr (kRegAcc) {
#pragma unroll
    for (int k = 0; k < C::per_thread; ++k) gacc[k] = make_float2(0.f, 0.f);
  }
  for (int b = b0; b < b1; ++b) {
    const int2 yx = spos[b];
    if (yx.x < 0) continue;                           // uniform over the block
    const float s = ssig[b];
    const float2* Op = Ol + (long long)yx.x * Wl + yx.y;
    res_rows_fwd<F>(Pm, Op, Wl, s, fr, xc, a.tw, v, t);
    __syncthreads();
    const float* Gb = Gall + (long long)b * F * F;
#pragma unroll
    for (int rho = 0; rho < R; ++rho) {
      const int c = v + C::VPR * rho;
      const int cc = (c + F / 2) & (F - 1);
      float2 z[N2];
#pragma unroll
      for (int n2 = 0; n2 < N2; ++n2) z[n2] = fr[(t + N1 * n2) * C::pitch + c];
      fft_fwd_I2O<F>(z, t, xc, a.tw, WarpSync{});
#pragma unroll
      for (int sl = 0; sl < N2; ++sl)
        z[sl] = cscale(z[sl], __ldg(Gb + ((idxO<F>(t, sl) + F / 2) & (F - 1)) * F + cc) * gscale);
      fft_inv_O2I<F>(z, t, xc, a.tw, WarpSync{});
#pragma unroll
      for (int n2 = 0; n2 < N2; ++n2) fr[(t + N1 * n2) * C::pitch + c] = z[n2];
    }
    __syncthreads();
    float2* Sb = S + ((long long)b * a.C + cm) * F * F;
#pragma unroll
    for (int rho = 0; rho < R; ++rho) {
      const int r = v + C::VPR * rho;
      float2 z[N2];
#pragma unroll
      for (int sl = 0; sl < N2; ++sl) z[sl] = fr[r * C::pitch + idxO<F>(t, sl)];
      fft_inv_O2I<F>(z, t, xc, a.tw, WarpSync{});       // chi = dL/dpsi of row r, natural order
#pragma unroll
      for (int n2 = 0; n2 < N2; ++n2) fr[r * C::pitch + t + N1 * n2] = z[n2];
    }
    __syncthreads();
    // both gradients element by element (consecutive threads on consecutive columns)
    auto grads = [&](int k) {
      const int e = threadIdx.x + k * C::threads;
      const int r = e / F, cidx = e % F;
      const float2 chi = fr[r * C::pitch + cidx];
      const float2 gp = cscale(cconjmul(__ldg(Op + (long long)r * Wl + cidx), chi), s);   // conj(sigma p) chi
      if constexpr (kRegAcc) {
        gacc[k] = cadd(gacc[k], gp);
      } else {
        gP[e] = cadd(gP[e], gp);
      }
      Sb[e] = cscale(cconjmul(__ldg(Pm + e), chi), s);                                   // conj(sigma P) chi
    };
    if constexpr (kRegAcc) {
#pragma unroll
      for (int k = 0; k < C::per_thread; ++k) grads(k);
    } else {
#pragma unroll 4
      for (int k = 0; k < C::per_thread; ++k) grads(k);
    }
    __syncthreads();                                  // the frame is rewritten by the next position
  }
  if constexpr (kRegAcc) {
#pragma unroll
    for (int k = 0; k < C::per_thread; ++k) {
      const int e = threadIdx.x + k * C::threads;
      gP[e] = cadd(gP[e], gacc[k]);
    }
  }
}

}  // namespace ptycho
