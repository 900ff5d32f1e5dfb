// In-register radix DFTs and the two-stage 1D FFT used by every propagation kernel.
//
// The propagator D_{lambda,z} of Eq. 1 is an orthonormal 2D DFT here (far field).  A 2D
// DFT of an F x F frame is done as F-point 1D FFTs along rows, then along columns; each
// 1D FFT of length F = N1 * N2 is computed by a group of T = N1 threads that each hold
// P = N2 complex values in registers:
//
//   layout "I" (input):  thread t holds x[n], n = t + N1*n2,            slot n2 in [0, N2)
//   layout "O" (output): thread t holds X[k], k = N2*k1 + t + N1*q,     slot q*N1 + k1
//
//   forward  (I -> O):  DFT_N2 over n2 in registers; multiply by W_F^(t*k2);
//                       exchange through shared memory; N2/N1 DFT_N1 over n1.
//   inverse  (O -> I):  exact adjoint of the forward factorisation (conjugate DFT_N1,
//                       reverse exchange, conjugate twiddles, conjugate DFT_N2).
//
// Both directions are unscaled; the 1/F of the orthonormal 2D transform is applied by the
// kernels.  Twiddles between the stages come from a table computed in FP64 on the host.
// Small DFT constants are cos/sin of multiples of 2*pi/32, written out below.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace ptycho {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
// conj(a) * b
__device__ __forceinline__ float2 cconjmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// cos(2*pi*i/32) for i in [0, 8]
__host__ __device__ constexpr double kCos32(int i) {
  return i == 0 ? 1.0
       : i == 1 ? 0.98078528040323044913
       : i == 2 ? 0.92387953251128675613
       : i == 3 ? 0.83146961230254523708
       : i == 4 ? 0.70710678118654752440
       : i == 5 ? 0.55557023301960222474
       : i == 6 ? 0.38268343236508977173
       : i == 7 ? 0.19509032201612826785
       : 0.0;
}
// cos(2*pi*a/32) for any integer a, by symmetry
__host__ __device__ constexpr double cos32(int a) {
  return ((a % 32) + 32) % 32 > 16
             ? cos32(32 - (((a % 32) + 32) % 32))
             : (((a % 32) + 32) % 32 > 8 ? -kCos32(16 - (((a % 32) + 32) % 32))
                                         : kCos32(((a % 32) + 32) % 32));
}
__host__ __device__ constexpr double sin32(int a) { return cos32(8 - a); }

// Compile-time loop: f(std::integral_constant<int, I>) for I in [B, E).
template <int B, int E, class Fn>
__device__ __forceinline__ void static_for(Fn&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    static_for<B + 1, E>(f);
  }
}

// x * W_N^K with W_N = exp(-2*pi*i/N) (forward) or its conjugate (INV); N divides 32.
template <int N, bool INV, int K>
__device__ __forceinline__ float2 twiddle_const(float2 x) {
  constexpr int a = ((K * (32 / N)) % 32 + 32) % 32;
  if constexpr (a == 0) {
    return x;
  } else if constexpr (a == 16) {
    return make_float2(-x.x, -x.y);
  } else if constexpr (a == 8) {            // forward W = -i, inverse W = +i
    return INV ? make_float2(-x.y, x.x) : make_float2(x.y, -x.x);
  } else if constexpr (a == 24) {           // forward W = +i, inverse W = -i
    return INV ? make_float2(x.y, -x.x) : make_float2(-x.y, x.x);
  } else {
    constexpr float c = (float)cos32(a);
    constexpr float s = INV ? (float)sin32(a) : -(float)sin32(a);   // W = c + i*s
    return make_float2(fmaf(x.x, c, -x.y * s), fmaf(x.x, s, x.y * c));
  }
}

// In-place DFT of N values a[0], a[S], ..., a[(N-1)S]; natural order in and out.
template <int N, int S, bool INV>
struct Dft {
  static __device__ __forceinline__ void run(float2* a) {
    float2 e[N / 2], o[N / 2];
#pragma unroll
    for (int k = 0; k < N / 2; ++k) { e[k] = a[(2 * k) * S]; o[k] = a[(2 * k + 1) * S]; }
    Dft<N / 2, 1, INV>::run(e);
    Dft<N / 2, 1, INV>::run(o);
    static_for<0, N / 2>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      const float2 w = twiddle_const<N, INV, k>(o[k]);
      a[k * S] = cadd(e[k], w);
      a[(k + N / 2) * S] = csub(e[k], w);
    });
  }
};
template <int S, bool INV>
struct Dft<4, S, INV> {
  static __device__ __forceinline__ void run(float2* a) {
    const float2 x0 = a[0], x1 = a[S], x2 = a[2 * S], x3 = a[3 * S];
    const float2 s02 = cadd(x0, x2), d02 = csub(x0, x2);
    const float2 s13 = cadd(x1, x3), d13 = csub(x1, x3);
    // forward: X1 = d02 - i d13, X3 = d02 + i d13 ; inverse swaps the signs
    const float2 jd13 = INV ? make_float2(-d13.y, d13.x) : make_float2(d13.y, -d13.x);
    a[0] = cadd(s02, s13);
    a[S] = cadd(d02, jd13);
    a[2 * S] = csub(s02, s13);
    a[3 * S] = csub(d02, jd13);
  }
};
template <int S, bool INV>
struct Dft<2, S, INV> {
  static __device__ __forceinline__ void run(float2* a) {
    const float2 x0 = a[0], x1 = a[S];
    a[0] = cadd(x0, x1);
    a[S] = csub(x0, x1);
  }
};

// Geometry of the two-stage decomposition for each supported frame size.
template <int F> struct FftShape;
template <> struct FftShape<64>  { static constexpr int N1 = 4,  N2 = 16; };
template <> struct FftShape<128> { static constexpr int N1 = 8,  N2 = 16; };
template <> struct FftShape<256> { static constexpr int N1 = 16, N2 = 16; };
template <> struct FftShape<512> { static constexpr int N1 = 16, N2 = 32; };

// Shared-memory exchange buffer of one FFT vector: element (k2, n1) at k2*(N1+1) + n1.
// ``region`` is the stride between vectors; the row kernels use region_rows (vectors of a
// warp share 64-bit banks without conflict), the column kernels region_cols (odd).
template <int F>
struct Xch {
  static constexpr int N1 = FftShape<F>::N1, N2 = FftShape<F>::N2;
  static constexpr int base = N2 * (N1 + 1);
  static constexpr int region_rows = (N1 >= 16) ? base : base + ((N1 - (base % 16)) % 16 + 16) % 16;
  static constexpr int region_cols = base | 1;
  __device__ static __forceinline__ int idx(int k2, int n1) { return k2 * (N1 + 1) + n1; }
};

// x[k2] *= W_F^(t*k2) for k2 in [1, N2) (conjugated with CONJ), from the table tw[k2*N1 + t].
// With 32 values per thread (F = 512) the factor is formed as W^(t*b) * W^(4t*a), k2 = 4a + b,
// so that only the 10 table entries of k2 in {1, 2, 3} and of the multiples of 4 are loaded
// instead of 31 (one extra complex product, about 1 ulp, for the other 21).  Measured: 3.2 %
// faster on the 512^2, 6 x 10 step; with 16 values per thread the same split measured 1.4 %
// slower (256^2), so there every factor comes from the table.
template <int F, bool CONJ>
__device__ __forceinline__ void apply_twiddles(float2 (&x)[FftShape<F>::N2], int t, const float2* __restrict__ tw) {
  constexpr int N1 = FftShape<F>::N1, N2 = FftShape<F>::N2;
  if constexpr (N2 >= 32) {
    float2 wb[4], wa[N2 / 4];
    wb[0] = make_float2(1.f, 0.f);
    wa[0] = make_float2(1.f, 0.f);
#pragma unroll
    for (int b = 1; b < 4; ++b) wb[b] = __ldg(tw + b * N1 + t);
#pragma unroll
    for (int a = 1; a < N2 / 4; ++a) wa[a] = __ldg(tw + 4 * a * N1 + t);
#pragma unroll
    for (int k2 = 1; k2 < N2; ++k2) {
      const int a = k2 >> 2, b = k2 & 3;
      const float2 w = a == 0 ? wb[b] : (b == 0 ? wa[a] : cmul(wa[a], wb[b]));
      x[k2] = CONJ ? cmulc(x[k2], w) : cmul(x[k2], w);
    }
  } else {
#pragma unroll
    for (int k2 = 1; k2 < N2; ++k2) {
      const float2 w = __ldg(tw + k2 * N1 + t);
      x[k2] = CONJ ? cmulc(x[k2], w) : cmul(x[k2], w);
    }
  }
}

// Forward 1D FFT, layout I -> layout O.  ``x`` has N2 slots; ``xc`` is this vector's
// exchange region; ``tw`` is the table W_F^(t*k2) stored as tw[k2*N1 + t], so the N1 threads of
// one vector read a contiguous run.  SYNC is the barrier
// used between the exchange write and read (warp or block).
template <int F, class Sync>
__device__ __forceinline__ void fft_fwd_I2O(float2 (&x)[FftShape<F>::N2], int t, float2* xc,
                                            const float2* __restrict__ tw, Sync sync) {
  constexpr int N1 = FftShape<F>::N1, N2 = FftShape<F>::N2;
  Dft<N2, 1, false>::run(x);
  apply_twiddles<F, false>(x, t, tw);
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) xc[Xch<F>::idx(k2, t)] = x[k2];
  sync();
#pragma unroll
  for (int q = 0; q < N2 / N1; ++q)
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) x[q * N1 + n1] = xc[Xch<F>::idx(t + N1 * q, n1)];
  sync();  // the region may be reused by the caller right away
#pragma unroll
  for (int q = 0; q < N2 / N1; ++q) Dft<N1, 1, false>::run(x + q * N1);
}

// Inverse (adjoint, unscaled) 1D FFT, layout O -> layout I.
template <int F, class Sync>
__device__ __forceinline__ void fft_inv_O2I(float2 (&x)[FftShape<F>::N2], int t, float2* xc,
                                            const float2* __restrict__ tw, Sync sync) {
  constexpr int N1 = FftShape<F>::N1, N2 = FftShape<F>::N2;
#pragma unroll
  for (int q = 0; q < N2 / N1; ++q) Dft<N1, 1, true>::run(x + q * N1);
#pragma unroll
  for (int q = 0; q < N2 / N1; ++q)
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) xc[Xch<F>::idx(t + N1 * q, n1)] = x[q * N1 + n1];
  sync();
#pragma unroll
  for (int k2 = 0; k2 < N2; ++k2) x[k2] = xc[Xch<F>::idx(k2, t)];
  sync();
  apply_twiddles<F, true>(x, t, tw);
  Dft<N2, 1, true>::run(x);
}

// The same two transforms for N2 = 2 N1 (F = 512) with an exchange region of half the size: the
// transpose goes in two halves (rows k2 < N1, then k2 >= N1), two more barriers per transform.
// ``xc`` holds N1 x (N1 + 1) elements (XchHalf<F>).  Same arithmetic, same results.
template <int F>
struct XchHalf {
  static constexpr int N1 = FftShape<F>::N1;
  static constexpr int region_cols = (N1 * (N1 + 1)) | 1;
};

template <int F, class Sync>
__device__ __forceinline__ void fft_fwd_I2O_half(float2 (&x)[FftShape<F>::N2], int t, float2* xc,
                                                 const float2* __restrict__ tw, Sync sync) {
  constexpr int N1 = FftShape<F>::N1, N2 = FftShape<F>::N2;
  static_assert(N2 == 2 * N1, "two halves of N1 rows");
  Dft<N2, 1, false>::run(x);
  apply_twiddles<F, false>(x, t, tw);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
#pragma unroll
    for (int k = 0; k < N1; ++k) xc[k * (N1 + 1) + t] = x[h * N1 + k];       // rows k2 = h*N1 + k
    sync();
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) x[h * N1 + n1] = xc[t * (N1 + 1) + n1];  // row k2 = t + N1*h
    sync();
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) Dft<N1, 1, false>::run(x + q * N1);
}

template <int F, class Sync>
__device__ __forceinline__ void fft_inv_O2I_half(float2 (&x)[FftShape<F>::N2], int t, float2* xc,
                                                 const float2* __restrict__ tw, Sync sync) {
  constexpr int N1 = FftShape<F>::N1, N2 = FftShape<F>::N2;
  static_assert(N2 == 2 * N1, "two halves of N1 rows");
#pragma unroll
  for (int q = 0; q < 2; ++q) Dft<N1, 1, true>::run(x + q * N1);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) xc[t * (N1 + 1) + n1] = x[h * N1 + n1];  // row k2 = t + N1*h
    sync();
#pragma unroll
    for (int k = 0; k < N1; ++k) x[h * N1 + k] = xc[k * (N1 + 1) + t];       // rows k2 = h*N1 + k
    sync();
  }
  apply_twiddles<F, true>(x, t, tw);
  Dft<N2, 1, true>::run(x);
}

// Inverse (unscaled, the adjoint of the forward DFT) 512-point transform by a whole warp, 16 values
// per lane, for kernels that hold a spectrum row in shared memory in natural order.  With
// n = t + 32 n2 and k = c + 16 k1 (t, lane in [0, 32); c, n2 in [0, 16); k1 in [0, 32)):
//   x[t + 32 n2] = sum_c W16^(-n2 c) W512^(-t c) sum_k1 X[c + 16 k1] W32^(-t k1).
// The inner 32-point sum is split by the parity q of k1 = 2 s + q: lane u = c + 16 q takes the 16
// spectrum values X[u + 32 s] (a 16-point inverse DFT over s), lanes with q = 1 apply W32^(-j),
// and the pair (u, u ^ 16) combines E + T and E - T through a shuffle, giving Y[c][t] for
// t = j + 16 q.  Each element is multiplied by W512^(-t c) (the F = 512 table entry tw[t*16 + c]),
// the 16 x 32 block is transposed through ``xc`` (element (c, t) at c*33 + t: conflict-free in
// both directions), and lane t takes a 16-point inverse DFT over c.  ``spec`` may alias ``xc``
// (the spectrum is read before the first write).  Out: x[n2] = value at n = lane + 32 n2.
__device__ __forceinline__ void fft512_inv_warp(const float2* spec, float2 (&x)[16], int lane, float2* xc,
                                                const float2* __restrict__ tw) {
  constexpr int R = 33;
  const int c = lane & 15, q = lane >> 4;
#pragma unroll
  for (int s = 0; s < 16; ++s) x[s] = spec[lane + 32 * s];
  __syncwarp();                                       // spec may be xc
  Dft<16, 1, true>::run(x);
  if (q) {
    static_for<1, 16>([&](auto jc) {
      constexpr int j = decltype(jc)::value;
      x[j] = twiddle_const<32, true, j>(x[j]);
    });
  }
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const float ox = __shfl_xor_sync(0xffffffffu, x[j].x, 16), oy = __shfl_xor_sync(0xffffffffu, x[j].y, 16);
    x[j] = q ? make_float2(ox - x[j].x, oy - x[j].y) : make_float2(x[j].x + ox, x[j].y + oy);
  }
  // W512^(-t c) before the transpose: lane (c, q) reads tw[t*16 + c], t = j + 16 q, two
  // contiguous 128-byte runs per warp load (after the transpose the same factors would be a
  // 128-byte stride across the lanes)
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if (j > 0 || q) x[j] = cmulc(x[j], __ldg(tw + (j + 16 * q) * 16 + c));
    xc[c * R + j + 16 * q] = x[j];
  }
  __syncwarp();
#pragma unroll
  for (int k = 0; k < 16; ++k) x[k] = xc[k * R + lane];
  __syncwarp();                                       // the region may be reused right away
  Dft<16, 1, true>::run(x);
}
constexpr int kFft512WarpXch = 16 * 33;               // exchange elements of fft512_inv_warp

// Forward 512-point transform by a whole warp, the mirror of fft512_inv_warp.  In: x[n2] = value
// at n = lane + 32 n2.  With k = c + 16 k1 and n = t + 32 n2:
//   X[c + 16 k1] = sum_t W32^(t k1) W512^(t c) sum_n2 x[t + 32 n2] W16^(n2 c).
// Lane t takes the 16-point DFT over n2 (A[t][c]); A is transposed through ``xc`` (element
// (t, c) at t*17 + c); lane (c, q), q = lane >> 4, takes A[2 s + q][c] W512^((2 s + q) c) for
// s in [0, 16) (table entry tw[(2 s + q)*16 + c], contiguous over the warp), a 16-point DFT over
// s, W32^j on the q = 1 lanes and the butterfly with lane ^ 16.  Out: lane (c, q) holds
// X[c + 16 j + 256 q] in x[j] (for each j the warp covers two contiguous 16-element runs).
__device__ __forceinline__ void fft512_fwd_warp(float2 (&x)[16], int lane, float2* xc, const float2* __restrict__ tw) {
  constexpr int R = 17;
  const int c = lane & 15, q = lane >> 4;
  Dft<16, 1, false>::run(x);
#pragma unroll
  for (int k = 0; k < 16; ++k) xc[lane * R + k] = x[k];
  __syncwarp();
#pragma unroll
  for (int s = 0; s < 16; ++s) {
    const int t = 2 * s + q;
    x[s] = xc[t * R + c];
    if (s > 0 || q) x[s] = cmul(x[s], __ldg(tw + t * 16 + c));
  }
  __syncwarp();                                       // the region may be reused right away
  Dft<16, 1, false>::run(x);
  if (q) {
    static_for<1, 16>([&](auto jc) {
      constexpr int j = decltype(jc)::value;
      x[j] = twiddle_const<32, false, j>(x[j]);
    });
  }
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const float ox = __shfl_xor_sync(0xffffffffu, x[j].x, 16), oy = __shfl_xor_sync(0xffffffffu, x[j].y, 16);
    x[j] = q ? make_float2(ox - x[j].x, oy - x[j].y) : make_float2(x[j].x + ox, x[j].y + oy);
  }
}
constexpr int kFft512WarpXchF = 32 * 17;              // exchange elements of fft512_fwd_warp

// Index helpers for the two layouts.
template <int F> __device__ __forceinline__ int idxI(int t, int n2) { return t + FftShape<F>::N1 * n2; }
template <int F> __device__ __forceinline__ int idxO(int t, int slot) {
  constexpr int N1 = FftShape<F>::N1, N2 = FftShape<F>::N2;
  return N2 * (slot % N1) + t + N1 * (slot / N1);
}

struct WarpSync { __device__ __forceinline__ void operator()() const { __syncwarp(); } };
struct BlockSync { __device__ __forceinline__ void operator()() const { __syncthreads(); } };

}  // namespace ptycho
