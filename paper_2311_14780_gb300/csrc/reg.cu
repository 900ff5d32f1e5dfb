// Object regularisation: L1 and total variation of the object amplitude, the regularisers
// the paper names (Section "3D structure information characterisation"), added to the loss
// as the paper adapts the loss for regularised optimisation (Section "Universal Ptychography
// Algorithm").  With the smoothed amplitude a = sqrt(|O|^2 + eta^2) of every object pixel,
//   R = mu_l1 sum a + mu_tv sum sqrt(dx^2 + dy^2 + eta^2),
//   dx = a[r][c+1] - a[r][c] (0 in the last column), dy = a[r+1][c] - a[r][c] (0 in the last row),
// and, with g = dR/dRe + i dR/dIm = (dR/da) O / a,
//   dR/da[r][c] = mu_l1 + mu_tv (-(dx + dy)/t [r][c] + dx/t [r][c-1] + dy/t [r-1][c]).
//
// One block owns a kRegTX x kRegTY tile of one object, kRegRows rows per thread.  It stages the
// amplitudes of the tile and a one-pixel halo in shared memory, forms dx/t and dy/t for the tile
// and its upper and left halo, then every thread adds its pixels' gradients into gO (each pixel
// has one owner: no atomics) and the block's share of R goes to a per-tile FP64 partial; a second
// kernel adds the partials to the loss in a fixed order.  HBM-bound: O read, gO read and
// written, 24 B per pixel.
#include <math.h>

#include "plan.h"

namespace ptycho {
namespace {

constexpr int kRegTX = 32, kRegTY = 32;          // tile: columns x rows
constexpr int kRegRows = 4;                      // rows per thread (threads: kRegTX x kRegTY / kRegRows)
constexpr int kRegThreads = kRegTX * kRegTY / kRegRows;

struct RegArgs {
  const float2* O;
  float2* gO;
  long long off[kMaxL];
  int h[kMaxL], w[kMaxL];
  float mu1, mutv, eta;
  double* part;                                   // [L][max_tiles]
  int max_tiles;
};

// grid (max_tiles, L), block kRegThreads
__global__ void __launch_bounds__(kRegThreads) k_reg(RegArgs r) {
  __shared__ float as[kRegTY + 2][kRegTX + 2];    // pixel (r0 - 1 + i, c0 - 1 + j) at [i][j]
  __shared__ float qx[kRegTY + 1][kRegTX + 1];    // dx/t of pixel (r0 - 1 + i, c0 - 1 + j)
  __shared__ float qy[kRegTY + 1][kRegTX + 1];
  __shared__ double red[kRegThreads / 32];
  const int l = blockIdx.y, H = r.h[l], W = r.w[l];
  const int tx = (W + kRegTX - 1) / kRegTX, ntiles = tx * ((H + kRegTY - 1) / kRegTY);
  const int tile = blockIdx.x;
  double* part = r.part + (long long)l * r.max_tiles + tile;
  if (tile >= ntiles) {                           // uniform over the block
    if (threadIdx.x == 0) *part = 0.0;
    return;
  }
  const int r0 = (tile / tx) * kRegTY, c0 = (tile % tx) * kRegTX;
  const float2* Ol = r.O + r.off[l];
  const float e2 = r.eta * r.eta;
  for (int e = threadIdx.x; e < (kRegTY + 2) * (kRegTX + 2); e += kRegThreads) {
    const int i = e / (kRegTX + 2), j = e % (kRegTX + 2);
    const int rr = r0 - 1 + i, cc = c0 - 1 + j;
    float v = 0.f;
    if (rr >= 0 && rr < H && cc >= 0 && cc < W) {
      const float2 o = Ol[(long long)rr * W + cc];
      v = sqrtf(fmaf(o.x, o.x, fmaf(o.y, o.y, e2)));
    }
    as[i][j] = v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < (kRegTY + 1) * (kRegTX + 1); e += kRegThreads) {
    const int i = e / (kRegTX + 1), j = e % (kRegTX + 1);
    const int rr = r0 - 1 + i, cc = c0 - 1 + j;
    float px = 0.f, py = 0.f;
    if (rr >= 0 && rr < H && cc >= 0 && cc < W) {
      const float a = as[i][j];
      const float dx = cc + 1 < W ? as[i][j + 1] - a : 0.f;
      const float dy = rr + 1 < H ? as[i + 1][j] - a : 0.f;
      const float t = sqrtf(fmaf(dx, dx, fmaf(dy, dy, e2)));
      px = dx / t;
      py = dy / t;
    }
    qx[i][j] = px;
    qy[i][j] = py;
  }
  __syncthreads();
  const int tc = threadIdx.x % kRegTX, ty0 = threadIdx.x / kRegTX;
  const int cc = c0 + tc;
  double term = 0.0;
#pragma unroll
  for (int k = 0; k < kRegRows; ++k) {
    const int ty = ty0 + k * (kRegThreads / kRegTX);
    const int rr = r0 + ty;
    if (rr < H && cc < W) {
      const int i = ty + 1, j = tc + 1;
      const float a = as[i][j];
      const float dx = cc + 1 < W ? as[i][j + 1] - a : 0.f;
      const float dy = rr + 1 < H ? as[i + 1][j] - a : 0.f;
      const float t = sqrtf(fmaf(dx, dx, fmaf(dy, dy, e2)));
      const float dRda = r.mu1 + r.mutv * ((qx[i][j - 1] + qy[i - 1][j]) - (qx[i][j] + qy[i][j]));
      const long long idx = r.off[l] + (long long)rr * W + cc;
      const float2 o = Ol[(long long)rr * W + cc];
      const float s = dRda / a;
      const float2 g = r.gO[idx];
      r.gO[idx] = make_float2(fmaf(s, o.x, g.x), fmaf(s, o.y, g.y));
      term += (double)(r.mu1 * a) + (double)(r.mutv * t);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) term += __shfl_down_sync(0xffffffffu, term, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = term;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < kRegThreads / 32; ++k) s += red[k];
    *part = s;
  }
}

// *out += sum of the n partials (fixed order: a strided sum per thread, then a tree).
__global__ void __launch_bounds__(256) k_reg_reduce(const double* __restrict__ part, long long n, double* out) {
  __shared__ double red[256];
  double s = 0.0;
  for (long long i = threadIdx.x; i < n; i += 256) s += part[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out += red[0];
}

}  // namespace

bool reg_args_ok(float mu_l1, float mu_tv, float eta) {
  return isfinite(mu_l1) && isfinite(mu_tv) && isfinite(eta) && mu_l1 >= 0.f && mu_tv >= 0.f && eta > 0.f;
}

// Adds R to *loss (if not null) and dR to gO, on stream st.  Allocates the per-tile partials
// on first use.
int regularise(ptycho_plan& p, const float2* O, float mu_l1, float mu_tv, float eta, float2* gO, double* loss,
               cudaStream_t st) {
  if (mu_l1 == 0.f && mu_tv == 0.f) return PTYCHO_OK;
  int max_tiles = 0;
  for (int l = 0; l < p.L; ++l)
    max_tiles = std::max(max_tiles, ((p.obj_w[l] + kRegTX - 1) / kRegTX) * ((p.obj_h[l] + kRegTY - 1) / kRegTY));
  const long long n = (long long)p.L * max_tiles;
  if (n > p.reg_cap) {
    if (p.d_reg_part) cudaFree(p.d_reg_part);
    p.d_reg_part = nullptr;
    p.reg_cap = 0;
    if (cudaMalloc((void**)&p.d_reg_part, (size_t)n * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      p.d_reg_part = nullptr;
      return PTYCHO_ENOMEM;
    }
    p.reg_cap = n;
    p.bytes += n * (long long)sizeof(double);
  }
  RegArgs r;
  r.O = O;
  r.gO = gO;
  for (int l = 0; l < kMaxL; ++l) {
    r.off[l] = l < p.L ? p.obj_off[l] : 0;
    r.h[l] = l < p.L ? p.obj_h[l] : 0;
    r.w[l] = l < p.L ? p.obj_w[l] : 0;
  }
  r.mu1 = mu_l1;
  r.mutv = mu_tv;
  r.eta = eta;
  r.part = p.d_reg_part;
  r.max_tiles = max_tiles;
  long long ev = prof_begin(p, kReg, st);
  k_reg<<<dim3((unsigned)max_tiles, (unsigned)p.L), kRegThreads, 0, st>>>(r);
  ++p.last_launches;
  if (loss) {
    k_reg_reduce<<<1, 256, 0, st>>>(p.d_reg_part, n, loss);
    ++p.last_launches;
  }
  prof_end(p, ev, st);
  return cudaGetLastError() == cudaSuccess ? PTYCHO_OK : PTYCHO_ECUDA;
}

}  // namespace ptycho

extern "C" int ptycho_regularise(ptycho_plan_t* p, const float* O, float mu_l1, float mu_tv, float eta, float* gO,
                                 double* loss_dev, void* stream) {
  if (!p || !O || !gO || !ptycho::reg_args_ok(mu_l1, mu_tv, eta)) return PTYCHO_EINVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return PTYCHO_ECUDA;
  if (dev != p->dev) return PTYCHO_EINVAL;
  p->last_launches = 0;
  return ptycho::regularise(*p, reinterpret_cast<const float2*>(O), mu_l1, mu_tv, eta, reinterpret_cast<float2*>(gO),
                            loss_dev, static_cast<cudaStream_t>(stream));
}
