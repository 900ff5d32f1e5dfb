// C-ABI front end: geometry and position validation, the tilted-plane remap tables, the
// batching decision, workspace allocation and dispatch to the frame-size pipelines.
#include <math.h>

#include <algorithm>
#include <new>
#include <vector>

#include <cudaTypedefs.h>

#include "plan.h"

namespace ptycho {

// Fixed-order FP64 sum of the per-block loss partials (one block).
__global__ void __launch_bounds__(256) k_loss_reduce(const double* __restrict__ part, long long n, double* out) {
  pdl_wait();
  __shared__ double red[256];
  double s = 0.0;
  for (long long i = threadIdx.x; i < n; i += 256) s += part[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// Gradient of the power coefficients.  sigma_j multiplies every exit wave of frame j (f1),
// and the DFT is unitary, so sum_r conj(psi) chi = 2 sum_k G_k |Psi_k|^2 and
// dL/dsigma_j = (2 / sigma_j) sum over the camera grid of D * (R sum_lm |Psi_lm|^2), the
// quantity the loss kernel left per block in part.  One thread per position j sums, in
// entry order, the partials of every call entry i with bidx[i] = j; positions outside the
// call (and sigma_j = 0, where the derivative vanishes) get 0.
__global__ void __launch_bounds__(256)
k_sigma_grad(const int32_t* __restrict__ bidx, int nbatch, int J, const double* __restrict__ part, int nblk,
             const float* __restrict__ sigma, float* __restrict__ g) {
  pdl_wait();
  const int j = blockIdx.x * 256 + threadIdx.x;
  if (j >= J) return;
  double s = 0.0;
  for (int i = 0; i < nbatch; ++i) {
    if (__ldg(bidx + i) != j) continue;
    for (int k = 0; k < nblk; ++k) s += part[(long long)i * nblk + k];
  }
  const float sj = sigma ? __ldg(sigma + j) : 1.0f;
  g[j] = sj != 0.f ? (float)(2.0 * s / (double)sj) : 0.f;
}

__global__ void __launch_bounds__(256)
k_delta_grad(const int32_t* __restrict__ bidx, int nbatch, int L, int J, const double* __restrict__ dpart,
             int nstrips, float* __restrict__ g_delta) {
  pdl_wait();
  const int e = blockIdx.x * 256 + threadIdx.x;       // e = l*J + j
  if (e >= L * J) return;
  const int l = e / J, j = e % J;
  double sy = 0.0, sx = 0.0;
  for (int i = 0; i < nbatch; ++i) {
    if (__ldg(bidx + i) != j) continue;
    const double* d = dpart + ((long long)i * L + l) * nstrips * 2;
    for (int k = 0; k < nstrips; ++k) {
      sy += d[2 * k];
      sx += d[2 * k + 1];
    }
  }
  g_delta[2 * e] = (float)sy;
  g_delta[2 * e + 1] = (float)sx;
}

// out[i] = sum over the probe-gradient splits, in split order, of part[s][i].
__global__ void __launch_bounds__(256)
k_sum_splits(const float2* __restrict__ part, int nsplit, long long n, float2* __restrict__ out) {
  pdl_wait();
  for (long long i = blockIdx.x * 256ll + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
    float2 s = part[i];
    for (int k = 1; k < nsplit; ++k) s = cadd(s, part[(long long)k * n + i]);
    out[i] = s;
  }
}

// out[u] = sum over the scratch sets, in set order, of acc[set][u].
__global__ void __launch_bounds__(256)
k_sum_sets(const float* __restrict__ acc, int nsets, long long n, float* __restrict__ out) {
  pdl_wait();
  for (long long u = blockIdx.x * 256ll + threadIdx.x; u < n; u += (long long)gridDim.x * 256) {
    float s = 0.f;
    for (int k = 0; k < nsets; ++k) s += acc[(long long)k * n + u];
    out[u] = s;
  }
}

// Adam (Kingma & Ba) on real parameters; c1, c2 are the bias corrections 1/(1-beta^t).
__global__ void __launch_bounds__(256)
k_adam(float* __restrict__ theta, const float* __restrict__ grad, float* __restrict__ m, float* __restrict__ v,
       long long n, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float g = grad[i];
    const float mi = fmaf(b1, m[i], (1.f - b1) * g);
    const float vi = fmaf(b2, v[i], (1.f - b2) * g * g);
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  }
}

// step counter += 1 (one thread): the Adam bias correction of a replayed graph reads it
__global__ void k_tick(int* t) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *t += 1;
}

// Adam with the step counter read on the device (for graph replays).
__global__ void __launch_bounds__(256)
k_adam_dev(float* __restrict__ theta, const float* __restrict__ grad, float* __restrict__ m, float* __restrict__ v,
           long long n, float lr, float b1, float b2, float eps, const int* __restrict__ t_dev) {
  const float t = (float)(*t_dev);
  const float c1 = 1.0f / (1.0f - powf(b1, t));
  const float c2 = 1.0f / (1.0f - powf(b2, t));
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float g = grad[i];
    const float mi = fmaf(b1, m[i], (1.f - b1) * g);
    const float vi = fmaf(b2, v[i], (1.f - b2) * g * g);
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  }
}


long long prof_begin(ptycho_plan& p, int kind, cudaStream_t st) {
  if (!p.prof) return -1;
  const size_t i = p.ev_used;
  while (p.ev_pool.size() < 2 * (i + 1)) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    p.ev_pool.push_back(e);
  }
  p.ev_used = i + 1;
  p.ev_kind.resize(p.ev_used);
  p.ev_kind[i] = kind;
  cudaEventRecord(p.ev_pool[2 * i], st);
  return (long long)i;
}

void prof_end(ptycho_plan& p, long long idx, cudaStream_t st) {
  if (idx >= 0) cudaEventRecord(p.ev_pool[2 * idx + 1], st);
}

}  // namespace ptycho

using ptycho::CallArgs;
using ptycho::CallKind;

namespace {

// The default batching: about kBatchEvals evaluations per batch, but at least kMinBatchPositions
// positions, one buffer set of at most kMaxScratch.  Measured on 512^2 x 6 wavelengths x 10
// modes (120 MB of fields per position), where the per-batch work that does not grow with the
// batch (reading the probes in the forward and adjoint rows, adding into the probe gradient,
// the launches' tails) is largest: 17 / 20 / 26 / 34 / 45 / 60 / 75 / 100 positions per batch
// gave 143.0 / 141.5 / 140.3 / 138.7 / 137.0 / 136.1 / 135.6 / 134.8 ms per step (three batches
// in flight); 512^2 x 8 modes x 5 wavelengths: 41.8 ms with 25 positions, 40.9 with 58.
constexpr long long kMaxScratch = 8ll << 30;   // default upper bound of one buffer set
constexpr long long kBatchEvals = 1200;        // evaluations per batch the default aims for
constexpr long long kMinBatchPositions = 64;   // and at least this many positions (when they fit)
constexpr long long kMinBatches = 3;           // and at least this many batches per call (overlap)
constexpr long long kBatchRows = 32768;        // and at least this many 1D FFT rows per pass
constexpr int kDefaultOverlap = 3;             // position batches in flight
constexpr double kPi = 3.14159265358979323846;

bool supported_F(int F) { return F == 64 || F == 128 || F == 256 || F == 512; }

template <class T>
int dalloc(ptycho_plan* p, T** ptr, long long count) {
  if (count <= 0) { *ptr = nullptr; return PTYCHO_OK; }
  const size_t bytes = sizeof(T) * (size_t)count;
  if (cudaMalloc((void**)ptr, bytes) != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return PTYCHO_ENOMEM;
  }
  p->bytes += (long long)bytes;
  return PTYCHO_OK;
}

template <class T>
int upload(T* dst, const T* src, long long count) {
  if (count <= 0) return PTYCHO_OK;
  return cudaMemcpy(dst, src, sizeof(T) * (size_t)count, cudaMemcpyHostToDevice) == cudaSuccess ? PTYCHO_OK
                                                                                              : PTYCHO_ECUDA;
}

void build_remap(int F, double z, double p, double alpha, std::vector<int32_t>& base, std::vector<float2>& w,
                 std::vector<int32_t>& rt_ptr, std::vector<int32_t>& rt_idx, std::vector<float>& rt_w,
                 std::vector<float2>& dz);

// (Re)builds the remap tables of p for p->z: taps, index rates and the CSR transpose, whose
// index and weight arrays are reallocated to their new length.  Synchronous.
int load_remap(ptycho_plan* p) {
  const int F = p->F;
  const long long FF = (long long)F * F;
  std::vector<int32_t> base, rt_ptr, rt_idx;
  std::vector<float2> w, dz;
  std::vector<float> rt_w;
  build_remap(F, p->z, p->det_pixel, p->tilt_rad, base, w, rt_ptr, rt_idx, rt_w, dz);
  const long long n = std::max<long long>(1, (long long)rt_idx.size());
  if (n > p->rt_cap) {
    if (p->d_rt_idx) cudaFree(p->d_rt_idx);
    if (p->d_rt_w) cudaFree(p->d_rt_w);
    p->bytes -= p->rt_cap * (long long)(sizeof(int32_t) + sizeof(float));
    p->d_rt_idx = nullptr;
    p->d_rt_w = nullptr;
    p->rt_cap = 0;
    int rc = dalloc(p, &p->d_rt_idx, n);
    rc = rc ? rc : dalloc(p, &p->d_rt_w, n);
    if (rc) return rc;
    p->rt_cap = n;
  }
  int rc = upload(p->d_tap_base, base.data(), FF);
  rc = rc ? rc : upload(p->d_tap_w, w.data(), FF);
  rc = rc ? rc : upload(p->d_tap_dz, dz.data(), FF);
  rc = rc ? rc : upload(p->d_rt_ptr, rt_ptr.data(), FF + 1);
  rc = rc ? rc : upload(p->d_rt_idx, rt_idx.data(), (long long)rt_idx.size());
  rc = rc ? rc : upload(p->d_rt_w, rt_w.data(), (long long)rt_w.size());
  return rc;
}

// Bluestein tables of the chirp-z propagator, in FP64, rounded to float2:
//   chirp[l][n] = exp(-i pi zeta (n - F/2)^2 / F);
//   hf[l] = DFT_2F of the kernel h(m) = exp(+i pi zeta m^2 / F) for |m| < F at index m mod 2F
//           (index F: 0), ha[l] = DFT_2F of conj(h);  tw2[k2*N1 + t] = exp(-2 pi i t k2 / 2F).
int load_czt(ptycho_plan* p, const double* zoom) {
  const int F = p->F, N = 2 * F, L = p->L;
  int N1 = 0;
  switch (F) {
    case 64: N1 = ptycho::CztShape<64>::N1; break;
    case 128: N1 = ptycho::CztShape<128>::N1; break;
    case 256: N1 = ptycho::CztShape<256>::N1; break;
    default: N1 = ptycho::CztShape<512>::N1; break;
  }
  std::vector<float2> chirp((size_t)L * F), hf((size_t)L * N), ha((size_t)L * N), tw2((size_t)N);
  std::vector<double> hr(N), hi(N);
  for (int l = 0; l < L; ++l) {
    const double z = zoom[l];
    for (int n = 0; n < F; ++n) {
      const double c = (double)(n - F / 2), ang = -kPi * z * c * c / F;
      chirp[(size_t)l * F + n] = make_float2((float)cos(ang), (float)sin(ang));
    }
    for (int m = 0; m < N; ++m) {
      const int mm = m < F ? m : m - N;
      if (m == F) { hr[m] = hi[m] = 0.0; continue; }
      const double ang = kPi * z * (double)mm * (double)mm / F;
      hr[m] = cos(ang);
      hi[m] = sin(ang);
    }
    for (int k = 0; k < N; ++k) {
      double fr = 0.0, fi = 0.0, ar = 0.0, ai = 0.0;
      for (int m = 0; m < N; ++m) {
        const double ang = -2.0 * kPi * (double)(((long long)k * m) % N) / N;
        const double c = cos(ang), sn = sin(ang);
        fr += hr[m] * c - hi[m] * sn;                 // h * e
        fi += hr[m] * sn + hi[m] * c;
        ar += hr[m] * c + hi[m] * sn;                 // conj(h) * e
        ai += hr[m] * sn - hi[m] * c;
      }
      hf[(size_t)l * N + k] = make_float2((float)fr, (float)fi);
      ha[(size_t)l * N + k] = make_float2((float)ar, (float)ai);
    }
  }
  for (int t = 0; t < N1; ++t)
    for (int k2 = 0; k2 < N / N1; ++k2) {
      const double ang = -2.0 * kPi * (double)((t * k2) % N) / N;
      tw2[(size_t)k2 * N1 + t] = make_float2((float)cos(ang), (float)sin(ang));
    }
  int rc = dalloc(p, &p->d_czt_chirp, (long long)L * F);
  rc = rc ? rc : dalloc(p, &p->d_czt_hf, (long long)L * N);
  rc = rc ? rc : dalloc(p, &p->d_czt_ha, (long long)L * N);
  rc = rc ? rc : dalloc(p, &p->d_czt_tw2, (long long)N);
  rc = rc ? rc : upload(p->d_czt_chirp, chirp.data(), (long long)L * F);
  rc = rc ? rc : upload(p->d_czt_hf, hf.data(), (long long)L * N);
  rc = rc ? rc : upload(p->d_czt_ha, ha.data(), (long long)L * N);
  rc = rc ? rc : upload(p->d_czt_tw2, tw2.data(), (long long)N);
  return rc;
}

void free_plan(ptycho_plan* p) {
  for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
  for (cudaEvent_t e : p->ev_copy) cudaEventDestroy(e);
  if (p->ev_copy_start) cudaEventDestroy(p->ev_copy_start);
  if (p->copy_st) cudaStreamDestroy(p->copy_st);
  if (p->ev_fork) cudaEventDestroy(p->ev_fork);
  for (int i = 0; i < ptycho_plan::kMaxSets; ++i) {
    if (p->ev_radj[i]) cudaEventDestroy(p->ev_radj[i]);
    if (p->ev_og[i]) cudaEventDestroy(p->ev_og[i]);
    if (i < ptycho_plan::kMaxSets - 1) {
      if (p->ev_join[i]) cudaEventDestroy(p->ev_join[i]);
      if (p->side[i]) cudaStreamDestroy(p->side[i]);
    }
  }
  void* ptrs[] = {p->d_pos, p->d_ident, p->d_tw, p->d_tap_base, p->d_tap_w, p->d_rt_ptr, p->d_rt_idx,
                  p->d_rt_w, p->d_S, p->d_Ipart, p->d_D, p->d_Gt, p->d_loss_part, p->d_gO, p->d_gP, p->d_status,
                  p->d_sig_part, p->d_gbg_set, p->d_gsig, p->d_gbg, p->d_gPs, p->d_shT, p->d_shQ, p->d_shP,
                  p->d_dpart, p->d_gdelta, p->d_tap_dz, p->d_z_part, p->d_czt_chirp, p->d_czt_hf,
                  p->d_czt_ha, p->d_czt_tw2, p->d_reg_part};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  delete p;
}

// Tilted-plane remap R (model grid -> camera grid), following the reflection geometry of the
// section "Experimental setup": camera perpendicular to the specular beam at distance z,
// sample tilted by alpha from the normal.  Camera pixel (y, x) looks along (X, Y, z) with
// X = (x - F/2) p, Y = (y - F/2) p; its sample-frame direction cosines are a = X / R and
// b = (Y cos a + z sin a) / R - sin a.  The model grid is uniform in (b, a) with spacings
// (p/z) cos(alpha) and p/z around the specular direction.  Each camera pixel takes the
// bilinear interpolation of its four surrounding model pixels; it is invalid (masked) when
// they leave the grid.  Index decisions are taken in FP64.
// Also dz: per camera pixel, the rates d(row index)/dz and d(column index)/dz of its
// fractional model-grid position (row index = z b / (p cos alpha) + F/2, column index =
// z a / p + F/2, a and b the direction cosines below), for the gradient with respect to z.
void build_remap(int F, double z, double p, double alpha, std::vector<int32_t>& base, std::vector<float2>& w,
                 std::vector<int32_t>& rt_ptr, std::vector<int32_t>& rt_idx, std::vector<float>& rt_w,
                 std::vector<float2>& dz) {
  const double c = cos(alpha), s = sin(alpha);
  const double da = p / z, db = da * c;
  const int FF = F * F;
  base.assign(FF, -1);
  w.assign(FF, make_float2(0.f, 0.f));
  dz.assign(FF, make_float2(0.f, 0.f));
  std::vector<double> wy(FF, 0.0), wx(FF, 0.0);
  for (int y = 0; y < F; ++y) {
    for (int x = 0; x < F; ++x) {
      const double X = (x - F / 2.0) * p;
      const double Y = (y - F / 2.0) * p;
      const double R = sqrt(X * X + Y * Y + z * z);
      const double a = X / R;
      const double b = (Y * c + z * s) / R - s;
      const double yh = b / db + F / 2.0;
      const double xh = a / da + F / 2.0;
      if (yh >= 0.0 && yh < F - 1 && xh >= 0.0 && xh < F - 1) {
        const int iy = (int)floor(yh), ix = (int)floor(xh);
        base[y * F + x] = iy * F + ix;
        wy[y * F + x] = yh - iy;
        wx[y * F + x] = xh - ix;
        w[y * F + x] = make_float2((float)(yh - iy), (float)(xh - ix));
        const double R3 = R * R * R;
        const double b_z = s / R - (Y * c + z * s) * z / R3;
        dz[y * F + x] = make_float2((float)((b + z * b_z) / (p * c)), (float)((X / p) * (1.0 / R - z * z / R3)));
      }
    }
  }
  // exact transpose: entries grouped by model pixel, camera pixels in increasing order
  std::vector<int32_t> count(FF + 1, 0);
  for (int q = 0; q < FF; ++q) {
    if (base[q] < 0) continue;
    const int u = base[q];
    count[u + 1]++; count[u + 2]++; count[u + F + 1]++; count[u + F + 2]++;
  }
  rt_ptr.assign(FF + 1, 0);
  for (int u = 0; u < FF; ++u) rt_ptr[u + 1] = rt_ptr[u] + count[u + 1];
  rt_idx.assign(rt_ptr[FF], 0);
  rt_w.assign(rt_ptr[FF], 0.f);
  std::vector<int32_t> fill(rt_ptr.begin(), rt_ptr.end() - 1);
  for (int q = 0; q < FF; ++q) {
    if (base[q] < 0) continue;
    const int u = base[q];
    const double v = wy[q], h = wx[q];
    const int us[4] = {u, u + 1, u + F, u + F + 1};
    const double ws[4] = {(1 - v) * (1 - h), (1 - v) * h, v * (1 - h), v * h};
    for (int k = 0; k < 4; ++k) {
      rt_idx[fill[us[k]]] = q;
      rt_w[fill[us[k]]] = (float)ws[k];
      fill[us[k]]++;
    }
  }
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to libcuda).
// Looked up once per process (a thread-safe static initialisation).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    cudaGetLastError();
    return (PFN_cuTensorMapEncodeTiled_v12000) nullptr;
  }();
  return fn;
}

// 2D map over a scratch set: rows of F complex64 (8-byte elements), box W x min(F, 256).
bool make_column_map(CUtensorMap* map, void* base, int F, long long rows, int W) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)F, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)F * 8};
  const cuuint32_t box[2] = {(cuuint32_t)W, (cuuint32_t)(F < 256 ? F : 256)};
  const cuuint32_t estride[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, base, dims, strides, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int check_device(const ptycho_plan* p) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return PTYCHO_ECUDA;
  return dev == p->dev ? PTYCHO_OK : PTYCHO_EINVAL;
}

int dispatch(ptycho_plan* p, const CallArgs& c, cudaStream_t st) {
  switch (p->F) {
    case 64: return ptycho::run_pipeline<64>(*p, c, st);
    case 128: return ptycho::run_pipeline<128>(*p, c, st);
    case 256: return ptycho::run_pipeline<256>(*p, c, st);
    case 512: return ptycho::run_pipeline<512>(*p, c, st);
  }
  return PTYCHO_EUNSUPPORTED;
}

int fill_batch(ptycho_plan* p, CallArgs& c, const int32_t* batch_idx, int nbatch) {
  if (batch_idx) {
    if (nbatch < 1 || nbatch > p->J) return PTYCHO_EINVAL;
    c.bidx = batch_idx;
    c.nbatch = nbatch;
  } else {
    c.bidx = p->d_ident;
    c.nbatch = p->J;
  }
  return PTYCHO_OK;
}

}  // namespace

extern "C" {

const char* ptycho_strerror(int code) {
  switch (code) {
    case PTYCHO_OK: return "success";
    case PTYCHO_EINVAL: return "invalid argument (shape, size, NULL pointer, option or device)";
    case PTYCHO_ERANGE: return "a scan position puts a patch outside its object";
    case PTYCHO_ENOMEM: return "device memory allocation failed";
    case PTYCHO_ECUDA: return "a CUDA call or kernel launch failed";
    case PTYCHO_ETIMEDOUT: return "a bounded device wait timed out";
    case PTYCHO_EUNSUPPORTED: return "unsupported configuration (frame size or wavelength count)";
    case PTYCHO_ETOOLARGE: return "problem does not fit the fixed array of the allocation-free entry point";
    case PTYCHO_EBUSY: return "no free serving slot, or the HBM budget is exhausted";
  }
  return "unknown error";
}

int ptycho_plan_create(const ptycho_geom_t* g, ptycho_plan_t** out) {
  return ptycho::create_plan(g, ptycho::BatchTarget{kBatchEvals, kMinBatchPositions, kMaxScratch}, out);
}

}  // extern "C"

namespace ptycho {

int create_plan(const ptycho_geom_t* g, const BatchTarget& target, ptycho_plan_t** out) {
  if (!g || !out) return PTYCHO_EINVAL;
  *out = nullptr;
  if (g->L < 1 || g->M < 1 || g->J < 1 || !g->obj_h || !g->obj_w || !g->pos) return PTYCHO_EINVAL;
  if (g->L > ptycho::kMaxL || !supported_F(g->F)) return PTYCHO_EUNSUPPORTED;
  if (g->loss != PTYCHO_LOSS_AMPLITUDE && g->loss != PTYCHO_LOSS_POISSON && g->loss != PTYCHO_LOSS_POISSON_GAUSSIAN)
    return PTYCHO_EINVAL;
  if (g->loss == PTYCHO_LOSS_POISSON_GAUSSIAN && !(g->read_noise_var >= 0.f && isfinite(g->read_noise_var)))
    return PTYCHO_EINVAL;
  if (g->zoom) {
    for (int l = 0; l < g->L; ++l)
      if (!(g->zoom[l] > 0.0 && g->zoom[l] <= 4.0)) return PTYCHO_EINVAL;
  }
  if (!(g->eps >= 0.f) || !isfinite(g->eps)) return PTYCHO_EINVAL;
  if (g->remap && !(g->z > 0.0 && g->det_pixel > 0.0 && isfinite(g->tilt_rad) && fabs(g->tilt_rad) < kPi / 2))
    return PTYCHO_EINVAL;
  const int F = g->F;
  for (int l = 0; l < g->L; ++l)
    if (g->obj_h[l] < F || g->obj_w[l] < F) return PTYCHO_EINVAL;
  for (int l = 0; l < g->L; ++l)
    for (int j = 0; j < g->J; ++j) {
      const int y = g->pos[(l * g->J + j) * 2], x = g->pos[(l * g->J + j) * 2 + 1];
      if (y < 0 || x < 0 || y > g->obj_h[l] - F || x > g->obj_w[l] - F) return PTYCHO_ERANGE;
    }

  ptycho_plan* p = new (std::nothrow) ptycho_plan();
  if (!p) return PTYCHO_ENOMEM;
  if (cudaGetDevice(&p->dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->dev) != cudaSuccess) {
    delete p;
    return PTYCHO_ECUDA;
  }
  p->L = g->L; p->M = g->M; p->F = F; p->J = g->J;
  p->remap = g->remap ? 1 : 0;
  p->loss_kind = g->loss;
  p->read_var = g->loss == PTYCHO_LOSS_POISSON_GAUSSIAN ? g->read_noise_var : 0.f;
  p->flags = g->flags & (PTYCHO_FLAG_RECOMPUTE_COLUMNS | PTYCHO_FLAG_OBJ_GRAD_ATOMIC | PTYCHO_FLAG_NARROW_COLUMNS |
                         PTYCHO_FLAG_NO_PDL | PTYCHO_FLAG_RESIDENT_FRAMES);
  // measured: recomputing the column DFT beats keeping Psi from F = 256 up
  if (!(g->flags & (PTYCHO_FLAG_RECOMPUTE_COLUMNS | PTYCHO_FLAG_KEEP_PSI)) && g->F >= 256)
    p->flags |= PTYCHO_FLAG_RECOMPUTE_COLUMNS;
  p->eps = g->eps;
  long long off = 0;
  for (int l = 0; l < g->L; ++l) {
    p->obj_h[l] = g->obj_h[l];
    p->obj_w[l] = g->obj_w[l];
    p->obj_off[l] = off;
    off += (long long)g->obj_h[l] * g->obj_w[l];
  }
  p->O_numel = off;
  p->P_numel = (long long)g->L * g->M * F * F;
  p->pos_host.assign(g->pos, g->pos + (size_t)g->L * g->J * 2);

  // batching: a batch keeps the fields of all L*M modes of B positions in the scratch (store
  // mode, no recompute) with B chosen so that one launch carries about kBatchEvals
  // evaluations; a small scratch stays in L2, a large one spills to HBM, which costs less than
  // launching small batches.  Only when one position's fields exceed the budget are the modes
  // split into chunks that the adjoint recomputes (small-mode problems also get at least
  // kBatchRows FFT rows per pass).  An explicit scratch_bytes fits as many
  // positions as the budget holds.
  const long long FF8 = (long long)F * F * (long long)sizeof(float2);
  const long long LM = (long long)g->L * g->M;
  p->scratch_budget = g->scratch_bytes > 0 ? g->scratch_bytes : target.max_set_bytes;
  if (LM * FF8 <= p->scratch_budget) {
    p->store = 1;
    p->C = (int)LM;
    p->nchunks = 1;
    long long B = p->scratch_budget / (LM * FF8);
    if (g->scratch_bytes <= 0) {
      B = std::min<long long>(B, std::max({(target.evals + LM - 1) / LM, (kBatchRows + LM * F - 1) / (LM * F),
                                           target.min_positions}));
      B = std::min<long long>(B, std::max<long long>(1, (g->J + kMinBatches - 1) / kMinBatches));
    }
    p->B = (int)std::max<long long>(1, std::min<long long>(B, ptycho::kMaxB));
    p->B = std::min(p->B, g->J);
    if (g->scratch_bytes <= 0) {                      // the same number of batches, sizes within one position
      const int nbat = (g->J + p->B - 1) / p->B;
      p->B = (g->J + nbat - 1) / nbat;
    }
  } else {
    p->store = 0;
    p->B = 1;
    p->C = (int)std::max<long long>(1, std::min<long long>(LM, p->scratch_budget / FF8));
    p->nchunks = (int)((LM + p->C - 1) / p->C);
  }
  int colblocks = 0;
  switch (F) {
    case 64: colblocks = F / ptycho::ColCfg<64>::W; break;
    case 128: colblocks = F / ptycho::ColCfg<128>::W; break;
    case 256: colblocks = F / ptycho::ColCfg<256>::W; break;
    default: colblocks = F / ptycho::ColCfg<512>::W; break;
  }
  const long long want_cols = 2ll * p->sms;   // column blocks wanted: mode groups only below two per SM
  long long G = (want_cols + (long long)colblocks * p->B - 1) / ((long long)colblocks * p->B);
  if (g->col_groups > 0) G = g->col_groups;
  G = std::max<long long>(1, std::min<long long>(G, p->C));
  p->MG = (int)((p->C + G - 1) / G);
  p->G = (p->C + p->MG - 1) / p->MG;
  if (p->store && (g->flags & PTYCHO_FLAG_STAGED_COLUMNS) && g->col_groups <= 0) {
    p->col_staged = 1;
    p->G = 1;
    p->MG = p->C;
  }

  // adjoint row pass over all modes of a wavelength per block (see PTYCHO_FLAG_UNFUSED_ROW_ADJ)
  {
    int T = 0, smem = 0;
    switch (F) {
      case 64: T = ptycho::FftShape<64>::N1; break;
      case 128: T = ptycho::FftShape<128>::N1; break;
      case 256: T = ptycho::FftShape<256>::N1; break;
      default: T = ptycho::FftShape<512>::N1; break;
    }
    // measured at F = 512: with 16 threads per row the fused kernel's registers (two 32-value rows
    // per thread) cost more occupancy than the probe reuse saves below 8 modes (4 modes x 3
    // wavelengths: 8 % slower; from 8 modes up faster: 8 x 3 by 2 %, 10 x 6 by 7 %); with one warp
    // per row it is faster from 2 modes up (2 x 3: 9.44 vs 9.76 ms, 4 x 3: 14.47 vs 17.32, 6 x 3:
    // 19.56 vs 24.81, 7 x 2: 16.35 vs 19.60) and slower with one mode (1 x 3: 6.67 vs 6.35)
    if (p->store && T * g->M <= 256) {
      int rpb = 1;
      while (2 * rpb * T * g->M <= 128 && 2 * rpb <= F) rpb *= 2;
      switch (F) {
        case 64: smem = ptycho::row_adj_l_smem<64>(g->M, rpb); break;
        case 128: smem = ptycho::row_adj_l_smem<128>(g->M, rpb); break;
        case 256: smem = ptycho::row_adj_l_smem<256>(g->M, rpb); break;
        default: smem = ptycho::row_adj_l_smem<512>(g->M, rpb); break;
      }
      if (smem <= ptycho::kRowAdjLSmemMax) {
        p->adj_l_ok = 1;
        p->rpb_adj = rpb;
        // one warp per row at F = 512 (half the registers per thread, two 10-warp blocks per SM):
        // measured 144.0 vs 153.3 ms per step on 512^2 x 6 wavelengths x 10 modes
        p->adj_l_w = F == 512 && 32 * g->M * rpb <= ptycho::kRowAdjWThreads &&
                     ptycho::row_adj_w_smem(g->M, rpb) <= ptycho::kRowAdjLSmemMax &&
                     !(g->flags & (PTYCHO_FLAG_ROW_ADJ_PROBE_SMEM | PTYCHO_FLAG_ROW_ADJ_PROBE_L2 |
                                   PTYCHO_FLAG_ROWS_16_THREADS));
        p->adj_l = !(g->flags & PTYCHO_FLAG_UNFUSED_ROW_ADJ) &&
                   (F <= 256 || g->M >= 8 || (p->adj_l_w && g->M >= 2) || (g->flags & PTYCHO_FLAG_FUSED_ROW_ADJ));
        // probe rows through L1/L2 and two blocks per SM: measured 1.4 % faster on config 4 (175.8
        // vs 178.2 ms per step) and 2.9 % on 512^2 x 8 modes x 3 wavelengths; equal on config 2
        const bool pl2_fits = T * g->M * rpb <= ptycho::kRowAdjL2Threads;
        p->adj_l_pl2 = pl2_fits && !(g->flags & PTYCHO_FLAG_ROW_ADJ_PROBE_SMEM) &&
                       (F == 512 || (g->flags & PTYCHO_FLAG_ROW_ADJ_PROBE_L2));
        // enough blocks for three per SM: split the batch's positions, each split summing its
        // probe gradient into a buffer of its own (bounded to 512 MB in all)
        const long long base = (long long)(F / rpb) * g->L;
        long long ns = (3ll * p->sms + base - 1) / base;
        ns = std::min<long long>(ns, std::min<long long>(64, p->B));
        while (ns > 1 && ns * p->P_numel * (long long)sizeof(float2) > (512ll << 20)) --ns;
        p->nsplit_adj = (int)std::max<long long>(1, ns);
        // the forward row pass: same blocks, positions split for four blocks per SM.  Default at
        // 512^2 from 4 modes, where the probes of all modes outgrow the L2 and the fused pass reads
        // each probe row once per block instead of once per position: measured 153.4 vs 157.2 ms
        // on config 4, 45.9 vs 47.4 ms on 8 modes x 5 wavelengths, 15.8 vs 16.4 on 4 x 3; slower
        // with one mode (3.62 vs 3.37 ms) and at 256^2 (3.32 vs 3.27 ms on config 2)
        const bool fwd_default = F == 512 && g->M >= 4 && !(g->flags & PTYCHO_FLAG_UNFUSED_ROW_FWD);
        if (((g->flags & PTYCHO_FLAG_FUSED_ROW_FWD) && !(g->flags & PTYCHO_FLAG_UNFUSED_ROW_FWD)) || fwd_default) {
          p->fwd_l = 1;
          p->nsplit_fwd = (int)std::max<long long>(1, std::min<long long>((4ll * p->sms + base - 1) / base, p->B));
          // one warp per row at F = 512 (opt-in): measured 146.4 vs 144.0 ms per step on 512^2 x
          // 6 wavelengths x 10 modes, the pass itself shorter but the other streams' passes longer
          p->fwd_l_w = F == 512 && 32 * g->M * rpb <= ptycho::kRowAdjWThreads &&
                       (g->flags & PTYCHO_FLAG_FWD_ROWS_WARP) && !(g->flags & PTYCHO_FLAG_ROWS_16_THREADS);
        }
      }
    }
  }

  // frame-resident passes (F <= 128, opt-in; measured slower than the scratch passes): all
  // modes of a position in one chunk; the forward's blocks (position, mode group) and the
  // adjoint's (probe mode, position split) aim at two waves of resident blocks (one block per SM
  // at F = 128, two at F = 64); each split sums its probe gradient into a buffer of its own
  // (bounded to 512 MB in all)
  if (F <= 128 && p->store && !g->zoom && (g->flags & PTYCHO_FLAG_RESIDENT_FRAMES) &&
      !(g->flags & PTYCHO_FLAG_OBJ_GRAD_ATOMIC)) {
    const long long per_sm = F <= 64 ? 2 : 1;
    const long long want = 2 * per_sm * p->sms;
    long long Gr = (want + p->B - 1) / p->B;
    Gr = std::max<long long>(1, std::min<long long>(Gr, LM));
    p->MG_res = (int)((LM + Gr - 1) / Gr);
    p->G_res = (int)((LM + p->MG_res - 1) / p->MG_res);
    long long ns = (want + LM - 1) / LM;
    ns = std::max<long long>(1, std::min<long long>(ns, p->B));
    while (ns > 1 && ns * p->P_numel * (long long)sizeof(float2) > (512ll << 20)) --ns;
    p->nsplit_res = (int)ns;
    p->res = 1;
  }

  // chirp-z propagator: its own passes (the per-mode row adjoint, the mode-group columns with
  // the column transform recomputed in the adjoint); all modes of a position in the scratch
  if (g->zoom) {
    if (!p->store) {
      free_plan(p);
      return PTYCHO_EUNSUPPORTED;
    }
    p->czt = 1;
    p->adj_l = 0;
    p->fwd_l = 0;
    p->col_staged = 0;
    p->flags |= PTYCHO_FLAG_RECOMPUTE_COLUMNS;
  }

  int rc = PTYCHO_OK;
  const long long FF = (long long)F * F;
  rc = rc ? rc : dalloc(p, &p->d_pos, (long long)g->L * g->J * 2);
  rc = rc ? rc : dalloc(p, &p->d_ident, g->J);
  rc = rc ? rc : dalloc(p, &p->d_tw, F);
  // overlap consecutive batches (several buffer sets) when the fields are kept between passes
  {
    const int want = g->overlap > 0 ? std::min(g->overlap, ptycho_plan::kMaxSets) : kDefaultOverlap;
    const int nbat = (g->J + p->B - 1) / p->B;
    p->nsets = p->store ? std::max(1, std::min(want, nbat)) : 1;
  }
  if (cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming) != cudaSuccess) rc = PTYCHO_ECUDA;
  for (int i = 0; i < p->nsets && !rc; ++i) {
    if (cudaEventCreateWithFlags(&p->ev_radj[i], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_og[i], cudaEventDisableTiming) != cudaSuccess)
      rc = PTYCHO_ECUDA;
    if (i > 0 && !rc &&
        (cudaStreamCreateWithFlags(&p->side[i - 1], cudaStreamNonBlocking) != cudaSuccess ||
         cudaEventCreateWithFlags(&p->ev_join[i - 1], cudaEventDisableTiming) != cudaSuccess))
      rc = PTYCHO_ECUDA;
  }
  rc = rc ? rc : dalloc(p, &p->d_S, (long long)p->nsets * p->B * p->C * FF);
  rc = rc ? rc : dalloc(p, &p->d_Ipart, (long long)p->nsets * p->B * std::max(p->G, p->res ? p->G_res : 1) * FF);
  rc = rc ? rc : dalloc(p, &p->d_D, (long long)p->nsets * p->B * FF);
  rc = rc ? rc : dalloc(p, &p->d_loss_part, (long long)g->J * (FF / (ptycho::kLossThreads * ptycho::kLossPx)));
  rc = rc ? rc : dalloc(p, &p->d_sig_part, (long long)g->J * (FF / (ptycho::kLossThreads * ptycho::kLossPx)));
  rc = rc ? rc : dalloc(p, &p->d_gbg_set, (long long)p->nsets * FF);
  rc = rc ? rc : dalloc(p, &p->d_gsig, g->J);
  rc = rc ? rc : dalloc(p, &p->d_gbg, FF);
  rc = rc ? rc : dalloc(p, &p->d_gO, p->O_numel);
  rc = rc ? rc : dalloc(p, &p->d_gP, p->P_numel);
  {
    const int ns = std::max(p->adj_l_ok ? p->nsplit_adj : 1, p->res ? p->nsplit_res : 1);
    if (ns > 1) rc = rc ? rc : dalloc(p, &p->d_gPs, (long long)ns * p->P_numel);
  }
  rc = rc ? rc : dalloc(p, &p->d_status, 1);
  if (!rc && cudaMemset(p->d_status, 0, sizeof(int)) != cudaSuccess) rc = PTYCHO_ECUDA;
  if (rc) { free_plan(p); return rc; }
  {
    int W = 0;
    switch (F) {
      case 64: W = ptycho::ColCfg<64>::W; break;
      case 128: W = ptycho::ColCfg<128>::W; break;
      case 256: W = ptycho::ColCfg<256>::W; break;
      default: W = ptycho::ColCfg<512>::W; break;
    }
    const long long rows = (long long)p->B * p->C * F;
    // measured: the staged column passes pay off at F = 512 from two fields per position up (one
    // field: the plain-load passes, two blocks per SM, are 10 % faster), and at F = 128 once a
    // position has four or more fields (3-6 % on 128^2 with L*M = 5..40; 2 % slower with L*M = 1;
    // at F = 256 and F = 64 they measured slower or equal)
    const bool tma_default = (F >= 512 && p->C >= 2) || (F == 128 && p->C >= 4);
    p->has_tma = (g->flags & PTYCHO_FLAG_NO_TMA) || p->czt ? 0 : ((g->flags & PTYCHO_FLAG_TMA) || tma_default) ? 1 : 0;
    // F = 512: the staged column passes with the half-size exchange, two blocks per SM
    p->col_tma2 = F == 512 && !(g->flags & PTYCHO_FLAG_COLS_ONE_BLOCK) ? 1 : 0;
    for (int i = 0; i < p->nsets; ++i)
      if (p->has_tma && !make_column_map(&p->tmap_S[i], p->d_S + (long long)i * p->B * p->C * FF, F, rows, W))
        p->has_tma = 0;
  }

  std::vector<int32_t> ident(g->J);
  for (int j = 0; j < g->J; ++j) ident[j] = j;
  // twiddles W_F^(t*k2) of the two-stage FFT, tw[k2*N1 + t], in FP64 then rounded
  int N1 = 0, N2 = 0;
  switch (F) {
    case 64: N1 = ptycho::FftShape<64>::N1; N2 = ptycho::FftShape<64>::N2; break;
    case 128: N1 = ptycho::FftShape<128>::N1; N2 = ptycho::FftShape<128>::N2; break;
    case 256: N1 = ptycho::FftShape<256>::N1; N2 = ptycho::FftShape<256>::N2; break;
    default: N1 = ptycho::FftShape<512>::N1; N2 = ptycho::FftShape<512>::N2; break;
  }
  std::vector<float2> tw((size_t)N1 * N2);
  for (int t = 0; t < N1; ++t)
    for (int k2 = 0; k2 < N2; ++k2) {
      const double ang = -2.0 * kPi * (double)((t * k2) % F) / (double)F;
      tw[(size_t)k2 * N1 + t] = make_float2((float)cos(ang), (float)sin(ang));
    }
  rc = rc ? rc : upload(p->d_pos, p->pos_host.data(), (long long)p->pos_host.size());
  rc = rc ? rc : upload(p->d_ident, ident.data(), g->J);
  rc = rc ? rc : upload(p->d_tw, tw.data(), (long long)tw.size());
  if (!rc && p->remap) {
    p->z = g->z;
    p->det_pixel = g->det_pixel;
    p->tilt_rad = g->tilt_rad;
    rc = dalloc(p, &p->d_Gt, (long long)p->nsets * p->B * FF);
    rc = rc ? rc : dalloc(p, &p->d_tap_base, FF);
    rc = rc ? rc : dalloc(p, &p->d_tap_w, FF);
    rc = rc ? rc : dalloc(p, &p->d_tap_dz, FF);
    rc = rc ? rc : dalloc(p, &p->d_rt_ptr, FF + 1);
    rc = rc ? rc : dalloc(p, &p->d_z_part, (long long)g->J * (FF / (ptycho::kLossThreads * ptycho::kLossPx)));
    rc = rc ? rc : load_remap(p);
  }
  if (!rc && p->czt) rc = load_czt(p, g->zoom);
  if (rc) { free_plan(p); return rc; }
  *out = p;
  return PTYCHO_OK;
}

}  // namespace ptycho

extern "C" {

int ptycho_plan_destroy(ptycho_plan_t* p) {
  if (!p) return PTYCHO_OK;
  cudaDeviceSynchronize();
  free_plan(p);
  return PTYCHO_OK;
}

int64_t ptycho_plan_workspace_bytes(const ptycho_plan_t* p) { return p ? p->bytes : 0; }
int64_t ptycho_plan_numel_O(const ptycho_plan_t* p) { return p ? p->O_numel : 0; }
int64_t ptycho_plan_numel_P(const ptycho_plan_t* p) { return p ? p->P_numel : 0; }
int64_t ptycho_plan_last_launches(const ptycho_plan_t* p) { return p ? p->last_launches : 0; }

int ptycho_plan_profile(ptycho_plan_t* p, int enable) {
  if (!p) return PTYCHO_EINVAL;
  p->prof = enable ? 1 : 0;
  p->ev_used = 0;
  p->ev_kind.clear();
  return PTYCHO_OK;
}

int ptycho_plan_profile_read(ptycho_plan_t* p, double* ms, int64_t* launches) {
  if (!p || !ms || !launches) return PTYCHO_EINVAL;
  for (int k = 0; k < ptycho::kNumKinds; ++k) { ms[k] = 0.0; launches[k] = 0; }
  for (size_t i = 0; i < p->ev_used; ++i) {
    if (cudaEventSynchronize(p->ev_pool[2 * i + 1]) != cudaSuccess) return PTYCHO_ECUDA;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, p->ev_pool[2 * i], p->ev_pool[2 * i + 1]) != cudaSuccess) return PTYCHO_ECUDA;
    ms[p->ev_kind[i]] += t;
    launches[p->ev_kind[i]] += 1;
  }
  p->ev_used = 0;
  p->ev_kind.clear();
  return PTYCHO_OK;
}

const char* ptycho_kernel_name(int kind) {
  static const char* names[] = {"row_fwd", "col_fwd", "loss", "col_adj", "row_adj", "obj_grad", "loss_reduce", "adam",
                                "remap_adj", "shift", "regulariser", "res_fwd", "res_adj"};
  return (kind >= 0 && kind < ptycho::kNumKinds) ? names[kind] : "unknown";
}

int ptycho_plan_status(ptycho_plan_t* p, int32_t* flags) {
  if (!p || !flags) return PTYCHO_EINVAL;
  int rc = check_device(p);
  if (rc) return rc;
  int v = 0;
  if (cudaMemcpy(&v, p->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return PTYCHO_ECUDA;
  if (cudaMemset(p->d_status, 0, sizeof(int)) != cudaSuccess) return PTYCHO_ECUDA;
  *flags = v;
  return PTYCHO_OK;
}

int ptycho_forward(ptycho_plan_t* p, const float* O, const float* P, const float* sigma, const float* bg,
                   float* I_pred, void* stream) {
  if (!p || !O || !P || !I_pred) return PTYCHO_EINVAL;
  int rc = check_device(p);
  if (rc) return rc;
  CallArgs c{};
  c.kind = CallKind::Forward;
  c.O = reinterpret_cast<const float2*>(O);
  c.P = reinterpret_cast<const float2*>(P);
  c.sigma = sigma;
  c.bg = bg;
  c.I_pred = I_pred;
  fill_batch(p, c, nullptr, 0);
  return dispatch(p, c, (cudaStream_t)stream);
}

int ptycho_plan_set_distance(ptycho_plan_t* p, double z) {
  if (!p) return PTYCHO_EINVAL;
  if (!p->remap) return PTYCHO_EUNSUPPORTED;
  if (!(z > 0.0) || !isfinite(z)) return PTYCHO_EINVAL;
  int rc = check_device(p);
  if (rc) return rc;
  if (cudaDeviceSynchronize() != cudaSuccess) return PTYCHO_ECUDA;   // no call of this plan in flight
  const double old = p->z;
  p->z = z;
  rc = load_remap(p);
  if (rc) {
    p->z = old;
    load_remap(p);
  }
  return rc;
}

int ptycho_plan_set_offsets(ptycho_plan_t* p, float* delta) {
  if (!p) return PTYCHO_EINVAL;
  int rc = check_device(p);
  if (rc) return rc;
  if (!delta) {
    p->d_delta = nullptr;
    return PTYCHO_OK;
  }
  if (!p->store || !p->adj_l_ok || p->czt) return PTYCHO_EUNSUPPORTED;
  if (!p->d_shT) {
    const long long n = (long long)p->nsets * p->B * p->L * p->F * p->F;
    int W = 0;
    switch (p->F) {
      case 64: W = ptycho::ColCfg<64>::W; break;
      case 128: W = ptycho::ColCfg<128>::W; break;
      case 256: W = ptycho::ColCfg<256>::W; break;
      default: W = ptycho::ColCfg<512>::W; break;
    }
    rc = dalloc(p, &p->d_shT, n);
    rc = rc ? rc : dalloc(p, &p->d_shQ, n);
    rc = rc ? rc : dalloc(p, &p->d_shP, n);
    rc = rc ? rc : dalloc(p, &p->d_dpart, (long long)p->J * p->L * (p->F / W) * 2);
    rc = rc ? rc : dalloc(p, &p->d_gdelta, 2ll * p->L * p->J);
    if (rc) {                                         // leave the plan as it was
      void* bufs[] = {p->d_shT, p->d_shQ, p->d_shP, p->d_dpart, p->d_gdelta};
      for (void* q : bufs)
        if (q) cudaFree(q);
      p->d_shT = p->d_shQ = p->d_shP = nullptr;
      p->d_dpart = nullptr;
      p->d_gdelta = nullptr;
      return rc;
    }
  }
  p->d_delta = delta;
  return PTYCHO_OK;
}

int ptycho_loss(ptycho_plan_t* p, const float* O, const float* P, const float* sigma, const float* bg,
                const float* I_meas, const uint8_t* mask, int mask_per_frame, const int32_t* batch_idx,
                int nbatch, double* loss_dev, void* stream) {
  if (!p || !O || !P || !I_meas || !loss_dev) return PTYCHO_EINVAL;
  int rc = check_device(p);
  if (rc) return rc;
  CallArgs c{};
  c.kind = CallKind::Loss;
  c.O = reinterpret_cast<const float2*>(O);
  c.P = reinterpret_cast<const float2*>(P);
  c.sigma = sigma;
  c.bg = bg;
  c.Imeas = I_meas;
  c.mask = mask;
  c.mask_per_frame = mask_per_frame ? 1 : 0;
  c.loss = loss_dev;
  rc = fill_batch(p, c, batch_idx, nbatch);
  if (rc) return rc;
  return dispatch(p, c, (cudaStream_t)stream);
}

int ptycho_adjoint(ptycho_plan_t* p, const float* O, const float* P, const float* sigma, const float* bg,
                   const float* I_meas, const uint8_t* mask, int mask_per_frame, const int32_t* batch_idx,
                   int nbatch, float* gO, float* gP, double* loss_dev, void* stream) {
  return ptycho_adjoint_ex(p, O, P, sigma, bg, I_meas, mask, mask_per_frame, batch_idx, nbatch, gO, gP, nullptr,
                           nullptr, nullptr, nullptr, loss_dev, stream);
}

int ptycho_adjoint_ex(ptycho_plan_t* p, const float* O, const float* P, const float* sigma, const float* bg,
                      const float* I_meas, const uint8_t* mask, int mask_per_frame, const int32_t* batch_idx,
                      int nbatch, float* gO, float* gP, float* g_sigma, float* g_bg, float* g_delta,
                      double* g_z, double* loss_dev, void* stream) {
  if (!p || !O || !P || !I_meas || !gO || !gP) return PTYCHO_EINVAL;
  if (g_delta && !p->d_delta) return PTYCHO_EINVAL;   // a position gradient needs registered offsets
  if (g_z && !p->remap) return PTYCHO_EINVAL;         // z enters through the remap only
  int rc = check_device(p);
  if (rc) return rc;
  CallArgs c{};
  c.kind = CallKind::Adjoint;
  c.O = reinterpret_cast<const float2*>(O);
  c.P = reinterpret_cast<const float2*>(P);
  c.sigma = sigma;
  c.bg = bg;
  c.Imeas = I_meas;
  c.mask = mask;
  c.mask_per_frame = mask_per_frame ? 1 : 0;
  c.gO = reinterpret_cast<float2*>(gO);
  c.gP = reinterpret_cast<float2*>(gP);
  c.g_sigma = g_sigma;
  c.g_bg = g_bg;
  c.g_delta = g_delta;
  c.g_z = g_z;
  c.loss = loss_dev;
  rc = fill_batch(p, c, batch_idx, nbatch);
  if (rc) return rc;
  return dispatch(p, c, (cudaStream_t)stream);
}

int ptycho_step(ptycho_plan_t* p, ptycho_adam_t* s, float* O, float* P, float* sigma, float* bg,
                const float* I_meas, const uint8_t* mask, int mask_per_frame, const int32_t* batch_idx,
                int nbatch, double* loss_dev, void* stream) {
  if (!p || !s || !O || !P || !I_meas || !s->mO || !s->vO || !s->mP || !s->vP) return PTYCHO_EINVAL;
  if (!(s->beta1 >= 0.f && s->beta1 < 1.f && s->beta2 >= 0.f && s->beta2 < 1.f && s->eps >= 0.f)) return PTYCHO_EINVAL;
  const bool opt_sigma = s->lr_sigma > 0.f, opt_bg = s->lr_bg > 0.f, opt_delta = s->lr_delta > 0.f;
  if (opt_sigma && (!sigma || !s->m_sigma || !s->v_sigma)) return PTYCHO_EINVAL;
  if (opt_bg && (!bg || !s->m_bg || !s->v_bg)) return PTYCHO_EINVAL;
  if (opt_delta && (!p->d_delta || !s->m_delta || !s->v_delta)) return PTYCHO_EINVAL;
  const bool reg = s->reg_l1 != 0.f || s->reg_tv != 0.f;
  if (reg && !ptycho::reg_args_ok(s->reg_l1, s->reg_tv, s->reg_eta)) return PTYCHO_EINVAL;
  int rc = ptycho_adjoint_ex(p, O, P, sigma, bg, I_meas, mask, mask_per_frame, batch_idx, nbatch,
                             reinterpret_cast<float*>(p->d_gO), reinterpret_cast<float*>(p->d_gP),
                             opt_sigma ? p->d_gsig : nullptr, opt_bg ? p->d_gbg : nullptr,
                             opt_delta ? p->d_gdelta : nullptr, s->g_z, loss_dev, stream);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if (reg) {
    // the regulariser's value joins the loss and its gradient the object gradient
    rc = ptycho::regularise(*p, reinterpret_cast<const float2*>(O), s->reg_l1, s->reg_tv, s->reg_eta, p->d_gO,
                            loss_dev, st);
    if (rc) return rc;
  }
  const long long nO = 2 * p->O_numel, nP = 2 * p->P_numel;
  const long long FF = (long long)p->F * p->F;
  const long long nD = 2ll * p->L * p->J;
  const int grid = 4 * p->sms;
  if (s->t_dev) {
    // device step counter: the update can be captured once and replayed
    ptycho::k_tick<<<1, 32, 0, st>>>(s->t_dev);
    ++p->last_launches;
    if (cudaGetLastError() != cudaSuccess) return PTYCHO_ECUDA;
    long long ev = ptycho::prof_begin(*p, ptycho::kAdam, st);
    ptycho::k_adam_dev<<<grid, 256, 0, st>>>(O, reinterpret_cast<const float*>(p->d_gO), s->mO, s->vO, nO, s->lr_O,
                                             s->beta1, s->beta2, s->eps, s->t_dev);
    ptycho::k_adam_dev<<<grid, 256, 0, st>>>(P, reinterpret_cast<const float*>(p->d_gP), s->mP, s->vP, nP, s->lr_P,
                                             s->beta1, s->beta2, s->eps, s->t_dev);
    p->last_launches += 2;
    if (opt_sigma) {
      ptycho::k_adam_dev<<<(p->J + 255) / 256, 256, 0, st>>>(sigma, p->d_gsig, s->m_sigma, s->v_sigma, p->J,
                                                             s->lr_sigma, s->beta1, s->beta2, s->eps, s->t_dev);
      ++p->last_launches;
    }
    if (opt_bg) {
      ptycho::k_adam_dev<<<(int)((FF + 255) / 256), 256, 0, st>>>(bg, p->d_gbg, s->m_bg, s->v_bg, FF, s->lr_bg,
                                                                   s->beta1, s->beta2, s->eps, s->t_dev);
      ++p->last_launches;
    }
    if (opt_delta) {
      ptycho::k_adam_dev<<<(int)((nD + 255) / 256), 256, 0, st>>>(p->d_delta, p->d_gdelta, s->m_delta, s->v_delta, nD,
                                                                   s->lr_delta, s->beta1, s->beta2, s->eps, s->t_dev);
      ++p->last_launches;
    }
    if (cudaGetLastError() != cudaSuccess) return PTYCHO_ECUDA;
    ptycho::prof_end(*p, ev, st);
    return PTYCHO_OK;
  }
  s->t += 1;
  const double c1 = 1.0 / (1.0 - pow((double)s->beta1, (double)s->t));
  const double c2 = 1.0 / (1.0 - pow((double)s->beta2, (double)s->t));
  long long ev = ptycho::prof_begin(*p, ptycho::kAdam, st);
  ptycho::k_adam<<<grid, 256, 0, st>>>(O, reinterpret_cast<const float*>(p->d_gO), s->mO, s->vO, nO, s->lr_O,
                                       s->beta1, s->beta2, s->eps, (float)c1, (float)c2);
  ++p->last_launches;
  if (cudaGetLastError() != cudaSuccess) return PTYCHO_ECUDA;
  ptycho::prof_end(*p, ev, st);
  ev = ptycho::prof_begin(*p, ptycho::kAdam, st);
  ptycho::k_adam<<<grid, 256, 0, st>>>(P, reinterpret_cast<const float*>(p->d_gP), s->mP, s->vP, nP, s->lr_P,
                                       s->beta1, s->beta2, s->eps, (float)c1, (float)c2);
  ++p->last_launches;
  if (cudaGetLastError() != cudaSuccess) return PTYCHO_ECUDA;
  ptycho::prof_end(*p, ev, st);
  if (opt_sigma) {
    ptycho::k_adam<<<(p->J + 255) / 256, 256, 0, st>>>(sigma, p->d_gsig, s->m_sigma, s->v_sigma, p->J, s->lr_sigma,
                                                       s->beta1, s->beta2, s->eps, (float)c1, (float)c2);
    ++p->last_launches;
  }
  if (opt_bg) {
    ptycho::k_adam<<<(int)((FF + 255) / 256), 256, 0, st>>>(bg, p->d_gbg, s->m_bg, s->v_bg, FF, s->lr_bg, s->beta1,
                                                             s->beta2, s->eps, (float)c1, (float)c2);
    ++p->last_launches;
  }
  if (opt_delta) {
    ptycho::k_adam<<<(int)((nD + 255) / 256), 256, 0, st>>>(p->d_delta, p->d_gdelta, s->m_delta, s->v_delta, nD,
                                                             s->lr_delta, s->beta1, s->beta2, s->eps, (float)c1,
                                                             (float)c2);
    ++p->last_launches;
  }
  if (cudaGetLastError() != cudaSuccess) return PTYCHO_ECUDA;
  return PTYCHO_OK;
}

int ptycho_step_host(ptycho_plan_t* p, ptycho_adam_t* s, float* O, float* P, float* sigma, float* bg,
                     const float* I_meas_host, float* I_meas_dev, const uint8_t* mask, int mask_per_frame,
                     const int32_t* batch_idx, int nbatch, double* loss_dev, double* loss_host, void* stream) {
  if (!p || !I_meas_host || !I_meas_dev || !loss_dev || !loss_host) return PTYCHO_EINVAL;
  int rc = check_device(p);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t frame = sizeof(float) * (size_t)p->F * (size_t)p->F;
  const int nbat = (p->J + p->B - 1) / p->B;
  if (batch_idx || !p->store || p->nchunks != 1) {
    // positions in any order (or one position at a time): one copy before the step
    if (cudaMemcpyAsync(I_meas_dev, I_meas_host, frame * (size_t)p->J, cudaMemcpyHostToDevice, st) != cudaSuccess) {
      cudaGetLastError();
      return PTYCHO_ECUDA;
    }
    rc = ptycho_step(p, s, O, P, sigma, bg, I_meas_dev, mask, mask_per_frame, batch_idx, nbatch, loss_dev, stream);
  } else {
    // all positions in order: batch k's frames are copied on a side stream after the work queued
    // on stream so far, and its loss kernel waits only for them, so the copies of later batches
    // overlap the transforms of earlier ones
    if (!p->copy_st && (cudaStreamCreateWithFlags(&p->copy_st, cudaStreamNonBlocking) != cudaSuccess ||
                        cudaEventCreateWithFlags(&p->ev_copy_start, cudaEventDisableTiming) != cudaSuccess)) {
      cudaGetLastError();
      return PTYCHO_ECUDA;
    }
    while ((int)p->ev_copy.size() < nbat) {
      cudaEvent_t e;
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return PTYCHO_ECUDA;
      p->ev_copy.push_back(e);
    }
    if (cudaEventRecord(p->ev_copy_start, st) != cudaSuccess ||
        cudaStreamWaitEvent(p->copy_st, p->ev_copy_start, 0) != cudaSuccess)
      return PTYCHO_ECUDA;
    for (int k = 0; k < nbat; ++k) {
      const size_t off = (size_t)k * p->B, n = (size_t)std::min(p->B, p->J - k * p->B);
      if (cudaMemcpyAsync(reinterpret_cast<char*>(I_meas_dev) + off * frame,
                          reinterpret_cast<const char*>(I_meas_host) + off * frame, n * frame,
                          cudaMemcpyHostToDevice, p->copy_st) != cudaSuccess ||
          cudaEventRecord(p->ev_copy[k], p->copy_st) != cudaSuccess) {
        cudaGetLastError();
        return PTYCHO_ECUDA;
      }
    }
    p->imeas_ready = p->ev_copy.data();
    rc = ptycho_step(p, s, O, P, sigma, bg, I_meas_dev, mask, mask_per_frame, batch_idx, nbatch, loss_dev, stream);
    p->imeas_ready = nullptr;
  }
  if (rc) return rc;
  if (cudaMemcpyAsync(loss_host, loss_dev, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess) {
    cudaGetLastError();
    return PTYCHO_ECUDA;
  }
  return PTYCHO_OK;
}

}  // extern "C"
