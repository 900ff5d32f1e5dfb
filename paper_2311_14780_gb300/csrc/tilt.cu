// Data-side tilt correction: the tilted-plane remap of the measurement model applied once
// to the measured patterns, the way the paper preprocesses its reflection data (Section
// "Experimental setup and ptychography reconstruction": each camera pattern is interpolated
// non-uniformly onto a grid uniform in sample-plane spatial frequency, and the correction
// produces the mask of the reduced field of view; pixels outside the value thresholds are
// discarded).  The corrected patterns are then fitted by a plan built without the in-model
// remap.
//
// The camera position of a model pixel depends only on the geometry, so it is computed once
// per geometry: k_tilt_taps places every model pixel on the camera in FP64 (the camera index
// decides which four taps are read and whether the pixel is kept) and writes a table of
// bilinear weights and tap offsets (20 bytes per pixel).  k_tilt_apply streams the frames:
// one thread per model pixel reads its taps once and runs over a chunk of frames,
// kTiltUnroll frames at a time so that 4 x kTiltUnroll independent loads are in flight.  The
// apply pass is HBM-bound: per pattern F^2 x (4 B read + 4 B written + 1 B mask).
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include <cuda_runtime.h>

#include "ptycho.h"

namespace {

constexpr int kTiltThreads = 256;               // apply pass
constexpr int kTapThreads = 64;                  // table pass (FP64-bound: small blocks spread it over the SMs)
constexpr int kTiltUnroll = 4;                   // frames per thread and iteration
constexpr int kTiltChunk = 16;                   // frames per work item of the apply pass
constexpr int kTiltBlocksPerSM = 4;              // resident apply blocks per SM (<= 64 registers)

struct TiltGeom {
  double z, p;          // distance to the camera and camera pixel pitch (m)
  double da, db;        // model-grid spacings in direction cosines: p/z and (p/z) cos(tilt)
  double s, c;          // sin(tilt), cos(tilt)
  int F;
};

// Camera position (fractional indices y, x) of model pixel (i, k).  The model index gives
// the in-plane direction cosines b = (i - F/2) db, a = (k - F/2) da of the reflected ray;
// rotated by the tilt about the camera's x axis the ray is (a, b + sin, w) with
// w = sqrt(1 - a^2 - (b + sin)^2) >= 0 (it leaves the sample surface), so in the camera
// frame d_y = (b + sin) cos - w sin, d_z = (b + sin) sin + w cos, and it meets the camera at
// X = z a / d_z, Y = z d_y / d_z.  False when the ray does not exist or misses the camera.
// Every FP64 operation is rounded on its own (no contraction into FMAs), so the camera index,
// and the floor and range decisions taken from it, are those of the same formula evaluated
// in plain IEEE double arithmetic.
__device__ bool camera_index(const TiltGeom& g, int i, int k, double* y, double* x) {
  const double half = 0.5 * (double)g.F;
  const double b = __dmul_rn(__dsub_rn((double)i, half), g.db);
  const double a = __dmul_rn(__dsub_rn((double)k, half), g.da);
  const double u = __dadd_rn(b, g.s);
  const double w2 = __dsub_rn(__dsub_rn(1.0, __dmul_rn(a, a)), __dmul_rn(u, u));
  if (!(w2 > 0.0)) return false;
  const double w = __dsqrt_rn(w2);
  const double dy = __dsub_rn(__dmul_rn(u, g.c), __dmul_rn(w, g.s));
  const double dz = __dadd_rn(__dmul_rn(u, g.s), __dmul_rn(w, g.c));
  if (!(dz > 0.0)) return false;
  const double X = __ddiv_rn(__dmul_rn(g.z, a), dz);
  const double Y = __ddiv_rn(__dmul_rn(g.z, dy), dz);
  *y = __dadd_rn(__ddiv_rn(Y, g.p), half);
  *x = __dadd_rn(__ddiv_rn(X, g.p), half);
  return true;
}

// One thread per model pixel: w[pix] = weights of (y0, x0), (y0, x0+1), (y0+1, x0),
// (y0+1, x0+1); base[pix] = camera offset of the top-left tap, or -1 when the pixel is not kept.
// grid ceil(F^2 / kTapThreads)
__global__ void __launch_bounds__(kTapThreads)
k_tilt_taps(TiltGeom g, float4* __restrict__ w, int32_t* __restrict__ base) {
  const int F = g.F;
  const long long FF = (long long)F * F;
  const long long pix = (long long)blockIdx.x * kTapThreads + threadIdx.x;
  if (pix >= FF) return;
  int32_t b = -1;
  float4 wt = make_float4(0.f, 0.f, 0.f, 0.f);
  double y = 0.0, x = 0.0;
  if (camera_index(g, (int)(pix / F), (int)(pix % F), &y, &x) && y >= 0.0 && y < (double)(F - 1) && x >= 0.0 &&
      x < (double)(F - 1)) {
    const double fy = floor(y), fx = floor(x);
    const double u = y - fy, v = x - fx;
    b = (int32_t)fy * F + (int32_t)fx;
    wt = make_float4((float)((1.0 - u) * (1.0 - v)), (float)((1.0 - u) * v), (float)(u * (1.0 - v)), (float)(u * v));
  }
  w[pix] = wt;
  base[pix] = b;
}

__device__ __forceinline__ bool in_range(float v, float lo, float hi) { return (v >= lo) & (v < hi); }

// Persistent: work item i covers pixel block i % nblk and frames [kTiltChunk * (i / nblk), ...);
// block b takes items b, b + gridDim.x, ...   grid min(items, kTiltBlocksPerSM * SMs)
__global__ void __launch_bounds__(kTiltThreads, kTiltBlocksPerSM)
k_tilt_apply(const float* __restrict__ cam, long long J, int F, const float4* __restrict__ w,
             const int32_t* __restrict__ base, float lo, float hi, float* __restrict__ out, uint8_t* __restrict__ mask) {
  const long long FF = (long long)F * F;
  const long long nblk = (FF + kTiltThreads - 1) / kTiltThreads;
  const long long items = nblk * ((J + kTiltChunk - 1) / kTiltChunk);
  for (long long it = blockIdx.x; it < items; it += gridDim.x) {
    const long long pix = (it % nblk) * kTiltThreads + threadIdx.x;
    if (pix >= FF) continue;
    const long long j0 = (it / nblk) * kTiltChunk;
    const int n = (int)(j0 + kTiltChunk < J ? kTiltChunk : J - j0);
    const int32_t b = __ldg(base + pix);
    float* o = out + j0 * FF + pix;
    uint8_t* mk = mask ? mask + j0 * FF + pix : nullptr;
    if (b < 0) {                                      // not kept in any frame
      for (int k = 0; k < n; ++k) {
        o[k * FF] = 0.f;
        if (mk) mk[k * FF] = 0;
      }
      continue;
    }
    const float4 wt = __ldg(w + pix);
    const float* c = cam + j0 * FF + b;
    int k = 0;
    for (; k + kTiltUnroll <= n; k += kTiltUnroll) {
      float v[kTiltUnroll][4];
#pragma unroll
      for (int f = 0; f < kTiltUnroll; ++f) {
        const float* cf = c + (k + f) * FF;
        v[f][0] = __ldg(cf);
        v[f][1] = __ldg(cf + 1);
        v[f][2] = __ldg(cf + F);
        v[f][3] = __ldg(cf + F + 1);
      }
#pragma unroll
      for (int f = 0; f < kTiltUnroll; ++f) {
        const bool keep = in_range(v[f][0], lo, hi) & in_range(v[f][1], lo, hi) & in_range(v[f][2], lo, hi) &
                          in_range(v[f][3], lo, hi);
        const float val = fmaf(wt.w, v[f][3], fmaf(wt.z, v[f][2], fmaf(wt.y, v[f][1], wt.x * v[f][0])));
        o[(k + f) * FF] = keep ? val : 0.f;
        if (mk) mk[(k + f) * FF] = keep ? 1 : 0;
      }
    }
    for (; k < n; ++k) {
      const float* cf = c + k * FF;
      const float v0 = __ldg(cf), v1 = __ldg(cf + 1), v2 = __ldg(cf + F), v3 = __ldg(cf + F + 1);
      const bool keep = in_range(v0, lo, hi) & in_range(v1, lo, hi) & in_range(v2, lo, hi) & in_range(v3, lo, hi);
      const float val = fmaf(wt.w, v3, fmaf(wt.z, v2, fmaf(wt.y, v1, wt.x * v0)));
      o[k * FF] = keep ? val : 0.f;
      if (mk) mk[k * FF] = keep ? 1 : 0;
    }
  }
}

int check_geometry(int32_t F, double z, double det_pixel, double tilt_rad) {
  if (F < 2 || F > 8192) return PTYCHO_EINVAL;
  if (!(z > 0.0) || !isfinite(z) || !(det_pixel > 0.0) || !isfinite(det_pixel) || !isfinite(tilt_rad) ||
      !(fabs(tilt_rad) < 0.5 * M_PI))
    return PTYCHO_EINVAL;
  return PTYCHO_OK;
}

int launch_taps(int32_t F, double z, double det_pixel, double tilt_rad, void* table, cudaStream_t st) {
  TiltGeom g;
  g.z = z;
  g.p = det_pixel;
  g.c = cos(tilt_rad);
  g.s = sin(tilt_rad);
  g.da = det_pixel / z;
  g.db = g.da * g.c;
  g.F = F;
  const long long FF = (long long)F * F;
  float4* w = static_cast<float4*>(table);
  k_tilt_taps<<<(unsigned)((FF + kTapThreads - 1) / kTapThreads), kTapThreads, 0, st>>>(
      g, w, reinterpret_cast<int32_t*>(w + FF));
  return cudaGetLastError() == cudaSuccess ? PTYCHO_OK : PTYCHO_ECUDA;
}

int launch_apply(int32_t F, int64_t J, const void* table, const float* I_cam, float lo, float hi, float* I_model,
                 uint8_t* mask, cudaStream_t st) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return PTYCHO_ECUDA;
  const long long FF = (long long)F * F;
  const long long items = ((FF + kTiltThreads - 1) / kTiltThreads) * ((J + kTiltChunk - 1) / kTiltChunk);
  const long long grid = std::min<long long>(items, (long long)kTiltBlocksPerSM * sms);
  const float4* w = static_cast<const float4*>(table);
  k_tilt_apply<<<(unsigned)grid, kTiltThreads, 0, st>>>(I_cam, J, F, w, reinterpret_cast<const int32_t*>(w + FF), lo,
                                                        hi, I_model, mask);
  return cudaGetLastError() == cudaSuccess ? PTYCHO_OK : PTYCHO_ECUDA;
}

bool overlaps(const void* a, const void* b, long long bytes_a, long long bytes_b) {
  const char* x = static_cast<const char*>(a);
  const char* y = static_cast<const char*>(b);
  return x < y + bytes_b && y < x + bytes_a;
}

int check_apply(int32_t F, int64_t J, const void* table, const float* I_cam, float lo, float hi, float* I_model,
                uint8_t* mask) {
  if (F < 2 || F > 8192 || J < 0) return PTYCHO_EINVAL;
  if (isnan(lo) || isnan(hi) || !(lo < hi)) return PTYCHO_EINVAL;
  if (J == 0) return PTYCHO_OK;
  if (!I_cam || !I_model || !table || (reinterpret_cast<uintptr_t>(table) & 15)) return PTYCHO_EINVAL;
  const long long FF = (long long)F * F, img = J * FF * (long long)sizeof(float);
  const long long tb = FF * (long long)(sizeof(float4) + sizeof(int32_t));
  // the outputs must overlap neither the input nor the table, nor each other
  if (overlaps(I_cam, I_model, img, img) || overlaps(table, I_model, tb, img)) return PTYCHO_EINVAL;
  if (mask && (overlaps(mask, I_model, J * FF, img) || overlaps(mask, I_cam, J * FF, img) || overlaps(mask, table, J * FF, tb)))
    return PTYCHO_EINVAL;
  return PTYCHO_OK;
}

}  // namespace

extern "C" {

int64_t ptycho_tilt_table_bytes(int32_t F) {
  if (F < 2 || F > 8192) return -1;
  return (int64_t)F * F * (int64_t)(sizeof(float4) + sizeof(int32_t));
}

int ptycho_tilt_table(int32_t F, double z, double det_pixel, double tilt_rad, void* table, void* stream) {
  const int rc = check_geometry(F, z, det_pixel, tilt_rad);
  if (rc) return rc;
  if (!table || (reinterpret_cast<uintptr_t>(table) & 15)) return PTYCHO_EINVAL;
  return launch_taps(F, z, det_pixel, tilt_rad, table, static_cast<cudaStream_t>(stream));
}

int ptycho_tilt_apply(int32_t F, int64_t J, const void* table, const float* I_cam, float lo, float hi,
                      float* I_model, uint8_t* mask, void* stream) {
  const int rc = check_apply(F, J, table, I_cam, lo, hi, I_model, mask);
  if (rc || J == 0) return rc;
  return launch_apply(F, J, table, I_cam, lo, hi, I_model, mask, static_cast<cudaStream_t>(stream));
}

int ptycho_tilt_correct(int32_t F, int64_t J, double z, double det_pixel, double tilt_rad, const float* I_cam,
                        float lo, float hi, float* I_model, uint8_t* mask, void* stream) {
  int rc = check_geometry(F, z, det_pixel, tilt_rad);
  if (rc) return rc;
  if (J < 0 || isnan(lo) || isnan(hi) || !(lo < hi)) return PTYCHO_EINVAL;
  if (J == 0) return PTYCHO_OK;
  if (!I_cam || !I_model) return PTYCHO_EINVAL;
  const long long FF = (long long)F * F, img = J * FF * (long long)sizeof(float);
  if (overlaps(I_cam, I_model, img, img) ||
      (mask && (overlaps(mask, I_model, J * FF, img) || overlaps(mask, I_cam, J * FF, img))))
    return PTYCHO_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  void* table = nullptr;
  if (cudaMallocAsync(&table, (size_t)ptycho_tilt_table_bytes(F), st) != cudaSuccess) {
    cudaGetLastError();
    return PTYCHO_ENOMEM;
  }
  rc = launch_taps(F, z, det_pixel, tilt_rad, table, st);
  if (!rc) rc = launch_apply(F, J, table, I_cam, lo, hi, I_model, mask, st);
  if (cudaFreeAsync(table, st) != cudaSuccess && !rc) rc = PTYCHO_ECUDA;
  return rc;
}

}  // extern "C"
