// Data-side tilt correction: the tilted-plane remap of the measurement model applied once
// to the measured patterns, the way the paper preprocesses its reflection data (Section
// "Experimental setup and ptychography reconstruction": each camera pattern is interpolated
// non-uniformly onto a grid uniform in sample-plane spatial frequency, and the correction
// produces the mask of the reduced field of view; pixels outside the value thresholds are
// discarded).  The corrected patterns are then fitted by a plan built without the in-model
// remap.
//
// One block owns kTiltPix consecutive model pixels and a range of frames.  Its first
// kTiltPix threads place their pixel on the camera in FP64 (the camera index decides which
// four taps are read and whether the pixel is kept) and leave the tap offset and the four
// bilinear weights in shared memory; then all kTiltLanes x kTiltPix threads stream the
// frames, kTiltUnroll frames per thread at a time so that 4 x kTiltUnroll independent loads
// are in flight.  HBM-bound: per pattern F^2 x (4 B read + 4 B write + 1 B mask).
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include <cuda_runtime.h>

#include "ptycho.h"

namespace {

constexpr int kTiltPix = 64;                     // model pixels per block
constexpr int kTiltLanes = 4;                    // frame lanes per pixel
constexpr int kTiltThreads = kTiltPix * kTiltLanes;
constexpr int kTiltUnroll = 4;                   // frames per lane and iteration

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

struct TiltTap {
  long long base;       // camera offset of the top-left tap, or -1 when the pixel is not kept
  float w[4];           // weights of (y0, x0), (y0, x0+1), (y0+1, x0), (y0+1, x0+1)
};

// grid (ceil(F^2 / kTiltPix), ceil(J / frames_per_block)), block kTiltThreads
__global__ void __launch_bounds__(kTiltThreads, 4)
k_tilt_correct(const float* __restrict__ cam, long long J, TiltGeom g, float lo, float hi, long long frames_per_block,
               float* __restrict__ out, uint8_t* __restrict__ mask) {
  __shared__ TiltTap tap[kTiltPix];
  const int F = g.F;
  const long long FF = (long long)F * F;
  const int q = threadIdx.x % kTiltPix, lane = threadIdx.x / kTiltPix;
  const long long pix = (long long)blockIdx.x * kTiltPix + q;
  if (lane == 0) {
    TiltTap t{-1, {0.f, 0.f, 0.f, 0.f}};
    double y = 0.0, x = 0.0;
    if (pix < FF && camera_index(g, (int)(pix / F), (int)(pix % F), &y, &x) && y >= 0.0 &&
        y < (double)(F - 1) && x >= 0.0 && x < (double)(F - 1)) {
      const double fy = floor(y), fx = floor(x);
      const double u = y - fy, v = x - fx;
      t.base = (long long)fy * F + (long long)fx;
      t.w[0] = (float)((1.0 - u) * (1.0 - v));
      t.w[1] = (float)((1.0 - u) * v);
      t.w[2] = (float)(u * (1.0 - v));
      t.w[3] = (float)(u * v);
    }
    tap[q] = t;
  }
  __syncthreads();
  if (pix >= FF) return;
  const TiltTap t = tap[q];
  const long long j0 = (long long)blockIdx.y * frames_per_block;
  const long long j1 = j0 + frames_per_block < J ? j0 + frames_per_block : J;
  for (long long jb = j0 + lane; jb < j1; jb += kTiltLanes * kTiltUnroll) {
    float v[kTiltUnroll][4];
#pragma unroll
    for (int f = 0; f < kTiltUnroll; ++f) {
      const long long j = jb + (long long)f * kTiltLanes;
      if (t.base >= 0 && j < j1) {
        const float* c = cam + j * FF + t.base;
        v[f][0] = __ldg(c);
        v[f][1] = __ldg(c + 1);
        v[f][2] = __ldg(c + F);
        v[f][3] = __ldg(c + F + 1);
      } else {
        v[f][0] = v[f][1] = v[f][2] = v[f][3] = 0.f;
      }
    }
#pragma unroll
    for (int f = 0; f < kTiltUnroll; ++f) {
      const long long j = jb + (long long)f * kTiltLanes;
      if (j >= j1) break;
      bool keep = t.base >= 0;
      float val = 0.f;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        keep = keep && v[f][e] >= lo && v[f][e] < hi;
        val = fmaf(t.w[e], v[f][e], val);
      }
      out[j * FF + pix] = keep ? val : 0.f;
      if (mask) mask[j * FF + pix] = keep ? 1 : 0;
    }
  }
}

}  // namespace

extern "C" int ptycho_tilt_correct(int32_t F, int64_t J, double z, double det_pixel, double tilt_rad,
                                   const float* I_cam, float lo, float hi, float* I_model, uint8_t* mask,
                                   void* stream) {
  if (F < 2 || F > 8192 || J < 0) return PTYCHO_EINVAL;
  if (!(z > 0.0) || !isfinite(z) || !(det_pixel > 0.0) || !isfinite(det_pixel) || !isfinite(tilt_rad) ||
      !(fabs(tilt_rad) < 0.5 * M_PI))
    return PTYCHO_EINVAL;
  if (isnan(lo) || isnan(hi) || !(lo < hi)) return PTYCHO_EINVAL;
  if (J == 0) return PTYCHO_OK;
  if (!I_cam || !I_model) return PTYCHO_EINVAL;
  const long long FF = (long long)F * F;
  // the output must not overlap the input (blocks read camera pixels of other blocks' outputs)
  {
    const char* a0 = reinterpret_cast<const char*>(I_cam);
    const char* b0 = reinterpret_cast<const char*>(I_model);
    const long long bytes = J * FF * (long long)sizeof(float);
    if (a0 < b0 + bytes && b0 < a0 + bytes) return PTYCHO_EINVAL;
  }
  TiltGeom g;
  g.z = z;
  g.p = det_pixel;
  g.c = cos(tilt_rad);
  g.s = sin(tilt_rad);
  g.da = det_pixel / z;
  g.db = g.da * g.c;
  g.F = F;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return PTYCHO_ECUDA;
  const long long gx = (FF + kTiltPix - 1) / kTiltPix;
  if (gx > 0x7fffffffll) return PTYCHO_EINVAL;
  // at least eight blocks per SM in all; each frame chunk places its pixels again (FP64)
  long long chunks = std::max<long long>(1, (8ll * sms + gx - 1) / gx);
  chunks = std::min<long long>(chunks, std::min<long long>(J, 65535));
  const long long per = (J + chunks - 1) / chunks;
  chunks = (J + per - 1) / per;
  k_tilt_correct<<<dim3((unsigned)gx, (unsigned)chunks), kTiltThreads, 0, static_cast<cudaStream_t>(stream)>>>(
      I_cam, J, g, lo, hi, per, I_model, mask);
  return cudaGetLastError() == cudaSuccess ? PTYCHO_OK : PTYCHO_ECUDA;
}
