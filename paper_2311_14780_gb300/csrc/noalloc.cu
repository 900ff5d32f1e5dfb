// Allocation-free forward model: the same row-DFT -> column-DFT -> measurement kernels as
// ptycho_forward, with every intermediate (twiddles, positions, the complex field scratch and
// the per-position intensity sums) placed in one fixed, file-scope device array instead of a
// plan's cudaMalloc'd workspace.
//
// Who needs it: callers that cannot call cudaMalloc once they are running, for example an
// application that hands all device memory to its own pool at start-up and forbids other
// allocations, a latency-critical loop that cannot accept the implicit synchronisation an
// allocation may cause, or a deployment whose rules ban dynamic allocation after
// initialisation.  This entry point never calls cudaMalloc, cudaFree or any routine that
// allocates device memory; it only copies small host tables into the fixed array.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "plan.h"

namespace {

// The fixed scratch.  Every GPU that loads this library reserves it until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[PTYCHO_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {};     // device address of g_noalloc_scratch, per device
int g_sms[kMaxDevices] = {};

// Once per device, with that device current: look up the array's device address (the host
// symbol is only a stand-in and must never be handed to a kernel).
int setup_device(int dev) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (g_scratch_ptr[dev]) return PTYCHO_OK;
  void* ptr = nullptr;
  if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
    cudaGetLastError();
    return PTYCHO_ECUDA;
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PTYCHO_ECUDA;
  g_sms[dev] = sms;
  g_scratch_ptr[dev] = ptr;
  return PTYCHO_OK;
}

long long align256(long long x) { return (x + 255) & ~255ll; }

int fft_shape(int F, int* N1, int* N2) {
  switch (F) {
    case 64: *N1 = ptycho::FftShape<64>::N1; *N2 = ptycho::FftShape<64>::N2; return PTYCHO_OK;
    case 128: *N1 = ptycho::FftShape<128>::N1; *N2 = ptycho::FftShape<128>::N2; return PTYCHO_OK;
    case 256: *N1 = ptycho::FftShape<256>::N1; *N2 = ptycho::FftShape<256>::N2; return PTYCHO_OK;
    case 512: *N1 = ptycho::FftShape<512>::N1; *N2 = ptycho::FftShape<512>::N2; return PTYCHO_OK;
  }
  return PTYCHO_EUNSUPPORTED;
}

}  // namespace

extern "C" int ptycho_forward_noalloc(int32_t L, int32_t M, int32_t F, int32_t J, const int32_t* obj_h,
                                      const int32_t* obj_w, const int32_t* pos, const float* O, const float* P,
                                      const float* sigma, const float* bg, float* I_pred, void* stream) {
  if (L < 1 || M < 1 || J < 1 || !obj_h || !obj_w || !pos || !O || !P || !I_pred) return PTYCHO_EINVAL;
  int N1 = 0, N2 = 0;
  if (L > ptycho::kMaxL || fft_shape(F, &N1, &N2) != PTYCHO_OK) return PTYCHO_EUNSUPPORTED;
  for (int l = 0; l < L; ++l)
    if (obj_h[l] < F || obj_w[l] < F) return PTYCHO_EINVAL;

  // layout of the fixed array: twiddles | positions | position list | status | intensity
  // sums [B][F][F] | field scratch [B][C][F][F]; decided (and a problem that cannot fit
  // refused) before any position is read
  const long long FF = (long long)F * F;
  const long long LJ = (long long)L * J;
  const long long off_tw = 0;
  const long long off_pos = align256(off_tw + (long long)F * (long long)sizeof(float2));
  const long long off_ident = align256(off_pos + LJ * 2 * (long long)sizeof(int32_t));
  const long long off_status = align256(off_ident + (long long)J * (long long)sizeof(int32_t));
  const long long off_data = align256(off_status + (long long)sizeof(int));
  const long long avail = (long long)PTYCHO_NOALLOC_SCRATCH_BYTES - off_data;
  const long long LM = (long long)L * M;
  const long long frame_c = FF * (long long)sizeof(float2), frame_f = FF * (long long)sizeof(float);
  int B = 1, C = 1, nchunks = 1;
  if (avail >= frame_f + LM * frame_c) {
    C = (int)LM;
    B = (int)std::min<long long>(J, avail / (frame_f + LM * frame_c));
    B = std::max(1, std::min(B, 32));
  } else if (avail >= frame_f + frame_c) {
    C = (int)((avail - frame_f) / frame_c);
    nchunks = (int)((LM + C - 1) / C);
  } else {
    return PTYCHO_ETOOLARGE;
  }
  if (off_data + align256((long long)B * frame_f) + (long long)B * C * frame_c > (long long)PTYCHO_NOALLOC_SCRATCH_BYTES)
    return PTYCHO_ETOOLARGE;

  for (long long e = 0; e < LJ; ++e) {
    const long long l = e / J;
    const int y = pos[2 * e], x = pos[2 * e + 1];
    if (y < 0 || x < 0 || y > obj_h[l] - F || x > obj_w[l] - F) return PTYCHO_ERANGE;
  }

  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PTYCHO_ECUDA;
  int rc = setup_device(dev);
  if (rc) return rc;
  unsigned char* base = static_cast<unsigned char*>(g_scratch_ptr[dev]);
  cudaStream_t st = (cudaStream_t)stream;

  // small host tables, copied into the fixed array on the caller's stream
  float2 tw[512];
  for (int t = 0; t < N1; ++t)
    for (int k2 = 0; k2 < N2; ++k2) {
      const double ang = -2.0 * 3.14159265358979323846 * (double)((t * k2) % F) / (double)F;
      tw[k2 * N1 + t] = make_float2((float)cos(ang), (float)sin(ang));
    }
  if (cudaMemcpyAsync(base + off_tw, tw, sizeof(float2) * (size_t)F, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(base + off_pos, pos, sizeof(int32_t) * (size_t)LJ * 2, cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaMemsetAsync(base + off_status, 0, sizeof(int), st) != cudaSuccess)
    return PTYCHO_ECUDA;
  // position list 0..J-1, written in chunks through a small host buffer
  int32_t ids[1024];
  for (int j0 = 0; j0 < J; j0 += 1024) {
    const int n = std::min(1024, J - j0);
    for (int k = 0; k < n; ++k) ids[k] = j0 + k;
    if (cudaMemcpyAsync(base + off_ident + (long long)j0 * sizeof(int32_t), ids, sizeof(int32_t) * (size_t)n,
                        cudaMemcpyHostToDevice, st) != cudaSuccess)
      return PTYCHO_ECUDA;
  }

  // a plan view over the fixed array (host struct only; nothing is allocated)
  ptycho_plan view;
  view.dev = dev;
  view.sms = g_sms[dev];
  view.L = L; view.M = M; view.F = F; view.J = J;
  view.remap = 0;
  long long o = 0;
  for (int l = 0; l < L; ++l) {
    view.obj_h[l] = obj_h[l];
    view.obj_w[l] = obj_w[l];
    view.obj_off[l] = o;
    o += (long long)obj_h[l] * obj_w[l];
  }
  view.O_numel = o;
  view.P_numel = LM * FF;
  view.store = 0;
  view.B = B; view.C = C; view.nchunks = nchunks; view.G = 1; view.MG = C;
  view.d_tw = reinterpret_cast<float2*>(base + off_tw);
  view.d_pos = reinterpret_cast<int32_t*>(base + off_pos);
  view.d_ident = reinterpret_cast<int32_t*>(base + off_ident);
  view.d_status = reinterpret_cast<int*>(base + off_status);
  view.d_Ipart = reinterpret_cast<float*>(base + off_data);
  view.d_S = reinterpret_cast<float2*>(base + off_data + align256((long long)B * frame_f));

  ptycho::CallArgs c{};
  c.kind = ptycho::CallKind::Forward;
  c.O = reinterpret_cast<const float2*>(O);
  c.P = reinterpret_cast<const float2*>(P);
  c.sigma = sigma;
  c.bg = bg;
  c.I_pred = I_pred;
  c.bidx = view.d_ident;
  c.nbatch = J;
  switch (F) {
    case 64: return ptycho::run_pipeline<64>(view, c, st);
    case 128: return ptycho::run_pipeline<128>(view, c, st);
    case 256: return ptycho::run_pipeline<256>(view, c, st);
    default: return ptycho::run_pipeline<512>(view, c, st);
  }
}
