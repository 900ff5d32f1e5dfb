// Host entry point of the plain (unfused) baseline; its kernels live in plain.cuh and are
// instantiated per frame size in kern_<F>.cu.
#include <math.h>

#include <algorithm>

#include "plan.h"

namespace {
constexpr long long kPlainBuffer = 512ll << 20;   // exit-wave buffer of the plain form (HBM)
}

extern "C" int ptycho_plain_step(ptycho_plan_t* p, ptycho_adam_t* s, float* O, float* P, const float* sigma,
                                 const float* bg, const float* I_meas, const uint8_t* mask, int mask_per_frame,
                                 double* loss_dev, void* stream) {
  if (!p || !s || !O || !P || !I_meas || !s->mO || !s->vO || !s->mP || !s->vP) return PTYCHO_EINVAL;
  if (s->lr_sigma > 0.f || s->lr_bg > 0.f || s->lr_delta > 0.f || p->d_delta || s->g_z || p->czt ||
      s->reg_l1 != 0.f || s->reg_tv != 0.f)
    return PTYCHO_EUNSUPPORTED;                      // O and P at integer positions only
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != p->dev) return PTYCHO_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const long long FF = (long long)p->F * p->F;
  const long long LM = (long long)p->L * p->M;
  const int Bp = (int)std::max<long long>(1, std::min<long long>(p->J, kPlainBuffer / (LM * FF * 8)));
  // the plain form allocates its buffers per call (stream-ordered), as an unfused framework
  // would: exit waves [Bp][L*M][F][F], then intensities, dL/dI and R^T dL/dI, [Bp][F][F] each
  void* buf = nullptr;
  const size_t psi_bytes = sizeof(float2) * (size_t)(Bp * LM * FF), frame_bytes = sizeof(float) * (size_t)(Bp * FF);
  if (cudaMallocAsync(&buf, psi_bytes + 3 * frame_bytes, st) != cudaSuccess) return PTYCHO_ENOMEM;
  float2* psi = static_cast<float2*>(buf);
  float* Ibuf = reinterpret_cast<float*>(static_cast<char*>(buf) + psi_bytes);
  float* Dbuf = reinterpret_cast<float*>(static_cast<char*>(buf) + psi_bytes + frame_bytes);
  float* Gbuf = reinterpret_cast<float*>(static_cast<char*>(buf) + psi_bytes + 2 * frame_bytes);
  ptycho::CallArgs c{};
  c.kind = ptycho::CallKind::Adjoint;
  c.O = reinterpret_cast<const float2*>(O);
  c.P = reinterpret_cast<const float2*>(P);
  c.sigma = sigma;
  c.bg = bg;
  c.Imeas = I_meas;
  c.mask = mask;
  c.mask_per_frame = mask_per_frame ? 1 : 0;
  c.bidx = p->d_ident;
  c.nbatch = p->J;
  c.gO = p->d_gO;
  c.gP = p->d_gP;
  c.loss = loss_dev;
  int rc = 0;
  switch (p->F) {
    case 64: rc = ptycho::plain_adjoint<64>(*p, c, psi, Ibuf, Dbuf, Gbuf, Bp, st); break;
    case 128: rc = ptycho::plain_adjoint<128>(*p, c, psi, Ibuf, Dbuf, Gbuf, Bp, st); break;
    case 256: rc = ptycho::plain_adjoint<256>(*p, c, psi, Ibuf, Dbuf, Gbuf, Bp, st); break;
    default: rc = ptycho::plain_adjoint<512>(*p, c, psi, Ibuf, Dbuf, Gbuf, Bp, st); break;
  }
  cudaFreeAsync(buf, st);
  if (rc) return rc;
  s->t += 1;
  const double c1 = 1.0 / (1.0 - pow((double)s->beta1, (double)s->t));
  const double c2 = 1.0 / (1.0 - pow((double)s->beta2, (double)s->t));
  const int grid = 4 * p->sms;
  ptycho::k_adam<<<grid, 256, 0, st>>>(O, reinterpret_cast<const float*>(p->d_gO), s->mO, s->vO, 2 * p->O_numel,
                                       s->lr_O, s->beta1, s->beta2, s->eps, (float)c1, (float)c2);
  ptycho::k_adam<<<grid, 256, 0, st>>>(P, reinterpret_cast<const float*>(p->d_gP), s->mP, s->vP, 2 * p->P_numel,
                                       s->lr_P, s->beta1, s->beta2, s->eps, (float)c1, (float)c2);
  p->last_launches += 2;
  return cudaGetLastError() == cudaSuccess ? PTYCHO_OK : PTYCHO_ECUDA;
}
