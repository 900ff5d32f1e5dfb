// Kernels and pipelines instantiated for 128x128 frames.
#include "pipeline.cuh"
#include "plain.cuh"

namespace ptycho {
template int run_pipeline<128>(ptycho_plan& p, const CallArgs& c, cudaStream_t st);
template int prepare_kernels<128>();
template int plain_adjoint<128>(ptycho_plan& p, const CallArgs& c, float2* psi, float* Ibuf, float* Dbuf, float* Gbuf,
                                int Bp, cudaStream_t st);
template int launch_round_multi<128>(const RoundTab& rt, const int* blocks, const int* d_tiles,
                                      const RowAdjClass* cls, int ncls, cudaStream_t st);
template cudaError_t prepare_multi<128>();
}  // namespace ptycho
