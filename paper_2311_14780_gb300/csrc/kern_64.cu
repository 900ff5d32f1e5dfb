// Kernels and pipelines instantiated for 64x64 frames.
#include "pipeline.cuh"
#include "plain.cuh"

namespace ptycho {
template int run_pipeline<64>(ptycho_plan& p, const CallArgs& c, cudaStream_t st);
template int prepare_kernels<64>();
template int plain_adjoint<64>(ptycho_plan& p, const CallArgs& c, float2* psi, float* Ibuf, float* Dbuf, float* Gbuf,
                                int Bp, cudaStream_t st);
template int launch_round_multi<64>(const RoundTab& rt, const int* blocks, const int* d_tiles,
                                      const RowAdjClass* cls, int ncls, cudaStream_t st);
template cudaError_t prepare_multi<64>();
}  // namespace ptycho
