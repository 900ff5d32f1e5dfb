// Kernels and pipeline instantiated for 64x64 frames.
#include "pipeline.cuh"

namespace ptycho {
template int run_pipeline<64>(ptycho_plan& p, const CallArgs& c, cudaStream_t st);
template int prepare_kernels<64>();
}  // namespace ptycho
