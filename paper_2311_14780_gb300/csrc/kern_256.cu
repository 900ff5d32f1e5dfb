// Kernels and pipeline instantiated for 256x256 frames.
#include "pipeline.cuh"

namespace ptycho {
template int run_pipeline<256>(ptycho_plan& p, const CallArgs& c, cudaStream_t st);
template int prepare_kernels<256>();
}  // namespace ptycho
