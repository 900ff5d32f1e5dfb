// Kernels and pipeline instantiated for 512x512 frames.
#include "pipeline.cuh"

namespace ptycho {
template int run_pipeline<512>(ptycho_plan& p, const CallArgs& c, cudaStream_t st);
template int prepare_kernels<512>();
}  // namespace ptycho
