// Kernels and pipeline instantiated for 128x128 frames.
#include "pipeline.cuh"

namespace ptycho {
template int run_pipeline<128>(ptycho_plan& p, const CallArgs& c, cudaStream_t st);
template int prepare_kernels<128>();
}  // namespace ptycho
