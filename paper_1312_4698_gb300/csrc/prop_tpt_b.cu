// Instantiations of the thread-per-trajectory FP64 kernel (split for parallel builds).
#include "propagate_tpt.cuh"

namespace scivr {
template cudaError_t launch_tpt_fp64<5>(const PropLaunch &, cudaStream_t);
template cudaError_t launch_tpt_fp64<6>(const PropLaunch &, cudaStream_t);
}  // namespace scivr
