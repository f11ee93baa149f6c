// Instantiations of the thread-per-trajectory FP64 kernel (split for parallel builds).
#include "propagate_tpt.cuh"

namespace scivr {
template cudaError_t launch_tpt_fp64<1>(const PropLaunch &, cudaStream_t);
template cudaError_t launch_tpt_fp64<2>(const PropLaunch &, cudaStream_t);
template cudaError_t launch_tpt_fp64<3>(const PropLaunch &, cudaStream_t);
template cudaError_t launch_tpt_fp64<4>(const PropLaunch &, cudaStream_t);
}  // namespace scivr
