// Instantiations of the lane-group propagation kernel (split for parallel builds).
#include "propagate_lg.cuh"

namespace scivr {

template cudaError_t launch_group_mixed<5>(const PropLaunch &, cudaStream_t);
template cudaError_t launch_group_fp64<5>(const PropLaunch &, cudaStream_t);
template cudaError_t launch_group_mixed<6>(const PropLaunch &, cudaStream_t);
template cudaError_t launch_group_fp64<6>(const PropLaunch &, cudaStream_t);

template cudaError_t launch_group_batch_mixed_F<5>(int, const PropLaunch *, const int2 *, int, int *, int, cudaStream_t);
template cudaError_t launch_group_batch_mixed_F<6>(int, const PropLaunch *, const int2 *, int, int *, int, cudaStream_t);

}  // namespace scivr
