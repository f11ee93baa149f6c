// Instantiations of the lane-group propagation kernel (split for parallel builds).
#include "propagate_lg.cuh"

namespace scivr {

template cudaError_t launch_group_mixed<7>(const PropLaunch &, cudaStream_t);
template cudaError_t launch_group_fp64<7>(const PropLaunch &, cudaStream_t);
template cudaError_t launch_group_mixed<8>(const PropLaunch &, cudaStream_t);
template cudaError_t launch_group_fp64<8>(const PropLaunch &, cudaStream_t);

template cudaError_t launch_group_batch_mixed_F<7>(int, const PropLaunch *, const int2 *, int, int *, int, cudaStream_t);
template cudaError_t launch_group_batch_mixed_F<8>(int, const PropLaunch *, const int2 *, int, int *, int, cudaStream_t);

}  // namespace scivr
