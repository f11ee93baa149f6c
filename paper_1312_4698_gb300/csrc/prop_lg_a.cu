// Instantiations of the lane-group propagation kernel (split for parallel builds).
#include "propagate_lg.cuh"

namespace scivr {

template cudaError_t launch_group_mixed<1>(const PropLaunch &, cudaStream_t);
template cudaError_t launch_group_fp64<1>(const PropLaunch &, cudaStream_t);
template cudaError_t launch_group_mixed<2>(const PropLaunch &, cudaStream_t);
template cudaError_t launch_group_fp64<2>(const PropLaunch &, cudaStream_t);
template cudaError_t launch_group_mixed<3>(const PropLaunch &, cudaStream_t);
template cudaError_t launch_group_fp64<3>(const PropLaunch &, cudaStream_t);
template cudaError_t launch_group_mixed<4>(const PropLaunch &, cudaStream_t);
template cudaError_t launch_group_fp64<4>(const PropLaunch &, cudaStream_t);

template cudaError_t launch_group_batch_mixed_F<1>(int, const PropLaunch *, const int2 *, int, int *, int, cudaStream_t);
template cudaError_t launch_group_batch_mixed_F<2>(int, const PropLaunch *, const int2 *, int, int *, int, cudaStream_t);
template cudaError_t launch_group_batch_mixed_F<3>(int, const PropLaunch *, const int2 *, int, int *, int, cudaStream_t);
template cudaError_t launch_group_batch_mixed_F<4>(int, const PropLaunch *, const int2 *, int, int *, int, cudaStream_t);

}  // namespace scivr
