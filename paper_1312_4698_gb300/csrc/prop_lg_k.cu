// Instantiations of the lane-group propagation kernel above F = 16 (two monodromy
// columns per lane, coupling tensors read from L2; mixed precision only; split for
// parallel builds).
#include "propagate_lg.cuh"

namespace scivr {

template cudaError_t launch_group_mixed<21>(const PropLaunch &, cudaStream_t);
template cudaError_t launch_group_mixed<22>(const PropLaunch &, cudaStream_t);

template cudaError_t launch_group_batch_mixed_F<21>(int, const PropLaunch *, const int2 *, int, int *, int, cudaStream_t);
template cudaError_t launch_group_batch_mixed_F<22>(int, const PropLaunch *, const int2 *, int, int *, int, cudaStream_t);

}  // namespace scivr
