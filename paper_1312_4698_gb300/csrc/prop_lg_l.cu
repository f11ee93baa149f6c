// Instantiations of the lane-group propagation kernel above F = 16 (two monodromy
// columns per lane, coupling tensors read from L2; mixed precision only; split for
// parallel builds).
#include "propagate_lg.cuh"

namespace scivr {

template cudaError_t launch_group_mixed<23>(const PropLaunch &, cudaStream_t);
template cudaError_t launch_group_mixed<24>(const PropLaunch &, cudaStream_t);

template cudaError_t launch_group_batch_mixed_F<23>(int, const PropLaunch *, const int2 *, int, int *, int, cudaStream_t);
template cudaError_t launch_group_batch_mixed_F<24>(int, const PropLaunch *, const int2 *, int, int *, int, cudaStream_t);

}  // namespace scivr
