// Instantiations of the lane-group propagation kernel for the wide groups (F > 9: one
// trajectory per warp, mixed precision only; split for parallel builds).
#include "propagate_lg.cuh"

namespace scivr {

template cudaError_t launch_group_mixed<16>(const PropLaunch &, cudaStream_t);

template cudaError_t launch_group_batch_mixed_F<16>(int, const PropLaunch *, const int2 *, int, int *, int, cudaStream_t);

}  // namespace scivr
