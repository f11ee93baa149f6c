// Instantiations of the lane-group propagation kernel (split for parallel builds).
#include "propagate_lg.cuh"

namespace scivr {

template <int F> constexpr int group_lanes() { return 2 * F <= 8 ? 8 : (2 * F <= 16 ? 16 : 32); }

template <int F> cudaError_t launch_group_mixed(const PropLaunch &L, cudaStream_t s)
{
    return launch_lg<F, group_lanes<F>(), float, group_lanes<F>() == 32 ? 2 : 4>(L, s);
}

template <int F> cudaError_t launch_group_fp64(const PropLaunch &L, cudaStream_t s)
{
    return launch_lg<F, group_lanes<F>(), double, group_lanes<F>() == 32 ? 2 : 4>(L, s);
}

template cudaError_t launch_group_mixed<9>(const PropLaunch &, cudaStream_t);
template cudaError_t launch_group_fp64<9>(const PropLaunch &, cudaStream_t);

}  // namespace scivr
