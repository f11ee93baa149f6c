// Instantiations of the lane-group propagation kernel (split for parallel builds).
#include "propagate_lg.cuh"

namespace scivr {

template <int F> constexpr int group_lanes() { return 2 * F <= 8 ? 8 : (2 * F <= 16 ? 16 : 32); }

template <int F> cudaError_t launch_group_mixed(const PropLaunch &L, cudaStream_t s)
{
    return launch_lg<F, group_lanes<F>(), float, group_lanes<F>() == 32 ? 2 : 4>(L, s);
}

template <int F>
cudaError_t launch_group_batch_mixed_F(int warps, const PropLaunch *items, const int2 *work, int n_work,
                                      int *counter, int n_sm, cudaStream_t s)
{
    constexpr int G = group_lanes<F>();
    if constexpr (G == 32) {
        if (warps == 1) return launch_lg_batch<F, G, float, 1>(items, work, n_work, counter, n_sm, s);
        if (warps == 2) return launch_lg_batch<F, G, float, 2>(items, work, n_work, counter, n_sm, s);
    } else {
        if (warps == 2) return launch_lg_batch<F, G, float, 2>(items, work, n_work, counter, n_sm, s);
        if (warps == 4) return launch_lg_batch<F, G, float, 4>(items, work, n_work, counter, n_sm, s);
    }
    return cudaErrorInvalidValue;
}

template <int F> cudaError_t launch_group_fp64(const PropLaunch &L, cudaStream_t s)
{
    return launch_lg<F, group_lanes<F>(), double, group_lanes<F>() == 32 ? 2 : 4>(L, s);
}

template cudaError_t launch_group_mixed<5>(const PropLaunch &, cudaStream_t);
template cudaError_t launch_group_fp64<5>(const PropLaunch &, cudaStream_t);
template cudaError_t launch_group_mixed<6>(const PropLaunch &, cudaStream_t);
template cudaError_t launch_group_fp64<6>(const PropLaunch &, cudaStream_t);

template cudaError_t launch_group_batch_mixed_F<5>(int, const PropLaunch *, const int2 *, int, int *, int, cudaStream_t);
template cudaError_t launch_group_batch_mixed_F<6>(int, const PropLaunch *, const int2 *, int, int *, int, cudaStream_t);

}  // namespace scivr
