// Propagation dispatch: picks the kernel instantiation for (F, precision).
#include "scivr_internal.cuh"

namespace scivr {

template <int F> cudaError_t launch_tpt_fp64(const PropLaunch &L, cudaStream_t s);

bool propagate_supported(int F, int precision)
{
    if (precision != SCIVR_FP64) return false;
    return F >= 1 && F <= 9;
}

cudaError_t launch_propagate(const PropLaunch &L, cudaStream_t s, int *n_launch)
{
    *n_launch = 1;
    switch (L.args.F) {
    case 1: return launch_tpt_fp64<1>(L, s);
    case 2: return launch_tpt_fp64<2>(L, s);
    case 3: return launch_tpt_fp64<3>(L, s);
    case 4: return launch_tpt_fp64<4>(L, s);
    case 5: return launch_tpt_fp64<5>(L, s);
    case 6: return launch_tpt_fp64<6>(L, s);
    case 7: return launch_tpt_fp64<7>(L, s);
    case 8: return launch_tpt_fp64<8>(L, s);
    case 9: return launch_tpt_fp64<9>(L, s);
    default: *n_launch = 0; return cudaErrorInvalidValue;
    }
}

}  // namespace scivr
