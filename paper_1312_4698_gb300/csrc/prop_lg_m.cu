// One persistent launch for a batch whose molecules span the batch recipe's F classes
// (3, 6, 9, 12, 15, 24): the multi-F lane-group kernel and its launcher.
#include "propagate_lg.cuh"

namespace scivr {

using BatchRecipeMulti = MultiLaunch<3, 6, 9, 12, 15, 24>;

bool multi_launch_holds(int F) { return BatchRecipeMulti::holds(F); }

int multi_launch_tile(int F) { return 4 * (32 / mixed_group_lanes(F)); }

cudaError_t launch_group_batch_multi(const PropLaunch *items, const int2 *work, int n_work, int *counter, int n_sm,
                                     cudaStream_t s)
{
    return BatchRecipeMulti::launch(items, work, n_work, counter, n_sm, s);
}

}  // namespace scivr
