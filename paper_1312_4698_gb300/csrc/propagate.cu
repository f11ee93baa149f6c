// Propagation dispatch: picks the kernel instantiation for (F, precision, schedule).
#include "scivr_internal.cuh"

namespace scivr {

template <int F> cudaError_t launch_tpt_fp64(const PropLaunch &L, cudaStream_t s);
template <int F> cudaError_t launch_group_mixed(const PropLaunch &L, cudaStream_t s);
template <int F> cudaError_t launch_group_fp64(const PropLaunch &L, cudaStream_t s);
template <int F>
cudaError_t launch_group_batch_mixed_F(int warps, const PropLaunch *items, const int2 *work, int n_work,
                                      int *counter, int n_sm, cudaStream_t s);

int batch_warp_candidates(int F, int *out)
{
    if (F < 1 || F > 24) return 0;
    if (F > 9) { out[0] = F <= 12 ? 8 : 4; return 1; }   // wide groups: one CTA per SM shares the tensors
    if (mixed_group_lanes(F) == 32) { out[0] = 1; out[1] = 2; }
    else { out[0] = 2; out[1] = 4; }
    return 2;
}

cudaError_t launch_group_batch_mixed(int F, int warps, const PropLaunch *items, const int2 *work, int n_work,
                                     int *counter, int n_sm, cudaStream_t s)
{
    switch (F) {
#define SCIVR_B(FF) case FF: return launch_group_batch_mixed_F<FF>(warps, items, work, n_work, counter, n_sm, s);
    SCIVR_B(1) SCIVR_B(2) SCIVR_B(3) SCIVR_B(4) SCIVR_B(5) SCIVR_B(6) SCIVR_B(7) SCIVR_B(8) SCIVR_B(9)
    SCIVR_B(10) SCIVR_B(11) SCIVR_B(12) SCIVR_B(13) SCIVR_B(14) SCIVR_B(15) SCIVR_B(16)
    SCIVR_B(17) SCIVR_B(18) SCIVR_B(19) SCIVR_B(20) SCIVR_B(21) SCIVR_B(22) SCIVR_B(23) SCIVR_B(24)
#undef SCIVR_B
    default: return cudaErrorInvalidValue;
    }
}

namespace {

constexpr int kMaxThreadF = 9;   // thread-per-trajectory FP64 kernel
constexpr int kMaxGroupF = 9;    // FP64 lane-group kernel
constexpr int kMaxMixedF = 24;   // mixed lane-group kernel (one trajectory per warp above F = 9, two columns per lane above F = 16)

// Schedule choice when the caller leaves it to the library: the lane-group
// kernel keeps every SM busy with few trajectories (it launches G lanes per
// trajectory); the thread kernel wins in FP64 once there are enough
// trajectories to fill the GPU with one warp per SM sub-partition.  The FP64
// crossover was measured on GB300 (400 steps of the F = 3, 6, 9 workloads): the
// thread kernel's time is flat up to ~16k trajectories while the lane-group
// time grows linearly, and they meet near 6k (F <= 3), 8.5k (F = 4..6) and 5k
// (F >= 7) trajectories.
int choose(int F, int precision, int64_t n_traj)
{
    if (precision == SCIVR_MIXED) return SCIVR_KERNEL_GROUP;
    if (F > kMaxGroupF) return SCIVR_KERNEL_THREAD;
    const int64_t crossover = F <= 3 ? 6144 : F <= 6 ? 8192 : 5120;
    return n_traj >= crossover ? SCIVR_KERNEL_THREAD : SCIVR_KERNEL_GROUP;
}

}  // namespace

bool propagate_supported(int F, int precision, int kernel)
{
    if (F < 1) return false;
    if (precision == SCIVR_MIXED) return kernel != SCIVR_KERNEL_THREAD && F <= kMaxMixedF;
    if (precision != SCIVR_FP64) return false;
    if (kernel == SCIVR_KERNEL_THREAD) return F <= kMaxThreadF;
    if (kernel == SCIVR_KERNEL_GROUP) return F <= kMaxGroupF;
    return F <= kMaxThreadF;
}

#define SCIVR_CASES(M, X) \
    case 1: return M<1>(X, s); case 2: return M<2>(X, s); case 3: return M<3>(X, s); \
    case 4: return M<4>(X, s); case 5: return M<5>(X, s); case 6: return M<6>(X, s); \
    case 7: return M<7>(X, s); case 8: return M<8>(X, s);

cudaError_t launch_propagate(const PropLaunch &L, cudaStream_t s, int *n_launch)
{
    *n_launch = 1;
    const int kern = L.args.kernel == SCIVR_KERNEL_AUTO ? choose(L.args.F, L.args.precision, L.n_traj)
                                                          : L.args.kernel;
    if (L.args.precision == SCIVR_MIXED) {
        switch (L.args.F) {
            SCIVR_CASES(launch_group_mixed, L)
            case 9: return launch_group_mixed<9>(L, s);
            case 10: return launch_group_mixed<10>(L, s);
            case 11: return launch_group_mixed<11>(L, s);
            case 12: return launch_group_mixed<12>(L, s);
            case 13: return launch_group_mixed<13>(L, s);
            case 14: return launch_group_mixed<14>(L, s);
            case 15: return launch_group_mixed<15>(L, s);
            case 16: return launch_group_mixed<16>(L, s);
            case 17: return launch_group_mixed<17>(L, s);
            case 18: return launch_group_mixed<18>(L, s);
            case 19: return launch_group_mixed<19>(L, s);
            case 20: return launch_group_mixed<20>(L, s);
            case 21: return launch_group_mixed<21>(L, s);
            case 22: return launch_group_mixed<22>(L, s);
            case 23: return launch_group_mixed<23>(L, s);
            case 24: return launch_group_mixed<24>(L, s);
            default: break;
        }
    } else if (kern == SCIVR_KERNEL_GROUP) {
        switch (L.args.F) { SCIVR_CASES(launch_group_fp64, L) case 9: return launch_group_fp64<9>(L, s); default: break; }
    } else {
        switch (L.args.F) {
            SCIVR_CASES(launch_tpt_fp64, L)
            case 9: return launch_tpt_fp64<9>(L, s);
            default: break;
        }
    }
    *n_launch = 0;
    return cudaErrorInvalidValue;
}

}  // namespace scivr
