// Arithmetic-rate probe: independent fused multiply-add chains on the FP32 or FP64
// pipe, the measured denominators of the propagation kernels' roofline (their work is
// plain FMA arithmetic on those two pipes).  Every SM runs enough warps to cover the
// FMA latency; each thread keeps kChains independent accumulators.
#include "scivr_internal.cuh"

namespace scivr {
namespace {

constexpr int kChains = 16, kThreads = 256, kBlocksPerSm = 8;

static __device__ double g_probe_sink;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_probe(long long iters, T seed)
{
    T acc[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc[c] = seed + (T)(threadIdx.x + c);
    const T a = (T)0.999999, b = (T)1e-7;
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc[c] = fma(acc[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += acc[c];
    if (s == (T)-12345.0) g_probe_sink = (double)s;   // never true; keeps the chains live
}

}  // namespace
}  // namespace scivr

using namespace scivr;

extern "C" int scivr_fma_probe(int32_t precision, int64_t iters, double *flops_per_launch, void *stream)
{
    if (precision != SCIVR_FP64 && precision != SCIVR_MIXED)
        return set_error(SCIVR_EINVAL, "scivr_fma_probe: precision must be SCIVR_FP64 or SCIVR_MIXED (FP32)");
    if (iters < 1 || !flops_per_launch) return set_error(SCIVR_EINVAL, "scivr_fma_probe: iters >= 1 and an output");
    int dev = 0, n_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_error(e, "scivr_fma_probe: device query");
    const unsigned blocks = (unsigned)(n_sm * kBlocksPerSm);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (precision == SCIVR_FP64) k_fma_probe<double><<<blocks, kThreads, 0, s>>>(iters, 1.0);
    else k_fma_probe<float><<<blocks, kThreads, 0, s>>>(iters, 1.0f);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "scivr_fma_probe: launch");
    count_launches(1);
    *flops_per_launch = 2.0 * kChains * (double)iters * blocks * kThreads;
    clear_error();
    return SCIVR_OK;
}
