// Plain Herman-Kluk SC-IVR spectrum (Eq. I(E)_SCIVR of arXiv:1312.4698) from
// the per-trajectory Herman-Kluk summands that scivr_propagate records with
// SCIVR_AMP_HK: the survival amplitude C(c dt) is their mean over the good
// trajectories (a column sum of the amplitude matrix, HBM-bound: one read of
// 16 n K bytes), then I(E_k) = (dt/pi) Re[C(0)/2 + sum_{c>=1} C(c dt) e^{i E_k c dt}].
// Column sums are deterministic: each block sums a fixed slice of rows for
// 256 consecutive columns (coalesced along the time axis), and the slices'
// partials are added in slice order.
#include <cmath>

#include "scivr_internal.cuh"

namespace scivr {
namespace {

constexpr int kRowsPerSlice = 4096;

__global__ void k_hk_colsum(const double2 *__restrict__ amp, int64_t amp_ld, const uint8_t *__restrict__ good,
                            int64_t n, int K, double2 *__restrict__ part)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.y * kRowsPerSlice;
    const int64_t r1 = r0 + kRowsPerSlice < n ? r0 + kRowsPerSlice : n;
    if (c >= K) return;
    double sr = 0.0, si = 0.0;
    for (int64_t j = r0; j < r1; ++j) {
        if (!good[j]) continue;   // bad rows never reach the sum, whatever they hold
        const double2 a = amp[j * amp_ld + c];
        sr += a.x;
        si += a.y;
    }
    part[(int64_t)blockIdx.y * K + c] = make_double2(sr, si);
}

__global__ void k_hk_count(const uint8_t *__restrict__ good, int64_t n, long long *__restrict__ ng)
{
    __shared__ long long red[256];
    long long cnt = 0;
    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) cnt += good[j] ? 1 : 0;
    red[threadIdx.x] = cnt;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) ng[0] = red[0];
}

__global__ void k_hk_reduce(const double2 *__restrict__ part, int n_slices, int K, const long long *__restrict__ ng,
                            double2 *__restrict__ C)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= K) return;
    double sr = 0.0, si = 0.0;
    for (int s = 0; s < n_slices; ++s) {
        const double2 v = part[(int64_t)s * K + c];
        sr += v.x;
        si += v.y;
    }
    const double inv = ng[0] > 0 ? 1.0 / (double)ng[0] : 0.0;
    C[c] = make_double2(sr * inv, si * inv);
}

// one thread per energy; the phase E_k c dt is formed in FP64 for every c
__global__ void k_hk_ft(const double2 *__restrict__ C, int K, double dt, double E_min, double dE, int n_E,
                        double *__restrict__ I_out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_E) return;
    const double E = E_min + k * dE;
    double acc = 0.5 * C[0].x;
    for (int c = 1; c < K; ++c) {
        double sn, cs;
        sincos(E * (c * dt), &sn, &cs);
        const double2 v = C[c];
        acc = fma(v.x, cs, fma(-v.y, sn, acc));
    }
    I_out[k] = dt / 3.141592653589793238462643383280 * acc;
}

}  // namespace

size_t spectrum_hk_scratch_bytes(int64_t n_traj, int n_steps)
{
    const int64_t slices = (n_traj + kRowsPerSlice - 1) / kRowsPerSlice;
    const int64_t K = n_steps + 1;
    return (size_t)(slices * K + K) * sizeof(double2) + 256;
}

cudaError_t launch_spectrum_hk(const double2 *amp, int64_t amp_ld, const uint8_t *good, int64_t n_traj, int n_steps,
                               double dt, double E_min, double E_max, int n_E, double *I_out, double2 *C_out,
                               int64_t *n_good_out, void *scratch, cudaStream_t s, int *n_launch)
{
    const int K = n_steps + 1;
    const int slices = (int)((n_traj + kRowsPerSlice - 1) / kRowsPerSlice);
    char *b = static_cast<char *>(scratch);
    double2 *part = reinterpret_cast<double2 *>(b);
    double2 *C = C_out ? C_out : reinterpret_cast<double2 *>(b + (size_t)slices * K * sizeof(double2));
    long long *ng = reinterpret_cast<long long *>(b + (size_t)(slices + 1) * K * sizeof(double2));
    if (n_good_out) ng = reinterpret_cast<long long *>(n_good_out);
    k_hk_count<<<1, 256, 0, s>>>(good, n_traj, ng);
    k_hk_colsum<<<dim3((K + 255) / 256, slices), 256, 0, s>>>(amp, amp_ld, good, n_traj, K, part);
    k_hk_reduce<<<(K + 255) / 256, 256, 0, s>>>(part, slices, K, ng, C);
    const double dE = n_E > 1 ? (E_max - E_min) / (n_E - 1) : 0.0;
    k_hk_ft<<<(n_E + 127) / 128, 128, 0, s>>>(C, K, dt, E_min, dE, n_E, I_out);
    *n_launch = 4;
    return cudaGetLastError();
}

}  // namespace scivr
