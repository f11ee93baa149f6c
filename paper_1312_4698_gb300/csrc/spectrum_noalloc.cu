// scivr_spectrum_noalloc: the FP64 spectrum (same result as scivr_spectrum)
// for callers that cannot allocate device memory.  Its scratch -- the good
// count and per-slice column partial sums -- lives in one file-scope device
// array, so the call itself allocates nothing.  The twiddle factors
// exp(i E_k c dt) are generated inside the contraction kernel (a per-CTA
// table of exp(i E_k kk dt), kk < 16, times exp(i E_k c0 dt) per 16-step
// block) instead of being stored in a scratch matrix.
#include <cmath>
#include <cstdio>
#include <mutex>
#include <string>

#include "scivr_internal.cuh"

namespace scivr {
namespace {

constexpr int kScratchDoubles = 1 << 19;        // 4 MiB, held by every device that loads the library
constexpr int kHeaderDoubles = 32;               // slot 0: good count (int64); padded to 256 bytes
constexpr int kMaxSlices = 16;
constexpr int kMaxDevices = 64;
constexpr int NB = 64, NK = 16, NTX = 16, NTY = 16;

static __device__ __align__(256) double g_spectrum_scratch[kScratchDoubles];

std::mutex g_setup_mu;
double *g_scratch_addr[kMaxDevices] = {};

__global__ void k_na_count_good(const uint8_t *__restrict__ good, int64_t n, double *__restrict__ scratch,
                                int64_t *__restrict__ n_good_out)
{
    __shared__ long long red[1024];
    long long acc = 0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc += good[i] ? 1 : 0;
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        reinterpret_cast<long long *>(scratch)[0] = red[0];   // written, never accumulated
        if (n_good_out) n_good_out[0] = red[0];
    }
}

// grid.x: energy strips of NB columns; grid.y: row slices.  Each CTA walks the
// row tiles m = slice, slice + n_slices, ... and keeps its column sums on chip.
__global__ void __launch_bounds__(256) k_na_ft(const AmpRef amp, int64_t amp_ld,
                                               const double *__restrict__ w, const uint8_t *__restrict__ good,
                                               int64_t n_traj, int K, int n_E, double E_min, double dE,
                                               double dt, int n_slices, double *__restrict__ part)
{
    __shared__ double2 As[NK][NB];
    __shared__ double2 Bs[NK][NB];
    __shared__ double2 Pw[NK][NB];      // exp(i E_col kk dt)
    __shared__ double2 Base[NB];        // exp(i E_col c0 dt)
    __shared__ double red[NTY][NB];
    const int tx = threadIdx.x % NTX, ty = threadIdx.x / NTX;
    const int col0 = blockIdx.x * NB;
    const int64_t n_mt = (n_traj + NB - 1) / NB;

    for (int li = threadIdx.x; li < NK * NB; li += 256) {
        const int kk = li / NB, cc = li % NB;
        const double E = E_min + (col0 + cc) * dE;
        double sn, cs;
        sincos(E * (kk * dt), &sn, &cs);
        Pw[kk][cc] = make_double2(cs, sn);
    }
    double colacc[4] = {0.0, 0.0, 0.0, 0.0};

    for (int64_t mt = blockIdx.y; mt < n_mt; mt += n_slices) {
        const int64_t row0 = mt * NB;
        double2 acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) acc[i][jj] = make_double2(0.0, 0.0);
        for (int c0 = 0; c0 < K; c0 += NK) {
            if (threadIdx.x < NB) {
                const double E = E_min + (col0 + threadIdx.x) * dE;
                double sn, cs;
                sincos(E * (c0 * dt), &sn, &cs);
                Base[threadIdx.x] = make_double2(cs, sn);
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int li = threadIdx.x + r * 256;
                const int rr = li / NK, kk = li % NK;
                const int64_t row = row0 + rr;
                const int c = c0 + kk;
                double2 v = make_double2(0.0, 0.0);
                if (row < n_traj && c < K) v = amp[row * amp_ld + c];
                As[kk][rr] = v;
            }
            __syncthreads();
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int li = threadIdx.x + r * 256;
                const int kk = li / NB, cc = li % NB;
                const double2 b = Base[cc], p = Pw[kk][cc];
                double2 v = make_double2(fma(b.x, p.x, -b.y * p.y), fma(b.x, p.y, b.y * p.x));
                if (c0 + kk >= K || col0 + cc >= n_E) v = make_double2(0.0, 0.0);
                Bs[kk][cc] = v;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < NK; ++kk) {
                double2 a[4], b[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + NTY * i];
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) b[jj] = Bs[kk][tx + NTX * jj];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) {
                        acc[i][jj].x = fma(a[i].x, b[jj].x, acc[i][jj].x);
                        acc[i][jj].x = fma(-a[i].y, b[jj].y, acc[i][jj].x);
                        acc[i][jj].y = fma(a[i].x, b[jj].y, acc[i][jj].y);
                        acc[i][jj].y = fma(a[i].y, b[jj].x, acc[i][jj].y);
                    }
            }
            __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int64_t row = row0 + ty + NTY * i;
            const bool ok = row < n_traj && good[row];
            const double wr = ok ? w[row] : 0.0;
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
                const double m2 = fma(acc[i][jj].x, acc[i][jj].x, acc[i][jj].y * acc[i][jj].y);
                colacc[jj] += ok ? wr * m2 : 0.0;
            }
        }
    }
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) red[ty][tx + NTX * jj] = colacc[jj];
    __syncthreads();
    if (threadIdx.x < NB) {
        double s = 0.0;
#pragma unroll
        for (int t = 0; t < NTY; ++t) s += red[t][threadIdx.x];
        const int col = col0 + threadIdx.x;
        if (col < n_E) part[(int64_t)blockIdx.y * n_E + col] = s;   // every (slice, col) is written
    }
}

__global__ void k_na_reduce(const double *__restrict__ scratch, const double *__restrict__ part,
                            int n_slices, int n_E, double scale, double *__restrict__ I_out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_E) return;
    double s = 0.0;
    for (int m = 0; m < n_slices; ++m) s += part[(int64_t)m * n_E + k];
    const long long ng = reinterpret_cast<const long long *>(scratch)[0];
    I_out[k] = ng > 0 ? s * (scale / (double)ng) : 0.0;
}

// Device address of this device's copy of g_spectrum_scratch, looked up with
// that device current.  Outside stream capture the address is looked up on
// every call (a device reset or a new primary context reloads the module at
// another address, so a remembered one could be stale); during capture the
// address remembered from the last call on this device is used.
cudaError_t scratch_address(cudaStream_t s, double **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (cap == cudaStreamCaptureStatusNone || !g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_spectrum_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

int spectrum_noalloc_max_energies() { return kScratchDoubles - kHeaderDoubles; }

cudaError_t launch_spectrum_noalloc(AmpRef amp, int64_t amp_ld, const double *w,
                                    const uint8_t *good, int64_t n_traj, int n_steps, double dt,
                                    double E_min, double E_max, int n_E, double *I_out,
                                    int64_t *n_good_out, cudaStream_t s, int *n_launch)
{
    *n_launch = 0;
    double *scratch = nullptr;
    cudaError_t e = scratch_address(s, &scratch);
    if (e != cudaSuccess) return e;
    const int K = n_steps + 1;
    const int64_t n_mt = (n_traj + NB - 1) / NB;
    int n_slices = (int)((kScratchDoubles - kHeaderDoubles) / n_E);
    if (n_slices > kMaxSlices) n_slices = kMaxSlices;
    if (n_slices > n_mt) n_slices = (int)n_mt;
    if (n_slices < 1) return cudaErrorInvalidValue;
    double *part = scratch + kHeaderDoubles;
    const double dE = (E_max - E_min) / (n_E - 1);
    const double scale = dt * dt / (kTwoPi * (n_steps * dt));
    k_na_count_good<<<1, 1024, 0, s>>>(good, n_traj, scratch, n_good_out);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    dim3 grid((unsigned)((n_E + NB - 1) / NB), (unsigned)n_slices);
    k_na_ft<<<grid, 256, 0, s>>>(amp, amp_ld, w, good, n_traj, K, n_E, E_min, dE, dt, n_slices, part);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_na_reduce<<<(n_E + 255) / 256, 256, 0, s>>>(scratch, part, n_slices, n_E, scale, I_out);
    *n_launch = 3;
    return cudaGetLastError();
}

}  // namespace scivr
