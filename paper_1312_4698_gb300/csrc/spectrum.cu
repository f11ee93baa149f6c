// Time -> energy Fourier step of the time-averaged spectrum, Eq. I(E)_discreto
// of arXiv:1312.4698, as a dense complex contraction with a fused epilogue:
//
//   X[j][k] = sum_c amp[j][c] tw[c][k],      tw[c][k] = exp(i E_k c dt)
//   part[m][k] = sum_{j in row tile m, good} w_j |X[j][k]|^2
//   I[k] = dt^2 / (2 pi T n_good) sum_m part[m][k]     (fixed order, deterministic)
//
// X is never written to memory.  The paper's design writes a private
// n_traj x k buffer per trajectory and reduces its columns in a second
// kernel (Sec. III.B); here the per-column weighted reduction happens in the
// GEMM epilogue and only ceil(n_traj / 64) partial rows reach global memory.
#include "scivr_internal.cuh"

namespace scivr {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, TX = 16, TY = 16;   // 256 threads, 4x4 outputs each

__global__ void k_count_good(const uint8_t *__restrict__ good, int64_t n, int64_t *__restrict__ out,
                             int64_t *__restrict__ out2)
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
        out[0] = red[0];
        if (out2) out2[0] = red[0];
    }
}

__global__ void k_twiddles(double2 *__restrict__ tw, int K, int n_E, double E_min, double dE,
                           double dt)
{
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= (int64_t)K * n_E) return;
    const int c = (int)(idx / n_E), k = (int)(idx % n_E);
    const double E = E_min + k * dE;
    double sn, cs;
    sincos(E * (c * dt), &sn, &cs);
    tw[idx] = make_double2(cs, sn);
}

__global__ void __launch_bounds__(256) k_ft_fp64(const AmpRef amp, int64_t amp_ld,
                                                 const double2 *__restrict__ tw, const double *__restrict__ w,
                                                 const uint8_t *__restrict__ good, int64_t n_traj, int K,
                                                 int n_E, double *__restrict__ part)
{
    __shared__ double2 As[BK][BM];
    __shared__ double2 Bs[BK][BN];
    __shared__ double red[TY][BN];
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int64_t row0 = (int64_t)blockIdx.x * BM;
    const int col0 = blockIdx.y * BN;

    double2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) acc[i][jj] = make_double2(0.0, 0.0);

    for (int c0 = 0; c0 < K; c0 += BK) {
        // amp tile: 64 rows x 16 steps, stored transposed
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int li = threadIdx.x + r * 256;
            const int rr = li / BK, kk = li % BK;
            const int64_t row = row0 + rr;
            const int c = c0 + kk;
            double2 v = make_double2(0.0, 0.0);
            if (row < n_traj && c < K) v = amp[row * amp_ld + c];
            As[kk][rr] = v;
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int li = threadIdx.x + r * 256;
            const int kk = li / BN, cc = li % BN;
            const int c = c0 + kk, col = col0 + cc;
            double2 v = make_double2(0.0, 0.0);
            if (c < K && col < n_E) v = tw[(int64_t)c * n_E + col];
            Bs[kk][cc] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            double2 a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + TY * i];
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) b[jj] = Bs[kk][tx + TX * jj];
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
    // epilogue: weighted |X|^2 summed over the tile's good rows
    double colsum[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t row = row0 + ty + TY * i;
        const bool ok = row < n_traj && good[row];
        const double wr = ok ? w[row] : 0.0;
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
            const double m2 = fma(acc[i][jj].x, acc[i][jj].x, acc[i][jj].y * acc[i][jj].y);
            colsum[jj] += ok ? wr * m2 : 0.0;
        }
    }
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) red[ty][tx + TX * jj] = colsum[jj];
    __syncthreads();
    if (threadIdx.x < BN) {
        double s = 0.0;
#pragma unroll
        for (int t = 0; t < TY; ++t) s += red[t][threadIdx.x];
        const int col = col0 + threadIdx.x;
        if (col < n_E) part[(int64_t)blockIdx.x * n_E + col] = s;
    }
}

__global__ void k_reduce_parts(const double *__restrict__ part, int n_mt, int n_E,
                               const int64_t *__restrict__ n_good, double scale,
                               double *__restrict__ I_out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_E) return;
    double s = 0.0;
    for (int m = 0; m < n_mt; ++m) s += part[(int64_t)m * n_E + k];
    const int64_t ng = n_good[0];
    I_out[k] = ng > 0 ? s * (scale / (double)ng) : 0.0;
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

size_t spectrum_fp64_scratch_bytes(int64_t n_traj, int n_steps, int n_E)
{
    const int64_t K = n_steps + 1;
    const int64_t n_mt = (n_traj + BM - 1) / BM;
    return align256(sizeof(int64_t)) + align256(sizeof(double2) * K * n_E) +
           align256(sizeof(double) * n_mt * n_E);
}

cudaError_t launch_spectrum_fp64(AmpRef amp, int64_t amp_ld, const double *w,
                                 const uint8_t *good, int64_t n_traj, int n_steps, double dt,
                                 double E_min, double E_max, int n_E, double *I_out,
                                 int64_t *n_good_out, void *scratch, cudaStream_t s, int *n_launch)
{
    const int K = n_steps + 1;
    const int64_t n_mt = (n_traj + BM - 1) / BM;
    char *base = static_cast<char *>(scratch);
    int64_t *ng = reinterpret_cast<int64_t *>(base);
    double2 *tw = reinterpret_cast<double2 *>(base + align256(sizeof(int64_t)));
    double *part = reinterpret_cast<double *>(base + align256(sizeof(int64_t)) +
                                              align256(sizeof(double2) * (size_t)K * n_E));
    const double dE = (E_max - E_min) / (n_E - 1);
    const double T = n_steps * dt;
    const double scale = dt * dt / (kTwoPi * T);
    cudaError_t e;
    k_count_good<<<1, 1024, 0, s>>>(good, n_traj, ng, n_good_out);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int64_t ntw = (int64_t)K * n_E;
    k_twiddles<<<(unsigned)((ntw + 255) / 256), 256, 0, s>>>(tw, K, n_E, E_min, dE, dt);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    dim3 grid((unsigned)n_mt, (unsigned)((n_E + BN - 1) / BN));
    k_ft_fp64<<<grid, 256, 0, s>>>(amp, amp_ld, tw, w, good, n_traj, K, n_E, part);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_reduce_parts<<<(n_E + 255) / 256, 256, 0, s>>>(part, (int)n_mt, n_E, ng, scale, I_out);
    *n_launch = 4;
    return cudaGetLastError();
}

}  // namespace scivr
