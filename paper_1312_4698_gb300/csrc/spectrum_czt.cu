// Time -> energy Fourier step of the time-averaged spectrum (Eq. I(E)_discreto of
// arXiv:1312.4698) in FP64 by the chirp-z transform: the same sums
//   X_j(E_k) = sum_{c=0}^{K-1} a_j(c) exp(i E_k c dt),  E_k = E_min + k dE,
// evaluated through Bluestein's identity k c = (k^2 + c^2 - (k - c)^2) / 2:
//   X_j(E_k) = exp(i w k^2/2) sum_c u_c v_{k-c},  w = dE dt,
//   u_c = a_j(c) exp(i (E_min c dt + w c^2/2)),  v_m = exp(-i w m^2/2),
// a linear convolution computed by FFTs of length L >= K + n_E - 1.  The output chirp
// has modulus one, so |X_j(E_k)|^2 = |(u * v)_k|^2.  Per trajectory this costs about
// 10 L log2 L FP64 flops instead of the direct sum's 8 K n_E: on GB300, whose FP64
// rate is 1/64 of FP32, the transform runs in O(L log L) on the FP64 pipe and keeps
// FP64 rounding (about log2(L) * 2^-53 of the largest |X|).
//
// Layout: one CTA per SM loops over trajectories (one at a time, the whole length-L
// complex vector in shared memory); an in-place radix-2 FFT with decimation in time
// (bit-reversed in, natural out) transforms u, the product with V = FFT(v) is
// conjugated (the inverse transform is conj(FFT(conj(.))) / L), and a decimation-in-
// frequency FFT (natural in, bit-reversed out) finishes.  Energies beyond L - K + 1
// are taken in blocks, each with its own input chirp.  Each CTA keeps its weighted
// |X|^2 sums in shared memory; a fixed-order reduction over CTAs follows
// (deterministic).
#include "scivr_internal.cuh"

namespace scivr {
namespace {

constexpr int kLog2L = 13, kL = 1 << kLog2L;    // 8192 points: 128 KB of FP64 complex
constexpr int kThreads = 512;

__device__ __forceinline__ double2 cmul(double2 x, double2 y)
{
    return make_double2(fma(x.x, y.x, -x.y * y.y), fma(x.x, y.y, x.y * y.x));
}

__device__ __forceinline__ unsigned brev(unsigned i) { return __brev(i) >> (32 - kLog2L); }

// tw[k] = exp(-2 pi i k / L), k < L/2.
__global__ void k_czt_twiddles(double2 *__restrict__ tw)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= kL / 2) return;
    double s, c;
    sincospi(-2.0 * k / kL, &s, &c);
    tw[k] = make_double2(c, s);
}

// Input chirps of the energy blocks: chirp[b][c] = exp(i (E_b c dt + w c^2/2)), c < K.
__global__ void k_czt_chirps(double2 *__restrict__ chirp, int K, int n_blk, int nb, double E_min, double dE,
                             double dt)
{
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n_blk * K) return;
    const int b = (int)(idx / K), c = (int)(idx % K);
    const double Eb = E_min + (double)b * nb * dE;
    const double w = dE * dt;
    // phase modulo 2 pi in FP64 (c^2 is exact); sincos keeps full accuracy for these arguments
    const double ph = Eb * (c * dt) + 0.5 * w * ((double)c * (double)c);
    double s, co;
    sincos(ph, &s, &co);
    chirp[idx] = make_double2(co, s);
}

// In-place radix-2 transform of x (forward, exp(-2 pi i ...)): decimation in time takes
// bit-reversed input to natural output; decimation in frequency natural to bit-reversed.
__device__ void fft_dit(double2 *x, const double2 *__restrict__ tw)
{
    for (int s = 1; s <= kLog2L; ++s) {
        const int half = 1 << (s - 1), step = kL >> s;
        for (int t = threadIdx.x; t < kL / 2; t += blockDim.x) {
            const int pos = t & (half - 1), i = ((t >> (s - 1)) << s) + pos, j = i + half;
            const double2 b = cmul(x[j], __ldg(tw + pos * step));
            const double2 a = x[i];
            x[i] = make_double2(a.x + b.x, a.y + b.y);
            x[j] = make_double2(a.x - b.x, a.y - b.y);
        }
        __syncthreads();
    }
}

__device__ void fft_dif(double2 *x, const double2 *__restrict__ tw)
{
    for (int s = kLog2L; s >= 1; --s) {
        const int half = 1 << (s - 1), step = kL >> s;
        for (int t = threadIdx.x; t < kL / 2; t += blockDim.x) {
            const int pos = t & (half - 1), i = ((t >> (s - 1)) << s) + pos, j = i + half;
            const double2 a = x[i], b = x[j];
            x[i] = make_double2(a.x + b.x, a.y + b.y);
            x[j] = cmul(make_double2(a.x - b.x, a.y - b.y), __ldg(tw + pos * step));
        }
        __syncthreads();
    }
}

// V = FFT(v), v at index m mod L for m in [-(K-1), nb - 1], v_m = exp(-i w m^2/2).
__global__ void __launch_bounds__(kThreads) k_czt_kernel_fft(const double2 *__restrict__ tw, int K, int nb, double w,
                                                             double2 *__restrict__ V)
{
    extern __shared__ __align__(16) double2 xs[];
    for (int idx = threadIdx.x; idx < kL; idx += blockDim.x) {
        const int n = (int)brev((unsigned)idx);
        const int m = n < nb ? n : n - kL;
        double2 v = make_double2(0.0, 0.0);
        if (m < nb && m > -K) {
            double s, c;
            sincos(-0.5 * w * ((double)m * (double)m), &s, &c);
            v = make_double2(c, s);
        }
        xs[idx] = v;
    }
    __syncthreads();
    fft_dit(xs, tw);
    for (int k = threadIdx.x; k < kL; k += blockDim.x) V[k] = xs[k];
}

// Weighted |X|^2 of the CTA's good trajectories for every energy block; per-CTA sums.
__global__ void __launch_bounds__(kThreads) k_czt(const AmpRef amp, int64_t amp_ld,
                                                  const double *__restrict__ w, const uint8_t *__restrict__ good,
                                                  int64_t n_traj, int K, int n_E, int n_blk, int nb,
                                                  const double2 *__restrict__ chirp, const double2 *__restrict__ V,
                                                  const double2 *__restrict__ tw, double *__restrict__ part)
{
    extern __shared__ __align__(16) double2 xs[];
    double *Ip = reinterpret_cast<double *>(xs + kL);   // [n_E]
    for (int k = threadIdx.x; k < n_E; k += blockDim.x) Ip[k] = 0.0;
    const double inv_L2 = 1.0 / ((double)kL * (double)kL);
    for (int64_t j = blockIdx.x; j < n_traj; j += gridDim.x) {
        if (!good[j]) continue;                       // uniform over the CTA
        const AmpRef a = amp.offset(j * amp_ld);
        const double wj = w[j] * inv_L2;
        for (int b = 0; b < n_blk; ++b) {
            const double2 *ch = chirp + (int64_t)b * K;
            for (int idx = threadIdx.x; idx < kL; idx += blockDim.x) {
                const int c = (int)brev((unsigned)idx);
                xs[idx] = c < K ? cmul(a[c], __ldg(ch + c)) : make_double2(0.0, 0.0);
            }
            __syncthreads();
            fft_dit(xs, tw);
            for (int k = threadIdx.x; k < kL; k += blockDim.x) {
                const double2 p = cmul(xs[k], __ldg(V + k));
                xs[k] = make_double2(p.x, -p.y);
            }
            __syncthreads();
            fft_dif(xs, tw);
            const int k0 = b * nb, nk = min(nb, n_E - k0);
            for (int k = threadIdx.x; k < nk; k += blockDim.x) {
                const double2 y = xs[brev((unsigned)k)];
                Ip[k0 + k] = fma(wj, fma(y.x, y.x, y.y * y.y), Ip[k0 + k]);
            }
            __syncthreads();
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n_E; k += blockDim.x) part[(int64_t)blockIdx.x * n_E + k] = Ip[k];
}

__global__ void k_czt_count_good(const uint8_t *__restrict__ good, int64_t n, int64_t *__restrict__ out,
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

__global__ void k_czt_reduce(const double *__restrict__ part, int n_cta, int n_E, const int64_t *__restrict__ ng,
                             double scale, double *__restrict__ I_out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_E) return;
    double s = 0.0;
    for (int m = 0; m < n_cta; ++m) s += part[(int64_t)m * n_E + k];
    I_out[k] = ng[0] > 0 ? s * (scale / (double)ng[0]) : 0.0;
}

inline size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

struct CztLayout {
    int K, nb, n_blk, n_cta;
    size_t off_ng, off_tw, off_V, off_chirp, off_part, total;
};

CztLayout czt_layout(int n_steps, int n_E, int n_sm)
{
    CztLayout L{};
    L.K = n_steps + 1;
    L.nb = kL - L.K + 1;
    L.n_blk = L.nb > 0 ? (n_E + L.nb - 1) / L.nb : 0;
    L.n_cta = n_sm;
    L.off_ng = 0;
    L.off_tw = a256(sizeof(int64_t));
    L.off_V = L.off_tw + a256(sizeof(double2) * kL / 2);
    L.off_chirp = L.off_V + a256(sizeof(double2) * kL);
    L.off_part = L.off_chirp + a256(sizeof(double2) * (size_t)L.n_blk * L.K);
    L.total = L.off_part + a256(sizeof(double) * (size_t)L.n_cta * n_E);
    return L;
}

int sm_count()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

}  // namespace

// Largest K = n_steps + 1 the chirp-z mode takes: an energy block must hold at least
// 1024 energies (L - K + 1 >= 1024).
int spectrum_czt_max_samples() { return kL - 1023; }

size_t spectrum_czt_scratch_bytes(int64_t n_traj, int n_steps, int n_E)
{
    (void)n_traj;
    return czt_layout(n_steps, n_E, sm_count()).total;
}

cudaError_t launch_spectrum_czt(AmpRef amp, int64_t amp_ld, const double *w, const uint8_t *good,
                                int64_t n_traj, int n_steps, double dt, double E_min, double E_max, int n_E,
                                double *I_out, int64_t *n_good_out, void *scratch, cudaStream_t s, int *n_launch)
{
    *n_launch = 0;
    const CztLayout L = czt_layout(n_steps, n_E, sm_count());
    if (L.K > spectrum_czt_max_samples()) return cudaErrorInvalidValue;
    char *base = static_cast<char *>(scratch);
    int64_t *ng = reinterpret_cast<int64_t *>(base + L.off_ng);
    double2 *tw = reinterpret_cast<double2 *>(base + L.off_tw);
    double2 *V = reinterpret_cast<double2 *>(base + L.off_V);
    double2 *chirp = reinterpret_cast<double2 *>(base + L.off_chirp);
    double *part = reinterpret_cast<double *>(base + L.off_part);
    const double dE = (E_max - E_min) / (n_E - 1);
    const double scale = dt * dt / (kTwoPi * (n_steps * dt));
    const size_t smem_fft = sizeof(double2) * kL;
    const size_t smem = smem_fft + sizeof(double) * (size_t)n_E;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_czt_kernel_fft, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_fft)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_czt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) return e;
    k_czt_count_good<<<1, 1024, 0, s>>>(good, n_traj, ng, n_good_out);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_czt_twiddles<<<kL / 2 / 256, 256, 0, s>>>(tw);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int64_t nch = (int64_t)L.n_blk * L.K;
    k_czt_chirps<<<(unsigned)((nch + 255) / 256), 256, 0, s>>>(chirp, L.K, L.n_blk, L.nb, E_min, dE, dt);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_czt_kernel_fft<<<1, kThreads, smem_fft, s>>>(tw, L.K, L.nb, dE * dt, V);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_czt<<<L.n_cta, kThreads, smem, s>>>(amp, amp_ld, w, good, n_traj, L.K, n_E, L.n_blk, L.nb, chirp, V, tw, part);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_czt_reduce<<<(n_E + 255) / 256, 256, 0, s>>>(part, L.n_cta, n_E, ng, scale, I_out);
    *n_launch = 6;
    return cudaGetLastError();
}

}  // namespace scivr
