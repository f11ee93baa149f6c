// Husimi sampling of initial conditions (Sec. III.A of arXiv:1312.4698).
//
// The paper samples (p0, q0) from the Husimi distribution of the reference
// coherent state chi and weights each trajectory accordingly.  Here:
//   q0_i = q_eq_i + z_i / sqrt(gamma_i),   p0_i = p_eq_i + z_{F+i} sqrt(gamma_i),
//   w    = 1 / |<p0 q0|chi>|^2 = exp( sum_i gamma_i dq_i^2 / 2 + dp_i^2 / (2 gamma_i) ).
// Normals come from Philox4x32-10 (Salmon et al., SC'11), counter-based so
// that every trajectory draws independently of launch shape, and Box-Muller.
#include "scivr_internal.cuh"

namespace scivr {
namespace {

struct SampleArgs {
    int F;
    double gamma[SCIVR_MAX_F], p_eq[SCIVR_MAX_F], q_eq[SCIVR_MAX_F];
};

__device__ __forceinline__ void philox_round(uint32_t &x0, uint32_t &x1, uint32_t &x2,
                                             uint32_t &x3, uint32_t k0, uint32_t k1)
{
    const uint32_t lo0 = 0xD2511F53u * x0, hi0 = __umulhi(0xD2511F53u, x0);
    const uint32_t lo1 = 0xCD9E8D57u * x2, hi1 = __umulhi(0xCD9E8D57u, x2);
    const uint32_t y0 = hi1 ^ x1 ^ k0, y2 = hi0 ^ x3 ^ k1;
    x0 = y0; x1 = lo1; x2 = y2; x3 = lo0;
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
    uint32_t x0 = c.x, x1 = c.y, x2 = c.z, x3 = c.w;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        philox_round(x0, x1, x2, x3, k0, k1);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return make_uint4(x0, x1, x2, x3);
}

__global__ void k_sample(const SampleArgs A, int64_t n_traj, uint64_t seed, double *__restrict__ p0,
                         double *__restrict__ q0, double *__restrict__ w)
{
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n_traj) return;
    const int F = A.F;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    double lw = 0.0;
    double z[4];
    for (int d = 0; d < 2 * F; ++d) {
        if ((d & 3) == 0) {
            const uint4 u = philox4x32_10(
                make_uint4((uint32_t)j, (uint32_t)((uint64_t)j >> 32), (uint32_t)(d >> 2), 0u), k0, k1);
            const uint32_t uu[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
            for (int pr = 0; pr < 2; ++pr) {
                const double u1 = ((double)uu[2 * pr] + 0.5) * 0x1p-32;
                const double u2 = ((double)uu[2 * pr + 1] + 0.5) * 0x1p-32;
                const double r = sqrt(-2.0 * log(u1));
                double sn, cs;
                sincos(kTwoPi * u2, &sn, &cs);
                z[2 * pr] = r * cs;
                z[2 * pr + 1] = r * sn;
            }
        }
        const double zd = z[d & 3];
        if (d < F) {
            const int i = d;
            const double dq = zd / sqrt(A.gamma[i]);
            q0[i * n_traj + j] = A.q_eq[i] + dq;
            lw = fma(0.5 * A.gamma[i] * dq, dq, lw);
        } else {
            const int i = d - F;
            const double dp = zd * sqrt(A.gamma[i]);
            p0[i * n_traj + j] = A.p_eq[i] + dp;
            lw = fma(dp, dp / (2.0 * A.gamma[i]), lw);
        }
    }
    w[j] = exp(lw);
}

}  // namespace

cudaError_t launch_sample(int F, const double *gamma, const double *p_eq, const double *q_eq,
                          int64_t n_traj, uint64_t seed, double *p0, double *q0, double *w,
                          cudaStream_t s, int *n_launch)
{
    SampleArgs A{};
    A.F = F;
    for (int i = 0; i < F; ++i) {
        A.gamma[i] = gamma[i];
        A.p_eq[i] = p_eq[i];
        A.q_eq[i] = q_eq[i];
    }
    const int threads = 256;
    const int64_t blocks = (n_traj + threads - 1) / threads;
    k_sample<<<(unsigned)blocks, threads, 0, s>>>(A, n_traj, seed, p0, q0, w);
    *n_launch = 1;
    return cudaGetLastError();
}

}  // namespace scivr
