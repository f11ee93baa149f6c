// Batched analytic potential evaluation (FP64): V, grad V and the Hessian of
// the separable diagonal, the coupling polynomial, or both, at n points -- the
// force-stage evaluation of the propagation (Sec. III.A), one thread per point.
#include "propagate_tpt.cuh"

namespace scivr {
namespace {

template <int F>
__global__ void k_pes_eval(PesDev pes, int64_t n, const double *__restrict__ q, int terms, double *__restrict__ V,
                           double *__restrict__ g, double *__restrict__ H)
{
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    double x[F], h[F][F], gg[F], v;
#pragma unroll
    for (int a = 0; a < F; ++a) x[a] = q[j * F + a];
    PesDev p = pes;
    if (terms == SCIVR_TERMS_DIAG) p.has3 = p.has4 = 0;
    tpt::pes_fp64<F>(p, x, h, gg, v);
    if (terms == SCIVR_TERMS_COUPLING) {
        // coupling = full - diagonal (the diagonal part is evaluated identically in both)
        double hd[F][F], gd[F], vd;
        p.has3 = p.has4 = 0;
        tpt::pes_fp64<F>(p, x, hd, gd, vd);
        v -= vd;
#pragma unroll
        for (int a = 0; a < F; ++a) {
            gg[a] -= gd[a];
#pragma unroll
            for (int b = 0; b < F; ++b) h[a][b] -= hd[a][b];
        }
    }
    V[j] = v;
    if (g)
#pragma unroll
        for (int a = 0; a < F; ++a) g[j * F + a] = gg[a];
    if (H)
#pragma unroll
        for (int a = 0; a < F; ++a)
#pragma unroll
            for (int b = 0; b < F; ++b) H[(j * F + a) * F + b] = h[a][b];
}

}  // namespace

cudaError_t launch_pes_eval(const PesDev &pes, int64_t n, const double *q, int terms, double *V, double *g, double *H,
                            cudaStream_t s)
{
    const unsigned blocks = (unsigned)((n + 127) / 128);
    switch (pes.F) {
#define SCIVR_P(FF) case FF: k_pes_eval<FF><<<blocks, 128, 0, s>>>(pes, n, q, terms, V, g, H); break;
    SCIVR_P(1) SCIVR_P(2) SCIVR_P(3) SCIVR_P(4) SCIVR_P(5) SCIVR_P(6) SCIVR_P(7) SCIVR_P(8) SCIVR_P(9)
#undef SCIVR_P
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace scivr
