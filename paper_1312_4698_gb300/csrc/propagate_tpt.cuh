#pragma once
// Thread-per-trajectory FP64 propagation kernel (Sec. III.A / III.B of arXiv:1312.4698).
//
// One CUDA thread owns one trajectory ("thread per trajectory").  All of its
// state -- p, q, S, the 2F x 2F monodromy matrix M, the Hessian and the LU
// work arrays -- lives in registers (spilling to L1-cached local memory for
// larger F), indexed only with compile-time constants.  The potential's
// coupling tensors are read with warp-uniform addresses (broadcast loads).
//
// Per step (Yoshida triple jump of exact sub-flows):
//   drift c1, kick d1, drift c2, kick d2, drift c3, kick d3, drift c4
//   drift tau: q += tau p,  S += tau p.p/2,  M_q += tau M_p
//   kick  tau: p -= tau grad V(q),  S -= tau V(q),  M_p -= tau H(q) M_q
// then det M (stability, Sec. II), det A (Herman-Kluk prefactor, Eq.
// prefactor), the continuous phase, and the amplitude of Eq. I(E)_discreto
// for every reference state.
#include <math_constants.h>

#include "cartesian.cuh"
#include "scivr_internal.cuh"

namespace scivr {
namespace tpt {

template <int F>
__device__ __forceinline__ constexpr int pidx(int a, int b)
{
    return a * F - a * (a - 1) / 2 + (b - a);
}

struct cplx {
    double re, im;
};

__device__ __forceinline__ cplx cmul(cplx x, cplx y)
{
    return {fma(x.re, y.re, -x.im * y.im), fma(x.re, y.im, x.im * y.re)};
}

// y - l * x
__device__ __forceinline__ cplx cfnma(cplx l, cplx x, cplx y)
{
    return {fma(-l.re, x.re, fma(l.im, x.im, y.re)), fma(-l.re, x.im, fma(-l.im, x.re, y.im))};
}

// V, grad V and the Hessian at q (FP64).
template <int F>
__device__ __forceinline__ void pes_fp64(const PesDev &pes, const double (&q)[F], double (&H)[F][F],
                                         double (&g)[F], double &V)
{
    if constexpr (F == 3) {
        if (pes.kind == SCIVR_PES_CART3) {   // Cartesian surface through the bond vectors
            double gq[3], Hq[3][3];
            V = cart3_eval_q(*pes.cart, q, gq, Hq);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                g[a] = gq[a];
#pragma unroll
                for (int b = 0; b < 3; ++b) H[a][b] = Hq[a][b];
            }
            return;
        }
    }
    constexpr int P = F * (F + 1) / 2;
    double qq[P];
#pragma unroll
    for (int a = 0; a < F; ++a)
#pragma unroll
        for (int b = a; b < F; ++b) qq[pidx<F>(a, b)] = q[a] * q[b];

    V = 0.0;
#pragma unroll
    for (int a = 0; a < F; ++a) {
        double Va, ga, ha;
        if (pes.diag_kind == SCIVR_DIAG_MORSE) {
            const double Dm = __ldg(pes.D + a), am = __ldg(pes.a + a);
            const double u = exp(-am * q[a]);
            const double omu = 1.0 - u;
            Va = Dm * omu * omu;
            ga = 2.0 * Dm * am * u * omu;
            ha = 2.0 * Dm * am * am * u * (2.0 * u - 1.0);
        } else {
            const double w2 = __ldg(pes.omega + a) * __ldg(pes.omega + a);
            Va = 0.5 * w2 * qq[pidx<F>(a, a)];
            ga = w2 * q[a];
            ha = w2;
        }
        V += Va;
        g[a] = ga;
        H[a][a] = ha;
#pragma unroll
        for (int b = a + 1; b < F; ++b) H[a][b] = 0.0;
    }
    if (!(pes.has3 | pes.has4)) {
#pragma unroll
        for (int a = 0; a < F; ++a)
#pragma unroll
            for (int b = a + 1; b < F; ++b) H[b][a] = 0.0;
        return;
    }
    double Vc = 0.0;
#pragma unroll
    for (int a = 0; a < F; ++a) {
#pragma unroll
        for (int b = a; b < F; ++b) {
            const int e = pidx<F>(a, b);
            double h3 = 0.0, h4 = 0.0;
            if (pes.has3) {
#pragma unroll
                for (int k = 0; k < F; ++k) h3 = fma(__ldg(pes.T3 + k * P + e), q[k], h3);
            }
            if (pes.has4) {
#pragma unroll
                for (int kl = 0; kl < P; ++kl) h4 = fma(__ldg(pes.T4 + kl * P + e), qq[kl], h4);
            }
            const double gc = fma(0.5, h3, h4 * (1.0 / 3.0));
            const double vc = fma(1.0 / 6.0, h3, h4 * (1.0 / 12.0));
            H[a][b] += h3 + h4;
            if (a == b) {
                g[a] = fma(gc, q[a], g[a]);
                Vc = fma(vc, qq[e], Vc);
            } else {
                g[a] = fma(gc, q[b], g[a]);
                g[b] = fma(gc, q[a], g[b]);
                Vc = fma(2.0 * vc, qq[e], Vc);
            }
        }
    }
    V += Vc;
#pragma unroll
    for (int a = 0; a < F; ++a)
#pragma unroll
        for (int b = a + 1; b < F; ++b) H[b][a] = H[a][b];
}

// Magnitude key of a double for pivot searches: the high word of |x|, an integer
// whose order is that of |x| up to its low 32 mantissa bits.  Comparing keys keeps
// the searches off the FP64 pipe (double comparisons execute there on GB300).
__device__ __forceinline__ int mag_key(double x) { return __double2hiint(x) & 0x7fffffff; }

// 1/x in FP64 from the FP32 reciprocal refined by two Newton steps (the error
// squares each step: 2^-23 -> 2^-46 -> below FP64 rounding); FP64 division
// outside the FP32 exponent range.
__device__ __forceinline__ double recip_fp64(double x)
{
    const double ax = fabs(x);
    if (!(ax > 1e-30 && ax < 1e30)) return 1.0 / x;
    double r = (double)__frcp_rn((float)x);
    r = r * fma(-x, r, 2.0);
    r = r * fma(-x, r, 2.0);
    return r;
}

// Determinant by LU with partial pivoting (row swaps as predicated moves).
template <int N>
__device__ __forceinline__ double det_real(double (&W)[N][N])
{
    double det = 1.0;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        int piv = k;
        int best = mag_key(W[k][k]);
#pragma unroll
        for (int i = k + 1; i < N; ++i) {
            const int v = mag_key(W[i][k]);
            if (v > best) { best = v; piv = i; }
        }
#pragma unroll
        for (int i = k + 1; i < N; ++i) {
            if (i == piv) {
#pragma unroll
                for (int c = k; c < N; ++c) {
                    const double t = W[k][c]; W[k][c] = W[i][c]; W[i][c] = t;
                }
            }
        }
        if (piv != k) det = -det;
        const double akk = W[k][k];
        det *= akk;
        const double inv = recip_fp64(akk);
#pragma unroll
        for (int i = k + 1; i < N; ++i) {
            const double l = W[i][k] * inv;
#pragma unroll
            for (int c = k + 1; c < N; ++c) W[i][c] = fma(-l, W[k][c], W[i][c]);
        }
    }
    return det;
}

template <int N>
__device__ __forceinline__ cplx det_complex(cplx (&A)[N][N])
{
    cplx det = {1.0, 0.0};
#pragma unroll
    for (int k = 0; k < N; ++k) {
        // pivot by max(|re|, |im|), within a factor sqrt(2) of |z|
        int piv = k;
        int best = max(mag_key(A[k][k].re), mag_key(A[k][k].im));
#pragma unroll
        for (int i = k + 1; i < N; ++i) {
            const int v = max(mag_key(A[i][k].re), mag_key(A[i][k].im));
            if (v > best) { best = v; piv = i; }
        }
#pragma unroll
        for (int i = k + 1; i < N; ++i) {
            if (i == piv) {
#pragma unroll
                for (int c = k; c < N; ++c) {
                    const cplx t = A[k][c]; A[k][c] = A[i][c]; A[i][c] = t;
                }
            }
        }
        if (piv != k) { det.re = -det.re; det.im = -det.im; }
        const cplx akk = A[k][k];
        det = cmul(det, akk);
        const double n2 = akk.re * akk.re + akk.im * akk.im;
        const double r = recip_fp64(n2);
        const cplx inv = {akk.re * r, -akk.im * r};
#pragma unroll
        for (int i = k + 1; i < N; ++i) {
            const cplx l = cmul(A[i][k], inv);
#pragma unroll
            for (int c = k + 1; c < N; ++c) A[i][c] = cfnma(l, A[k][c], A[i][c]);
        }
    }
    return det;
}

template <int F>
__global__ void __launch_bounds__(64) k_propagate_tpt_fp64(const PropLaunch L)
{
    constexpr int N2 = 2 * F;
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= L.n_traj) return;
    const PropArgs &A = L.args;
    const int64_t n = L.n_traj;

    double p[F], q[F], M[N2][N2];
#pragma unroll
    for (int a = 0; a < F; ++a) {
        p[a] = L.p0[a * n + j];
        q[a] = L.q0[a * n + j];
    }
#pragma unroll
    for (int r = 0; r < N2; ++r)
#pragma unroll
        for (int c = 0; c < N2; ++c) M[r][c] = (r == c) ? 1.0 : 0.0;

    double S = 0.0, theta = 0.0, arg_old = 0.0, detM = 1.0, stab = 0.0;
    cplx detA = {1.0, 0.0};
    bool good = true;
    double H[F][F], g[F], V;

    for (int step = 0; step <= A.n_steps; ++step) {
        if (step > 0) {
#pragma unroll
            for (int sub = 0; sub < 4; ++sub) {
                // drift
                const double tau = A.cdrift[sub] * A.dt;
                double kin = 0.0;
#pragma unroll
                for (int a = 0; a < F; ++a) kin = fma(0.5 * p[a], p[a], kin);
                S = fma(tau, kin, S);
#pragma unroll
                for (int a = 0; a < F; ++a) q[a] = fma(tau, p[a], q[a]);
#pragma unroll
                for (int a = 0; a < F; ++a)
#pragma unroll
                    for (int c = 0; c < N2; ++c) M[F + a][c] = fma(tau, M[a][c], M[F + a][c]);
                if (sub == 3) break;
                // kick
                const double tk = A.dkick[sub] * A.dt;
                pes_fp64<F>(L.pes, q, H, g, V);
                S = fma(-tk, V, S);
#pragma unroll
                for (int a = 0; a < F; ++a) p[a] = fma(-tk, g[a], p[a]);
#pragma unroll
                for (int c = 0; c < N2; ++c) {
#pragma unroll
                    for (int a = 0; a < F; ++a) {
                        double hm = 0.0;
#pragma unroll
                        for (int b = 0; b < F; ++b) hm = fma(H[a][b], M[F + b][c], hm);
                        M[a][c] = fma(-tk, hm, M[a][c]);
                    }
                }
            }
            // stability monitor |det(M^T M) - 1| = |det(M)^2 - 1|
            {
                double W[N2][N2];
#pragma unroll
                for (int r = 0; r < N2; ++r)
#pragma unroll
                    for (int c = 0; c < N2; ++c) W[r][c] = M[r][c];
                detM = det_real<N2>(W);
                const double dev = isfinite(detM) ? fabs(fma(detM, detM, -1.0)) : CUDART_INF;
                stab = dev > stab ? dev : stab;
                if (dev > A.stab_tol) good = false;
            }
            // Herman-Kluk prefactor matrix and its determinant
            {
                cplx Am[F][F];
#pragma unroll
                for (int a = 0; a < F; ++a)
#pragma unroll
                    for (int b = 0; b < F; ++b) {
                        const double sab = A.rg[a] * A.irg[b];   // sqrt(g_a / g_b)
                        const double sba = A.rg[b] * A.irg[a];   // sqrt(g_b / g_a)
                        const double pab = A.rg[a] * A.rg[b];
                        const double iab = A.irg[a] * A.irg[b];
                        const double re = fma(sab, M[F + a][F + b], sba * M[a][b]);
                        const double im = fma(-pab, M[F + a][b], iab * M[a][F + b]);
                        Am[a][b] = {0.5 * re, 0.5 * im};
                    }
                detA = det_complex<F>(Am);
                const double arg_new = atan2(detA.im, detA.re);
                double d = arg_new - arg_old + A.ref_step;
                d = fma(-kTwoPi, rint(d * kInvTwoPi), d);
                theta += d - A.ref_step;
                arg_old = arg_new;
            }
            bool finite = isfinite(S) && isfinite(theta);
#pragma unroll
            for (int a = 0; a < F; ++a) finite = finite && isfinite(p[a]) && isfinite(q[a]);
            if (!finite) good = false;
        }
        // amplitudes <chi_x|p q> e^{i (S + theta/2)}
        double re00 = 0.0;   // Re log <chi_0|p0 q0>, set by the x = 0 iteration (Herman-Kluk summand)
        for (int x = 0; x < A.n_chi; ++x) {
            double re = 0.0, im = 0.0;
#pragma unroll
            for (int a = 0; a < F; ++a) {
                const double dq = A.q_eq[x * F + a] - q[a];
                const double dp = A.p_eq[x * F + a] - p[a];
                re = fma(-A.qw[a] * dq, dq, re);
                re = fma(-A.pw[a] * dp, dp, re);
                im = fma(0.5 * (A.p_eq[x * F + a] + p[a]), dq, im);
            }
            double ph = im + S + 0.5 * theta;
            if (A.amplitude == SCIVR_AMP_HK) {
                // Herman-Kluk summand: |det A|^{1/2} and the division by the initial
                // overlap times the sampling weight (chi_log_overlap0)
                double re0, im0;
                chi_log_overlap0<F>(A, L.p0, L.q0, n, j, x, re00, re0, im0);
                re = re - re0 + 0.5 * log(hypot(detA.re, detA.im));
                ph -= im0;
            }
            double sn, cs;
            sincos(ph, &sn, &cs);
            const double mag = exp(re);
            amp_store(L, x * L.chi_stride + j * L.amp_ld + step, mag * cs, mag * sn);
        }
    }
    L.good[j] = good ? 1 : 0;
    const FinalDev &fo = L.fin;
    if (fo.p) for (int a = 0; a < F; ++a) fo.p[a * n + j] = p[a];
    if (fo.q) for (int a = 0; a < F; ++a) fo.q[a * n + j] = q[a];
    if (fo.S) fo.S[j] = S;
    if (fo.theta) fo.theta[j] = theta;
    if (fo.detM) fo.detM[j] = detM;
    if (fo.stab) fo.stab[j] = stab;
    if (fo.detA) { fo.detA[2 * j] = detA.re; fo.detA[2 * j + 1] = detA.im; }
    if (fo.M) {
#pragma unroll
        for (int r = 0; r < N2; ++r)
#pragma unroll
            for (int c = 0; c < N2; ++c) fo.M[j * N2 * N2 + r * N2 + c] = M[r][c];
    }
}

}  // namespace tpt

template <int F>
cudaError_t launch_tpt_fp64(const PropLaunch &L, cudaStream_t s)
{
    using namespace tpt;
    const int threads = 64;
    const int64_t blocks = (L.n_traj + threads - 1) / threads;
    k_propagate_tpt_fp64<F><<<(unsigned)blocks, threads, 0, s>>>(L);
    return cudaGetLastError();
}


}  // namespace scivr
