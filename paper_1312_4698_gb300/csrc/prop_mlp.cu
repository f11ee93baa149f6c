// Propagation on a potential with a learned residual (Sec. III.A schedule,
// split into stages so that every force evaluation of the network is one
// batched tensor-core evaluation over all trajectories).
//
// Per step of the fourth-order triple jump  D(c0) K(d0) D(c1) K(d1) D(c2) K(d2) D(c3):
//   network at q  ->  stage 1: K(d0) D(c1)
//   network at q  ->  stage 2: K(d1) D(c2)
//   network at q  ->  stage 3: K(d2) D(c3), det M (stability), det A and the
//                     continuous phase, the amplitude of Eq. I(E)_discreto,
//                     then D(c0) of the next step
// and stage 0 (before the first step) sets M = I, records c = 0 and drifts
// D(c0).  A kick uses V, grad V and the Hessian of the analytic surface (FP64,
// at q) plus those of the network (FP32, at q rounded to FP32).  State between
// stages lives in HBM: p, q, S, theta (FP64, structure of arrays) and M (FP32,
// element (r, c) of trajectory j at (r 2F + c) n + j).  One thread per
// trajectory; the kick and drift stream M column by column.
#include "propagate_tpt.cuh"

namespace scivr {
namespace pm {

struct State {
    double *p, *q;        // [F][n]
    float *M;             // [(2F)^2][n]
    double *S, *theta, *arg_old, *stab;
    float *qf;            // [n][F] network input
    const float *Vm, *gm, *Hm;   // network output at qf: [n], [n][F], [n][F][F]
    int *step;            // device step counter (column of the amplitude)
};

// Amplitude of step `step` for every reference state: the time-averaged summand,
// or with SCIVR_AMP_HK the Herman-Kluk summand (|det A|^{1/2} = sqrt(absA), divided
// by the initial overlap times the sampling weight, chi_log_overlap0).
template <int F>
__device__ __forceinline__ void record(const PropLaunch &L, int64_t j, int step, const double (&p)[F],
                                       const double (&q)[F], double S, double theta, double absA)
{
    const PropArgs &A = L.args;
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
            double re0, im0;
            chi_log_overlap0<F>(A, L.p0, L.q0, L.n_traj, j, x, re00, re0, im0);
            re = re - re0 + 0.5 * log(absA);
            ph -= im0;
        }
        double sn, cs;
        sincos(ph, &sn, &cs);
        const double mag = exp(re);
        amp_store(L, x * L.chi_stride + j * L.amp_ld + step, mag * cs, mag * sn);
    }
}

// Drift of (q, S) by td (FP64).
template <int F>
__device__ __forceinline__ void drift_qs(double td, const double (&p)[F], double (&q)[F], double &S)
{
    double kin = 0.0;
#pragma unroll
    for (int a = 0; a < F; ++a) kin = fma(0.5 * p[a], p[a], kin);
    S = fma(td, kin, S);
#pragma unroll
    for (int a = 0; a < F; ++a) q[a] = fma(td, p[a], q[a]);
}

// KIND 0: set-up and the first drift; 1: a kick and a drift (stage = 1, 2);
// 3: the last kick and drift of a step, the per-step diagnostics, and the next
// step's first drift.  COUPLED: the analytic part has coupling terms (else it
// is the separable diagonal alone and its Hessian is diagonal).  The kick and
// the drift update M in one pass over its columns (M_p -= tk H M_q, then
// M_q += td M_p); the final stage also copies M into the work array of its LU.
template <int F, int KIND, bool COUPLED>
__global__ void __launch_bounds__(KIND == 3 ? 64 : 128, KIND == 3 ? 2 : 3) k_mlp_stage(const PropLaunch L, State st, int stage)
{
    constexpr int N2 = 2 * F;
    constexpr int NT = 64;                    // threads per block of the final stage
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t n = L.n_traj;
    const PropArgs &A = L.args;
    if (KIND == 1 && stage == 1 && j == 0) *st.step += 1;   // read by stage 3 of this step (later in stream order)
    if (j >= n) return;
    float *Mj = st.M + j;                     // element (r, c) at Mj[(r 2F + c) n]
    extern __shared__ __align__(16) uint8_t fin_smem[];
    float *W = reinterpret_cast<float *>(fin_smem) + threadIdx.x;   // final stage: (r, c) at W[(r 2F + c) NT]
    double p[F], q[F], S;
    if (KIND == 0) {
#pragma unroll
        for (int a = 0; a < F; ++a) {
            p[a] = L.p0[a * n + j];
            q[a] = L.q0[a * n + j];
        }
        S = 0.0;
        st.theta[j] = 0.0;
        st.arg_old[j] = 0.0;
        st.stab[j] = 0.0;
        L.good[j] = 1;
        record<F>(L, j, 0, p, q, 0.0, 0.0, 1.0);
        const float td = A.tdrift_f[0];
        for (int c = 0; c < N2; ++c)
#pragma unroll
            for (int a = 0; a < F; ++a) {
                const float mp = a == c ? 1.0f : 0.0f;
                const float mq = (F + a == c ? 1.0f : 0.0f) + td * mp;
                Mj[((int64_t)a * N2 + c) * n] = mp;
                Mj[((int64_t)(F + a) * N2 + c) * n] = mq;
            }
        drift_qs<F>(A.tdrift[0], p, q, S);
    } else {
#pragma unroll
        for (int a = 0; a < F; ++a) {
            p[a] = st.p[a * n + j];
            q[a] = st.q[a * n + j];
        }
        S = st.S[j];
        // kick d_{stage-1}: analytic part (FP64) + network part (FP32)
        const double tk = A.tkick[stage - 1];
        const float tkf = A.tkick_f[stage - 1];
        float Hk[F][F];
#pragma unroll
        for (int a = 0; a < F; ++a)
#pragma unroll
            for (int b = 0; b < F; ++b) Hk[a][b] = tkf * st.Hm[(j * F + a) * F + b];
        double V = (double)st.Vm[j];
        if constexpr (COUPLED) {
            double H[F][F], g[F], Va;
            tpt::pes_fp64<F>(L.pes, q, H, g, Va);
            V += Va;
#pragma unroll
            for (int a = 0; a < F; ++a) {
                p[a] = fma(-tk, g[a] + (double)st.gm[j * F + a], p[a]);
#pragma unroll
                for (int b = 0; b < F; ++b) Hk[a][b] += (float)(tk * H[a][b]);
            }
        } else {
            // separable diagonal only: V, grad V and the (diagonal) Hessian per mode
#pragma unroll
            for (int a = 0; a < F; ++a) {
                double Va, ga, ha;
                if (L.pes.diag_kind == SCIVR_DIAG_MORSE) {
                    const double Dm = __ldg(L.pes.D + a), am = __ldg(L.pes.a + a);
                    const double u = exp(-am * q[a]);
                    const double omu = 1.0 - u;
                    Va = Dm * omu * omu;
                    ga = 2.0 * Dm * am * u * omu;
                    ha = 2.0 * Dm * am * am * u * (2.0 * u - 1.0);
                } else {
                    const double w2 = __ldg(L.pes.omega + a) * __ldg(L.pes.omega + a);
                    Va = 0.5 * w2 * q[a] * q[a];
                    ga = w2 * q[a];
                    ha = w2;
                }
                V += Va;
                p[a] = fma(-tk, ga + (double)st.gm[j * F + a], p[a]);
                Hk[a][a] += (float)(tk * ha);
            }
        }
        S = fma(-tk, V, S);
        const float td = A.tdrift_f[stage];
#pragma unroll 1
        for (int c = 0; c < N2; ++c) {
            float mp[F], mq[F];
#pragma unroll
            for (int a = 0; a < F; ++a) {
                mp[a] = Mj[((int64_t)a * N2 + c) * n];
                mq[a] = Mj[((int64_t)(F + a) * N2 + c) * n];
            }
#pragma unroll
            for (int a = 0; a < F; ++a) {
                float hm = 0.0f;
#pragma unroll
                for (int b = 0; b < F; ++b) hm = fmaf(Hk[a][b], mq[b], hm);
                mp[a] -= hm;
            }
#pragma unroll
            for (int a = 0; a < F; ++a) {
                mq[a] = fmaf(td, mp[a], mq[a]);
                Mj[((int64_t)a * N2 + c) * n] = mp[a];
                Mj[((int64_t)(F + a) * N2 + c) * n] = mq[a];
                if (KIND == 3) {
                    W[(a * N2 + c) * NT] = mp[a];
                    W[((F + a) * N2 + c) * NT] = mq[a];
                }
            }
        }
        drift_qs<F>(A.tdrift[stage], p, q, S);
    }
    if (KIND == 3) {
        const int step = *st.step;
        bool good = L.good[j] != 0;
        // stability |det(M)^2 - 1| (FP32 LU with partial pivoting) on the copy
        // in shared memory, laid out [element][thread] (bank-conflict free)
        // fully unrolled: every shared-memory offset is a compile-time constant
        // relative to the row pointers, and the pivot row sits in registers
        float det = 1.0f;
#pragma unroll
        for (int k = 0; k < N2; ++k) {
            int piv = k;
            float best = fabsf(W[(k * N2 + k) * NT]);
#pragma unroll 1
            for (int i = k + 1; i < N2; ++i) {
                const float v = fabsf(W[(i * N2 + k) * NT]);
                if (v > best) { best = v; piv = i; }
            }
            float rkv[N2];
            float *rp = W + piv * N2 * NT;
#pragma unroll
            for (int c = k; c < N2; ++c) rkv[c] = rp[c * NT];
            if (piv != k) {
#pragma unroll
                for (int c = k; c < N2; ++c) rp[c * NT] = W[(k * N2 + c) * NT];
                det = -det;
            }
            det *= rkv[k];
            const float inv = 1.0f / rkv[k];
#pragma unroll 1
            for (int i = k + 1; i < N2; ++i) {
                float *ri = W + i * N2 * NT;
                const float l = ri[k * NT] * inv;
#pragma unroll
                for (int c = k + 1; c < N2; ++c) ri[c * NT] = fmaf(-l, rkv[c], ri[c * NT]);
            }
        }
        const float dev = isfinite(det) ? fabsf(fmaf(det, det, -1.0f)) : __int_as_float(0x7f800000);
        const double stab = fmax(st.stab[j], (double)dev);
        st.stab[j] = stab;
        if (dev > A.stab_tol_f) good = false;
        // Herman-Kluk prefactor determinant (FP64, complex LU with partial
        // pivoting) in the same shared memory: (a, b) re at Z[(2 (a F + b)) NT], im at + NT
        double *Z = reinterpret_cast<double *>(fin_smem) + threadIdx.x;
        for (int a = 0; a < F; ++a)
            for (int b = 0; b < F; ++b) {
                const float mqq = Mj[((int64_t)(F + a) * N2 + F + b) * n];
                const float mpp = Mj[((int64_t)a * N2 + b) * n];
                const float mqp = Mj[((int64_t)(F + a) * N2 + b) * n];
                const float mpq = Mj[((int64_t)a * N2 + F + b) * n];
                Z[(2 * (a * F + b)) * NT] = 0.5 * fma(A.rg[a] * A.irg[b], (double)mqq, A.rg[b] * A.irg[a] * (double)mpp);
                Z[(2 * (a * F + b) + 1) * NT] = 0.5 * fma(-A.rg[a] * A.rg[b], (double)mqp, A.irg[a] * A.irg[b] * (double)mpq);
            }
        tpt::cplx dA = {1.0, 0.0};
#pragma unroll
        for (int k = 0; k < F; ++k) {
            int piv = k;
            double best = Z[(2 * (k * F + k)) * NT] * Z[(2 * (k * F + k)) * NT] +
                          Z[(2 * (k * F + k) + 1) * NT] * Z[(2 * (k * F + k) + 1) * NT];
#pragma unroll 1
            for (int i = k + 1; i < F; ++i) {
                const double vr = Z[(2 * (i * F + k)) * NT], vi = Z[(2 * (i * F + k) + 1) * NT];
                const double v = vr * vr + vi * vi;
                if (v > best) { best = v; piv = i; }
            }
            tpt::cplx rkv[F];
            double *rp = Z + 2 * piv * F * NT;
#pragma unroll
            for (int c = k; c < F; ++c) rkv[c] = {rp[2 * c * NT], rp[(2 * c + 1) * NT]};
            if (piv != k) {
#pragma unroll
                for (int c = k; c < F; ++c) {
                    rp[2 * c * NT] = Z[(2 * (k * F + c)) * NT];
                    rp[(2 * c + 1) * NT] = Z[(2 * (k * F + c) + 1) * NT];
                }
                dA.re = -dA.re; dA.im = -dA.im;
            }
            dA = tpt::cmul(dA, rkv[k]);
            const double rr = 1.0 / (rkv[k].re * rkv[k].re + rkv[k].im * rkv[k].im);
            const tpt::cplx inv = {rkv[k].re * rr, -rkv[k].im * rr};
#pragma unroll 1
            for (int i = k + 1; i < F; ++i) {
                double *ri = Z + 2 * i * F * NT;
                const tpt::cplx l = tpt::cmul({ri[2 * k * NT], ri[(2 * k + 1) * NT]}, inv);
#pragma unroll
                for (int c = k + 1; c < F; ++c) {
                    const tpt::cplx y = tpt::cfnma(l, rkv[c], {ri[2 * c * NT], ri[(2 * c + 1) * NT]});
                    ri[2 * c * NT] = y.re;
                    ri[(2 * c + 1) * NT] = y.im;
                }
            }
        }
        const double arg_new = atan2(dA.im, dA.re);
        double d = arg_new - st.arg_old[j] + A.ref_step;
        d = fma(-kTwoPi, rint(d * kInvTwoPi), d);
        const double theta = st.theta[j] + d - A.ref_step;
        st.theta[j] = theta;
        st.arg_old[j] = arg_new;
        bool finite = isfinite(S) && isfinite(theta);
#pragma unroll
        for (int a = 0; a < F; ++a) finite = finite && isfinite(p[a]) && isfinite(q[a]);
        if (!finite) good = false;
        L.good[j] = good ? 1 : 0;
        record<F>(L, j, step, p, q, S, theta, hypot(dA.re, dA.im));
        if (step == A.n_steps) {
            const FinalDev &fo = L.fin;
            if (fo.p) for (int a = 0; a < F; ++a) fo.p[a * n + j] = p[a];
            if (fo.q) for (int a = 0; a < F; ++a) fo.q[a * n + j] = q[a];
            if (fo.S) fo.S[j] = S;
            if (fo.theta) fo.theta[j] = theta;
            if (fo.detM) fo.detM[j] = (double)det;
            if (fo.stab) fo.stab[j] = stab;
            if (fo.detA) { fo.detA[2 * j] = dA.re; fo.detA[2 * j + 1] = dA.im; }
            if (fo.M)
                for (int r = 0; r < N2; ++r)
                    for (int c = 0; c < N2; ++c) fo.M[j * N2 * N2 + r * N2 + c] = Mj[((int64_t)r * N2 + c) * n];
            return;
        }
        // first drift of the next step
        const float td0 = A.tdrift_f[0];
#pragma unroll 1
        for (int c = 0; c < N2; ++c)
#pragma unroll
            for (int a = 0; a < F; ++a) {
                float *mq = Mj + ((int64_t)(F + a) * N2 + c) * n;
                *mq = fmaf(td0, Mj[((int64_t)a * N2 + c) * n], *mq);
            }
        drift_qs<F>(A.tdrift[0], p, q, S);
    }
#pragma unroll
    for (int a = 0; a < F; ++a) {
        st.p[a * n + j] = p[a];
        st.q[a * n + j] = q[a];
        st.qf[j * F + a] = (float)q[a];
    }
    st.S[j] = S;
}

inline size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

template <int F>
cudaError_t run(const PropLaunch &L, cudaStream_t s, int *n_launch)
{
    constexpr int N2 = 2 * F;
    const int64_t n = L.n_traj;
    size_t o = 0;
    const size_t oP = o; o += a256((size_t)F * n * 8);
    const size_t oQ = o; o += a256((size_t)F * n * 8);
    const size_t oM = o; o += a256((size_t)N2 * N2 * n * 4);
    const size_t oS = o; o += a256((size_t)n * 8);
    const size_t oT = o; o += a256((size_t)n * 8);
    const size_t oA = o; o += a256((size_t)n * 8);
    const size_t oB = o; o += a256((size_t)n * 8);
    const size_t oQf = o; o += a256((size_t)n * F * 4);
    const size_t oV = o; o += a256((size_t)n * 4);
    const size_t oG = o; o += a256((size_t)n * F * 4);
    const size_t oH = o; o += a256((size_t)n * F * F * 4);
    const size_t oStep = o; o += 256;
    const size_t oEval = o; o += mlp_eval_scratch_bytes(F, n, true);
    void *scr = nullptr;
    cudaError_t e = cudaMallocAsync(&scr, o, s);
    if (e != cudaSuccess) return e;
    char *b = static_cast<char *>(scr);
    State st{};
    st.p = reinterpret_cast<double *>(b + oP);
    st.q = reinterpret_cast<double *>(b + oQ);
    st.M = reinterpret_cast<float *>(b + oM);
    st.S = reinterpret_cast<double *>(b + oS);
    st.theta = reinterpret_cast<double *>(b + oT);
    st.arg_old = reinterpret_cast<double *>(b + oA);
    st.stab = reinterpret_cast<double *>(b + oB);
    st.qf = reinterpret_cast<float *>(b + oQf);
    float *Vm = reinterpret_cast<float *>(b + oV), *gm = reinterpret_cast<float *>(b + oG);
    float *Hm = reinterpret_cast<float *>(b + oH);
    st.Vm = Vm; st.gm = gm; st.Hm = Hm;
    st.step = reinterpret_cast<int *>(b + oStep);
    int nl = 0;
    e = cudaMemsetAsync(st.step, 0, sizeof(int), s);
    if (e == cudaSuccess) e = mlp_prepare();
    const unsigned blocks = (unsigned)((n + 127) / 128);
    // final stage: one [element][thread] work array per thread, 16 F^2 bytes (the
    // FP32 (2F)^2 LU and the FP64 complex F^2 LU need the same size)
    const size_t fin_smem = (size_t)64 * 16 * F * F;
    if (e == cudaSuccess) {
        e = cudaFuncSetAttribute(k_mlp_stage<F, 3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fin_smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_mlp_stage<F, 3, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fin_smem);
    }
    if (e == cudaSuccess) {
        k_mlp_stage<F, 0, false><<<blocks, 128, 0, s>>>(L, st, 0);
        nl += 1;
        for (int step = 1; step <= L.args.n_steps && e == cudaSuccess; ++step) {
            for (int stage = 1; stage <= 3; ++stage) {
                int ne = 0;
                e = mlp_eval(L.pes.mlp, F, n, st.qf, Vm, gm, Hm, b + oEval, s, &ne);
                nl += ne;
                if (e != cudaSuccess) break;
                const bool cpl = L.pes.has3 || L.pes.has4;
                if (stage < 3) {
                    if (cpl) k_mlp_stage<F, 1, true><<<blocks, 128, 0, s>>>(L, st, stage);
                    else k_mlp_stage<F, 1, false><<<blocks, 128, 0, s>>>(L, st, stage);
                } else {
                    const unsigned b64 = (unsigned)((n + 63) / 64);
                    if (cpl) k_mlp_stage<F, 3, true><<<b64, 64, fin_smem, s>>>(L, st, stage);
                    else k_mlp_stage<F, 3, false><<<b64, 64, fin_smem, s>>>(L, st, stage);
                }
                nl += 1;
            }
            if (e == cudaSuccess) e = cudaGetLastError();
        }
    }
    cudaError_t e2 = cudaFreeAsync(scr, s);
    *n_launch = nl;
    return e != cudaSuccess ? e : e2;
}

}  // namespace pm

cudaError_t launch_propagate_mlp(const PropLaunch &L, cudaStream_t s, int *n_launch)
{
    switch (L.args.F) {
#define SCIVR_PM(FF) case FF: return pm::run<FF>(L, s, n_launch);
    SCIVR_PM(1) SCIVR_PM(2) SCIVR_PM(3) SCIVR_PM(4) SCIVR_PM(5) SCIVR_PM(6) SCIVR_PM(7) SCIVR_PM(8) SCIVR_PM(9)
#undef SCIVR_PM
    default: *n_launch = 0; return cudaErrorInvalidValue;
    }
}

}  // namespace scivr
