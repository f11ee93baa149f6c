// C-ABI entry points of libscivr (declared in include/scivr.h): argument
// validation, potential packing, launch dispatch and error reporting.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "scivr_internal.cuh"

using namespace scivr;

namespace {

thread_local std::string g_last_error;
thread_local int64_t g_launches = 0;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *where)
{
    if (e == cudaErrorMemoryAllocation)
        return fail(SCIVR_ENOMEM, "%s: %s", where, cudaGetErrorString(e));
    return fail(SCIVR_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

void ok() { g_last_error.clear(); }

bool all_positive_finite(const double *x, int n)
{
    for (int i = 0; i < n; ++i)
        if (!(x[i] > 0.0) || !std::isfinite(x[i])) return false;
    return true;
}

bool all_finite(const double *x, int n)
{
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(x[i])) return false;
    return true;
}

inline int packed(int F, int a, int b)   // a <= b
{
    return a * F - a * (a - 1) / 2 + (b - a);
}

// Fourth-order triple jump (Yoshida 1990): with s = 2^{1/3},
// w1 = 1 / (2 - s), w0 = -s / (2 - s); drifts w1/2, (w0+w1)/2, (w0+w1)/2, w1/2
// and kicks w1, w0, w1 (fractions of dt).
void triple_jump(double c[4], double d[3])
{
    const double s = std::cbrt(2.0);
    const double w1 = 1.0 / (2.0 - s), w0 = -s / (2.0 - s);
    c[0] = c[3] = 0.5 * w1;
    c[1] = c[2] = 0.5 * (w0 + w1);
    d[0] = d[2] = w1;
    d[1] = w0;
}

}  // namespace

namespace scivr {

// Validate scivr_propagate's arguments and fill the kernel launch record.
// Returns SCIVR_OK or an error code (with the message set).
int prepare_propagate(scivr_pes pes, const scivr_prop_params *prm, int64_t n_traj, const double *p0,
                      const double *q0, void *amp, int64_t amp_ld, uint8_t *good,
                      const scivr_final_state *fin, PropLaunch *out)
{
    if (!pes || !prm) return fail(SCIVR_EINVAL, "scivr_propagate: NULL potential or parameters");
    const int F = pes->dev.F;
    if (!p0 || !q0 || !amp || !good) return fail(SCIVR_EINVAL, "scivr_propagate: NULL device pointer");
    if (n_traj < 1) return fail(SCIVR_EINVAL, "scivr_propagate: n_traj=%lld < 1", (long long)n_traj);
    if (prm->n_steps < 1) return fail(SCIVR_EINVAL, "scivr_propagate: n_steps=%d < 1", prm->n_steps);
    if (!(prm->dt > 0.0) || !std::isfinite(prm->dt)) return fail(SCIVR_EINVAL, "scivr_propagate: dt must be positive");
    if (!(prm->stab_tol >= 0.0)) return fail(SCIVR_EINVAL, "scivr_propagate: stab_tol must be >= 0");
    if (prm->n_chi < 1 || prm->n_chi > SCIVR_MAX_CHI)
        return fail(SCIVR_EINVAL, "scivr_propagate: n_chi=%d not in [1,%d]", prm->n_chi, SCIVR_MAX_CHI);
    if (!prm->gamma || !prm->p_eq || !prm->q_eq) return fail(SCIVR_EINVAL, "scivr_propagate: NULL gamma/chi");
    if (!all_positive_finite(prm->gamma, F)) return fail(SCIVR_EINVAL, "scivr_propagate: gamma must be positive");
    if (!all_finite(prm->p_eq, F * prm->n_chi) || !all_finite(prm->q_eq, F * prm->n_chi))
        return fail(SCIVR_EINVAL, "scivr_propagate: chi not finite");
    if (amp_ld < (int64_t)prm->n_steps + 1)
        return fail(SCIVR_EINVAL, "scivr_propagate: amp_ld=%lld < n_steps+1", (long long)amp_ld);
    if (prm->amp_prec != SCIVR_FP64 && prm->amp_prec != SCIVR_MIXED)
        return fail(SCIVR_EINVAL, "scivr_propagate: amp_prec %d invalid", prm->amp_prec);
    if (prm->amp_prec == SCIVR_MIXED && (prm->precision != SCIVR_MIXED || prm->amplitude != SCIVR_AMP_TA))
        return fail(SCIVR_EINVAL, "scivr_propagate: FP32 amplitude storage takes mixed precision and "
                                  "time-averaged amplitudes");
    if (reinterpret_cast<uintptr_t>(amp) % (prm->amp_prec == SCIVR_MIXED ? 8 : 16) != 0)
        return fail(SCIVR_EINVAL, "scivr_propagate: amp not aligned to its element (16 bytes, 8 for FP32)");
    if (prm->precision != SCIVR_FP64 && prm->precision != SCIVR_MIXED)
        return fail(SCIVR_EINVAL, "scivr_propagate: precision %d invalid", prm->precision);
    if (prm->kernel < SCIVR_KERNEL_AUTO || prm->kernel > SCIVR_KERNEL_GROUP)
        return fail(SCIVR_EINVAL, "scivr_propagate: kernel %d invalid", prm->kernel);
    if (prm->amplitude != SCIVR_AMP_TA && prm->amplitude != SCIVR_AMP_HK)
        return fail(SCIVR_EINVAL, "scivr_propagate: amplitude %d invalid", prm->amplitude);
    if (!propagate_supported(F, prm->precision, prm->kernel))
        return fail(SCIVR_EUNSUPPORTED, "scivr_propagate: precision %d / kernel %d not built for F=%d",
                    prm->precision, prm->kernel, F);
    if (pes->dev.kind == SCIVR_PES_CART3 && (prm->precision != SCIVR_FP64 || prm->kernel == SCIVR_KERNEL_GROUP))
        return fail(SCIVR_EUNSUPPORTED, "scivr_propagate: a Cartesian surface propagates in FP64 with the "
                                        "thread-per-trajectory schedule");

    PropLaunch L{};
    L.pes = pes->dev;
    PropArgs &A = L.args;
    A.F = F;
    A.n_steps = prm->n_steps;
    A.n_chi = prm->n_chi;
    A.precision = prm->precision;
    A.kernel = (pes->dev.kind == SCIVR_PES_CART3) ? SCIVR_KERNEL_THREAD : prm->kernel;
    A.amplitude = prm->amplitude;
    A.dt = prm->dt;
    A.stab_tol = prm->stab_tol;
    triple_jump(A.cdrift, A.dkick);
    for (int i = 0; i < 4; ++i) {
        A.tdrift[i] = A.cdrift[i] * prm->dt;
        A.tdrift_f[i] = (float)A.tdrift[i];
        A.tdrift_lo[i] = (float)(A.tdrift[i] - (double)A.tdrift_f[i]);
    }
    for (int i = 0; i < 3; ++i) {
        A.tkick[i] = A.dkick[i] * prm->dt;
        A.tkick_f[i] = (float)A.tkick[i];
        A.tkick_lo[i] = (float)(A.tkick[i] - (double)A.tkick_f[i]);
    }
    A.stab_tol_f = prm->stab_tol > 3.0e38 ? 3.0e38f : (float)prm->stab_tol;
    double ref = 0.0;
    for (int i = 0; i < F; ++i) {
        const double g = prm->gamma[i];
        A.gamma[i] = g;
        A.rg[i] = std::sqrt(g);
        A.irg[i] = 1.0 / std::sqrt(g);
        A.qw[i] = 0.25 * g;
        A.pw[i] = 0.25 / g;
        ref += g * prm->dt;
    }
    A.ref_step = ref;
    for (int i = 0; i < F * prm->n_chi; ++i) {
        A.p_eq[i] = prm->p_eq[i];
        A.q_eq[i] = prm->q_eq[i];
    }
    L.n_traj = n_traj;
    L.p0 = p0;
    L.q0 = q0;
    L.amp = static_cast<double2 *>(amp);
    L.amp_f32 = prm->amp_prec == SCIVR_MIXED;
    L.amp_ld = amp_ld;
    L.chi_stride = n_traj * amp_ld;
    L.good = good;
    if (fin) L.fin = FinalDev{fin->p, fin->q, fin->S, fin->theta, fin->detM, fin->detA, fin->M, fin->stab};
    *out = L;
    return SCIVR_OK;
}

// Validate scivr_spectrum's arguments (shared with the batch path).
int check_spectrum_args(const void *amp, int64_t amp_ld, int32_t amp_prec, const double *w, const uint8_t *good,
                        int64_t n_traj, int32_t n_steps, double dt, double E_min, double E_max, int32_t n_E,
                        int32_t ft_mode, const double *I_out, const char *who)
{
    if (!amp || !w || !good || !I_out) return fail(SCIVR_EINVAL, "%s: NULL device pointer", who);
    if (n_traj < 1) return fail(SCIVR_EINVAL, "%s: n_traj=%lld < 1", who, (long long)n_traj);
    if (n_steps < 1) return fail(SCIVR_EINVAL, "%s: n_steps=%d < 1", who, n_steps);
    if (n_E < 2) return fail(SCIVR_EINVAL, "%s: n_E=%d < 2", who, n_E);
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(SCIVR_EINVAL, "%s: dt must be positive", who);
    if (!std::isfinite(E_min) || !std::isfinite(E_max) || !(E_max > E_min))
        return fail(SCIVR_EINVAL, "%s: need finite E_min < E_max", who);
    if (amp_ld < (int64_t)n_steps + 1) return fail(SCIVR_EINVAL, "%s: amp_ld < n_steps+1", who);
    if (amp_prec != SCIVR_FP64 && amp_prec != SCIVR_MIXED)
        return fail(SCIVR_EINVAL, "%s: amp_prec %d invalid", who, amp_prec);
    if (reinterpret_cast<uintptr_t>(amp) % (amp_prec == SCIVR_MIXED ? 8 : 16) != 0)
        return fail(SCIVR_EINVAL, "%s: amp not aligned to its element (16 bytes, 8 for FP32)", who);
    if (ft_mode != SCIVR_FT_FP64 && ft_mode != SCIVR_FT_CZT64 && ft_tc_digits(ft_mode) == 0)
        return fail(SCIVR_EUNSUPPORTED, "%s: ft_mode %d not supported", who, ft_mode);
    if (ft_mode == SCIVR_FT_CZT64 && (n_steps + 1 > spectrum_czt_max_samples() || n_E > kCztMaxEnergies))
        return fail(SCIVR_EUNSUPPORTED, "%s: the chirp-z mode takes n_steps + 1 <= %d and n_E <= %d", who,
                    spectrum_czt_max_samples(), kCztMaxEnergies);
    return SCIVR_OK;
}

int set_error(int code, const char *msg) { return fail(code, "%s", msg); }
void clear_error() { ok(); }
void count_launches(int n) { g_launches += n; }
int cuda_error(cudaError_t e, const char *where) { return cuda_fail(e, where); }

}  // namespace scivr

extern "C" {

const char *scivr_last_error(void) { return g_last_error.c_str(); }

int64_t scivr_launch_count(int reset)
{
    const int64_t v = g_launches;
    if (reset) g_launches = 0;
    return v;
}

int32_t scivr_pes_modes(scivr_pes pes) { return pes ? pes->dev.F : 0; }

int scivr_create_pes(const scivr_pes_desc *d, scivr_pes *out)
{
    if (!d || !out) return fail(SCIVR_EINVAL, "scivr_create_pes: NULL argument");
    *out = nullptr;
    const int F = d->F;
    if (F < 1 || F > SCIVR_MAX_F) return fail(SCIVR_EINVAL, "scivr_create_pes: F=%d not in [1,%d]", F, SCIVR_MAX_F);
    if (d->kind != SCIVR_PES_POLY) return fail(SCIVR_EUNSUPPORTED, "scivr_create_pes: kind %d not supported", d->kind);
    if (d->diag_kind != SCIVR_DIAG_HARMONIC && d->diag_kind != SCIVR_DIAG_MORSE)
        return fail(SCIVR_EINVAL, "scivr_create_pes: diag_kind %d invalid", d->diag_kind);
    if (!d->omega || !all_positive_finite(d->omega, F))
        return fail(SCIVR_EINVAL, "scivr_create_pes: omega must be %d positive finite values", F);
    if (d->diag_kind == SCIVR_DIAG_MORSE) {
        if (!d->D || !all_positive_finite(d->D, F)) return fail(SCIVR_EINVAL, "scivr_create_pes: Morse D must be positive");
        if (!d->a || !all_positive_finite(d->a, F)) return fail(SCIVR_EINVAL, "scivr_create_pes: Morse a must be positive");
    }
    if (d->n3 < 0 || d->n4 < 0) return fail(SCIVR_EINVAL, "scivr_create_pes: negative monomial count");
    if (d->n3 > 0 && (!d->idx3 || !d->c3)) return fail(SCIVR_EINVAL, "scivr_create_pes: NULL cubic arrays");
    if (d->n4 > 0 && (!d->idx4 || !d->c4)) return fail(SCIVR_EINVAL, "scivr_create_pes: NULL quartic arrays");

    const int P = F * (F + 1) / 2;
    std::vector<double> T3((size_t)F * P, 0.0), T4((size_t)P * P, 0.0);
    // Hessian of c * prod_s q[idx[s]]: for every ordered pair of positions (s, t),
    // s != t, the remaining factors multiply into entry (idx[s], idx[t]).  Only the
    // upper triangle (a <= b) is kept; the lower triangle is its mirror.
    for (int m = 0; m < d->n3; ++m) {
        const int32_t *ix = d->idx3 + 3 * m;
        for (int s = 0; s < 3; ++s)
            if (ix[s] < 0 || ix[s] >= F || (s > 0 && ix[s] < ix[s - 1]))
                return fail(SCIVR_EINVAL, "scivr_create_pes: cubic monomial %d indices invalid or unsorted", m);
        if (!std::isfinite(d->c3[m])) return fail(SCIVR_EINVAL, "scivr_create_pes: cubic coefficient %d not finite", m);
        for (int s = 0; s < 3; ++s)
            for (int t = 0; t < 3; ++t) {
                if (s == t) continue;
                const int u = 3 - s - t;
                const int a = ix[s], b = ix[t];
                if (a > b) continue;
                T3[(size_t)ix[u] * P + packed(F, a, b)] += d->c3[m];
            }
    }
    for (int m = 0; m < d->n4; ++m) {
        const int32_t *ix = d->idx4 + 4 * m;
        for (int s = 0; s < 4; ++s)
            if (ix[s] < 0 || ix[s] >= F || (s > 0 && ix[s] < ix[s - 1]))
                return fail(SCIVR_EINVAL, "scivr_create_pes: quartic monomial %d indices invalid or unsorted", m);
        if (!std::isfinite(d->c4[m])) return fail(SCIVR_EINVAL, "scivr_create_pes: quartic coefficient %d not finite", m);
        for (int s = 0; s < 4; ++s)
            for (int t = 0; t < 4; ++t) {
                if (s == t) continue;
                int rest[2], nr = 0;
                for (int u = 0; u < 4; ++u)
                    if (u != s && u != t) rest[nr++] = ix[u];
                const int a = ix[s], b = ix[t];
                if (a > b) continue;
                const int k = rest[0] < rest[1] ? rest[0] : rest[1];
                const int l = rest[0] < rest[1] ? rest[1] : rest[0];
                T4[(size_t)packed(F, k, l) * P + packed(F, a, b)] += d->c4[m];
            }
    }
    // For a == b each ordered pair (s, t) with ix[s] == ix[t] was visited twice
    // (as (s,t) and (t,s)); for a < b only (s,t) with ix[s] < ix[t] survives the
    // a <= b filter, which counts each unordered pair once -- exactly the mixed
    // second derivative.  The diagonal entries therefore already hold the full
    // d^2/dq_a^2, so no further scaling is needed.

    std::vector<double> hostblob;
    auto push = [&](const double *x, size_t n) {
        const size_t off = hostblob.size();
        hostblob.insert(hostblob.end(), x, x + n);
        while (hostblob.size() % 32) hostblob.push_back(0.0);   // 256-byte alignment
        return off;
    };
    std::vector<double> zeros(F, 0.0);
    const size_t o_om = push(d->omega, F);
    const size_t o_D = push(d->diag_kind == SCIVR_DIAG_MORSE ? d->D : zeros.data(), F);
    const size_t o_a = push(d->diag_kind == SCIVR_DIAG_MORSE ? d->a : zeros.data(), F);
    const size_t o_T3 = push(T3.data(), T3.size());
    const size_t o_T4 = push(T4.data(), T4.size());
    std::vector<float> T3f(T3.begin(), T3.end()), T4f(T4.begin(), T4.end());
    // the same tensors with every row padded to a multiple of 4 floats (16-byte loads of four
    // consecutive Hessian entries; the kernels above F = 16 read them from global memory)
    const int P4 = (P + 3) & ~3;
    std::vector<float> T3p((size_t)F * P4, 0.0f), T4p((size_t)P * P4, 0.0f);
    for (int k = 0; k < F; ++k)
        for (int e = 0; e < P; ++e) T3p[(size_t)k * P4 + e] = T3f[(size_t)k * P + e];
    for (int kl = 0; kl < P; ++kl)
        for (int e = 0; e < P; ++e) T4p[(size_t)kl * P4 + e] = T4f[(size_t)kl * P + e];
    std::vector<float> diagf(3 * 64, 0.0f);   // omega, D, a in FP32, 64-float slots
    for (int i = 0; i < F; ++i) {
        diagf[i] = (float)d->omega[i];
        diagf[64 + i] = d->diag_kind == SCIVR_DIAG_MORSE ? (float)d->D[i] : 0.0f;
        diagf[128 + i] = d->diag_kind == SCIVR_DIAG_MORSE ? (float)d->a[i] : 0.0f;
    }
    const size_t nd = hostblob.size();
    const size_t bytes = nd * sizeof(double) +
                         (T3f.size() + T4f.size() + diagf.size() + T3p.size() + T4p.size() + 4 * 256) * sizeof(float);

    void *blob = nullptr;
    cudaError_t e = cudaMalloc(&blob, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "scivr_create_pes: cudaMalloc");
    char *b = static_cast<char *>(blob);
    e = cudaMemcpy(b, hostblob.data(), nd * sizeof(double), cudaMemcpyHostToDevice);
    const size_t o_T3f = nd * sizeof(double);
    const size_t o_T4f = o_T3f + ((T3f.size() * sizeof(float) + 255) & ~(size_t)255);
    if (e == cudaSuccess) e = cudaMemcpy(b + o_T3f, T3f.data(), T3f.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b + o_T4f, T4f.data(), T4f.size() * sizeof(float), cudaMemcpyHostToDevice);
    const size_t o_diagf = o_T4f + ((T4f.size() * sizeof(float) + 255) & ~(size_t)255);
    if (e == cudaSuccess) e = cudaMemcpy(b + o_diagf, diagf.data(), diagf.size() * sizeof(float), cudaMemcpyHostToDevice);
    const size_t o_T3p = o_diagf + ((diagf.size() * sizeof(float) + 255) & ~(size_t)255);
    const size_t o_T4p = o_T3p + ((T3p.size() * sizeof(float) + 255) & ~(size_t)255);
    if (e == cudaSuccess) e = cudaMemcpy(b + o_T3p, T3p.data(), T3p.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b + o_T4p, T4p.data(), T4p.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(blob);
        return cuda_fail(e, "scivr_create_pes: cudaMemcpy");
    }
    scivr_pes h = new scivr_pes_s{};
    h->blob = blob;
    h->mlp_blob = nullptr;
    PesDev &dv = h->dev;
    const double *db = reinterpret_cast<const double *>(b);
    dv.F = F;
    dv.P = P;
    dv.diag_kind = d->diag_kind;
    dv.has3 = d->n3 > 0;
    dv.has4 = d->n4 > 0;
    dv.omega = db + o_om;
    dv.D = db + o_D;
    dv.a = db + o_a;
    dv.T3 = db + o_T3;
    dv.T4 = db + o_T4;
    dv.T3f = reinterpret_cast<const float *>(b + o_T3f);
    dv.T4f = reinterpret_cast<const float *>(b + o_T4f);
    dv.P4 = P4;
    dv.T3p = reinterpret_cast<const float *>(b + o_T3p);
    dv.T4p = reinterpret_cast<const float *>(b + o_T4p);
    dv.omega_f = reinterpret_cast<const float *>(b + o_diagf);
    dv.D_f = dv.omega_f + 64;
    dv.a_f = dv.omega_f + 128;
    *out = h;
    ok();
    return SCIVR_OK;
}

int scivr_destroy_pes(scivr_pes pes)
{
    if (!pes) { ok(); return SCIVR_OK; }
    cudaError_t e = cudaDeviceSynchronize();
    cudaError_t e2 = cudaFree(pes->blob);
    if (pes->mlp_blob) {
        cudaError_t e3 = cudaFree(pes->mlp_blob);
        if (e2 == cudaSuccess) e2 = e3;
    }
    delete pes;
    if (e != cudaSuccess) return cuda_fail(e, "scivr_destroy_pes: synchronize");
    if (e2 != cudaSuccess) return cuda_fail(e2, "scivr_destroy_pes: cudaFree");
    ok();
    return SCIVR_OK;
}

int scivr_sample_initial(scivr_pes pes, const double *gamma, const double *p_eq, const double *q_eq,
                         int64_t n_traj, uint64_t seed, double *p0, double *q0, double *w, void *stream)
{
    if (!pes) return fail(SCIVR_EINVAL, "scivr_sample_initial: NULL potential");
    const int F = pes->dev.F;
    if (!gamma || !p_eq || !q_eq || !p0 || !q0 || !w) return fail(SCIVR_EINVAL, "scivr_sample_initial: NULL pointer");
    if (n_traj < 1) return fail(SCIVR_EINVAL, "scivr_sample_initial: n_traj=%lld < 1", (long long)n_traj);
    if (!all_positive_finite(gamma, F)) return fail(SCIVR_EINVAL, "scivr_sample_initial: gamma must be positive");
    if (!all_finite(p_eq, F) || !all_finite(q_eq, F)) return fail(SCIVR_EINVAL, "scivr_sample_initial: chi not finite");
    int nl = 0;
    cudaError_t e = launch_sample(F, gamma, p_eq, q_eq, n_traj, seed, p0, q0, w,
                                  static_cast<cudaStream_t>(stream), &nl);
    g_launches += nl;
    if (e != cudaSuccess) return cuda_fail(e, "scivr_sample_initial: launch");
    ok();
    return SCIVR_OK;
}

int scivr_propagate(scivr_pes pes, const scivr_prop_params *prm, int64_t n_traj, const double *p0,
                    const double *q0, void *amp, int64_t amp_ld, uint8_t *good,
                    const scivr_final_state *fin, void *stream)
{
    PropLaunch L{};
    const int rc = prepare_propagate(pes, prm, n_traj, p0, q0, amp, amp_ld, good, fin, &L);
    if (rc != SCIVR_OK) return rc;
    int nl = 0;
    cudaError_t e;
    if (pes->dev.mlp.H != 0) {
        if (prm->precision != SCIVR_MIXED || prm->kernel != SCIVR_KERNEL_AUTO)
            return fail(SCIVR_EUNSUPPORTED, "scivr_propagate: a learned residual needs SCIVR_MIXED and SCIVR_KERNEL_AUTO");
        e = launch_propagate_mlp(L, static_cast<cudaStream_t>(stream), &nl);
    } else {
        e = launch_propagate(L, static_cast<cudaStream_t>(stream), &nl);
    }
    g_launches += nl;
    if (e != cudaSuccess) return cuda_fail(e, "scivr_propagate: launch");
    ok();
    return SCIVR_OK;
}

int scivr_spectrum(const void *amp, int64_t amp_ld, int32_t amp_prec, const double *w,
                   const uint8_t *good, int64_t n_traj, int32_t n_steps, double dt, double E_min,
                   double E_max, int32_t n_E, int32_t ft_mode, double *I_out, int64_t *n_good_out,
                   void *stream)
{
    {
        const int rc = check_spectrum_args(amp, amp_ld, amp_prec, w, good, n_traj, n_steps, dt, E_min, E_max, n_E,
                                           ft_mode, I_out, "scivr_spectrum");
        if (rc != SCIVR_OK) return rc;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (ft_mode == SCIVR_FT_CZT64) {
        const size_t cb = spectrum_czt_scratch_bytes(n_traj, n_steps, n_E);
        void *scr = nullptr;
        cudaError_t e = cudaMallocAsync(&scr, cb, s);
        if (e != cudaSuccess) return cuda_fail(e, "scivr_spectrum: cudaMallocAsync");
        int nl = 0;
        e = launch_spectrum_czt(AmpRef{amp, amp_prec == SCIVR_MIXED}, amp_ld, w, good, n_traj, n_steps, dt, E_min,
                                E_max, n_E, I_out, n_good_out, scr, s, &nl);
        g_launches += nl;
        cudaError_t e2 = cudaFreeAsync(scr, s);
        if (e != cudaSuccess) return cuda_fail(e, "scivr_spectrum: chirp-z launch");
        if (e2 != cudaSuccess) return cuda_fail(e2, "scivr_spectrum: cudaFreeAsync");
        ok();
        return SCIVR_OK;
    }
    if (ft_mode != SCIVR_FT_FP64) {
        const size_t tb = spectrum_tc_scratch_bytes(ft_mode, n_traj, n_steps, n_E);
        void *scr = nullptr;
        cudaError_t e = cudaMallocAsync(&scr, tb, s);
        if (e != cudaSuccess) return cuda_fail(e, "scivr_spectrum: cudaMallocAsync");
        int nl = 0;
        e = launch_spectrum_tc(ft_mode, AmpRef{amp, amp_prec == SCIVR_MIXED}, amp_ld, w, good, n_traj, n_steps,
                               dt, E_min, E_max, n_E, I_out, n_good_out, scr, s, &nl);
        g_launches += nl;
        cudaError_t e2 = cudaFreeAsync(scr, s);
        if (e != cudaSuccess) return cuda_fail(e, "scivr_spectrum: tensor-core launch");
        if (e2 != cudaSuccess) return cuda_fail(e2, "scivr_spectrum: cudaFreeAsync");
        ok();
        return SCIVR_OK;
    }
    const size_t bytes = spectrum_fp64_scratch_bytes(n_traj, n_steps, n_E);
    void *scratch = nullptr;
    cudaError_t e = cudaMallocAsync(&scratch, bytes, s);
    if (e != cudaSuccess) return cuda_fail(e, "scivr_spectrum: cudaMallocAsync");
    int nl = 0;
    e = launch_spectrum_fp64(AmpRef{amp, amp_prec == SCIVR_MIXED}, amp_ld, w, good, n_traj, n_steps, dt,
                             E_min, E_max, n_E, I_out, n_good_out, scratch, s, &nl);
    g_launches += nl;
    cudaError_t e2 = cudaFreeAsync(scratch, s);
    if (e != cudaSuccess) return cuda_fail(e, "scivr_spectrum: launch");
    if (e2 != cudaSuccess) return cuda_fail(e2, "scivr_spectrum: cudaFreeAsync");
    ok();
    return SCIVR_OK;
}

int scivr_spectrum_hk(const void *amp, int64_t amp_ld, const uint8_t *good, int64_t n_traj, int32_t n_steps,
                      double dt, double E_min, double E_max, int32_t n_E, double *I_out, void *C_out,
                      int64_t *n_good_out, void *stream)
{
    // same argument rules as scivr_spectrum (weights are not used: the summands carry them)
    const double one = 1.0;
    int rc = check_spectrum_args(amp, amp_ld, SCIVR_FP64, &one, good, n_traj, n_steps, dt, E_min, E_max, n_E,
                                 SCIVR_FT_FP64, I_out, "scivr_spectrum_hk");
    if (rc != SCIVR_OK) return rc;
    if (C_out && reinterpret_cast<uintptr_t>(C_out) % 16 != 0)
        return fail(SCIVR_EINVAL, "scivr_spectrum_hk: C_out not 16-byte aligned");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void *scratch = nullptr;
    cudaError_t e = cudaMallocAsync(&scratch, spectrum_hk_scratch_bytes(n_traj, n_steps), s);
    if (e != cudaSuccess) return cuda_fail(e, "scivr_spectrum_hk: cudaMallocAsync");
    int nl = 0;
    e = launch_spectrum_hk(static_cast<const double2 *>(amp), amp_ld, good, n_traj, n_steps, dt, E_min, E_max, n_E,
                           I_out, static_cast<double2 *>(C_out), n_good_out, scratch, s, &nl);
    g_launches += nl;
    cudaError_t e2 = cudaFreeAsync(scratch, s);
    if (e != cudaSuccess) return cuda_fail(e, "scivr_spectrum_hk: launch");
    if (e2 != cudaSuccess) return cuda_fail(e2, "scivr_spectrum_hk: cudaFreeAsync");
    ok();
    return SCIVR_OK;
}

int scivr_check_status(void *stream)
{
    cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "scivr_check_status: synchronize");
    int st = 0, st_mlp = 0;
    e = read_and_clear_status(&st);
    if (e == cudaSuccess) e = read_and_clear_status_mlp(&st_mlp);
    if (e != cudaSuccess) return cuda_fail(e, "scivr_check_status: status word");
    if (st == 0) st = st_mlp;
    if (st == SCIVR_ETIMEOUT) return fail(SCIVR_ETIMEOUT, "scivr_check_status: a bounded device wait expired");
    if (st != 0) return fail(SCIVR_ECUDA, "scivr_check_status: device status %d", st);
    ok();
    return SCIVR_OK;
}

int scivr_selftest_wait_timeout(double seconds, void *stream)
{
    if (!(seconds > 0.0) || seconds > 10.0)
        return fail(SCIVR_EINVAL, "scivr_selftest_wait_timeout: seconds must lie in (0, 10]");
    cudaError_t e = launch_wait_selftest(seconds, static_cast<cudaStream_t>(stream));
    g_launches += 1;
    if (e != cudaSuccess) return cuda_fail(e, "scivr_selftest_wait_timeout: launch");
    ok();
    return SCIVR_OK;
}

int scivr_spectrum_noalloc(const void *amp, int64_t amp_ld, int32_t amp_prec, const double *w,
                           const uint8_t *good, int64_t n_traj, int32_t n_steps, double dt,
                           double E_min, double E_max, int32_t n_E, int32_t ft_mode, double *I_out,
                           int64_t *n_good_out, void *stream)
{
    if (!amp || !w || !good || !I_out) return fail(SCIVR_EINVAL, "scivr_spectrum_noalloc: NULL device pointer");
    if (n_traj < 1) return fail(SCIVR_EINVAL, "scivr_spectrum_noalloc: n_traj=%lld < 1", (long long)n_traj);
    if (n_steps < 1) return fail(SCIVR_EINVAL, "scivr_spectrum_noalloc: n_steps=%d < 1", n_steps);
    if (n_E < 2) return fail(SCIVR_EINVAL, "scivr_spectrum_noalloc: n_E=%d < 2", n_E);
    if (n_E > spectrum_noalloc_max_energies())
        return fail(SCIVR_EINVAL, "scivr_spectrum_noalloc: n_E=%d exceeds the fixed scratch limit of %d energies",
                    n_E, spectrum_noalloc_max_energies());
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(SCIVR_EINVAL, "scivr_spectrum_noalloc: dt must be positive");
    if (!std::isfinite(E_min) || !std::isfinite(E_max) || !(E_max > E_min))
        return fail(SCIVR_EINVAL, "scivr_spectrum_noalloc: need finite E_min < E_max");
    if (amp_ld < (int64_t)n_steps + 1) return fail(SCIVR_EINVAL, "scivr_spectrum_noalloc: amp_ld < n_steps+1");
    if (amp_prec != SCIVR_FP64 && amp_prec != SCIVR_MIXED)
        return fail(SCIVR_EINVAL, "scivr_spectrum_noalloc: amp_prec %d invalid", amp_prec);
    if (reinterpret_cast<uintptr_t>(amp) % (amp_prec == SCIVR_MIXED ? 8 : 16) != 0)
        return fail(SCIVR_EINVAL, "scivr_spectrum_noalloc: amp not aligned to its element (16 bytes, 8 for FP32)");
    if (ft_mode != SCIVR_FT_FP64)
        return fail(SCIVR_EUNSUPPORTED, "scivr_spectrum_noalloc: ft_mode %d not supported", ft_mode);
    int nl = 0;
    cudaError_t e = launch_spectrum_noalloc(AmpRef{amp, amp_prec == SCIVR_MIXED}, amp_ld, w, good, n_traj,
                                            n_steps, dt, E_min, E_max, n_E, I_out, n_good_out,
                                            static_cast<cudaStream_t>(stream), &nl);
    g_launches += nl;
    if (e != cudaSuccess) return cuda_fail(e, "scivr_spectrum_noalloc");
    ok();
    return SCIVR_OK;
}

}  // extern "C"
