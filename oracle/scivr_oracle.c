/*
 * scivr_oracle.c -- plain, slow FP64 CPU oracle for TA-SC-IVR power spectra.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library or its CUDA kernels may
 * call, link or include this file; only the tests, the package's smoke check
 * and the benchmark's CPU-baseline leg use it.  It shares no code, header,
 * table or constant generator with the GPU path.
 *
 * What it computes, step by step, in the paper's order and notation
 * (Tamascelli, Dambrosio, Conte, Ceotto, "GPU accelerated SC-IVR molecular
 * dynamics", arXiv:1312.4698):
 *
 *   1. Potential V(q), gradient and Hessian of a Morse (or harmonic) diagonal
 *      plus cubic and quartic coupling monomials (Sec. IV; analytic forms).
 *   2. Husimi sampling of (p0, q0) around chi = |p_eq, q_eq> and the weights
 *      w_j (Sec. III.A, after Eq. I(E)_discreto).
 *   3. Fourth-order symplectic propagation of (p, q), the action S and the
 *      2F x 2F monodromy matrix M = d(p_t, q_t)/d(p_0, q_0) (Sec. II, Eq.
 *      prefactor; Sec. III.A).  Integrator: Yoshida's triple-jump composition
 *      of exact drift and kick sub-flows (the paper only says "fourth order
 *      symplectic"; this is the reading used throughout).
 *   4. Stability monitor: bad once |det(M^T M) - 1| > tol (Sec. II and III.A).
 *   5. Herman-Kluk prefactor matrix A (Eq. prefactor), its complex
 *      determinant and the continuous phase phi_t = arg(det A)/2 (Eq.
 *      sep_approx and the phase definition just before it).
 *   6. Coherent-state overlap <chi|p_t, q_t> (Eq. coherent_state) and the
 *      amplitude a(c) = <chi|p_c q_c> exp(i (S_c + phi_c)) (Eq. I(E)_discreto).
 *   7. The discrete time-averaged spectrum, Eq. I(E)_discreto, as a direct
 *      O(K * N_E) Fourier sum per good trajectory.
 *   8. The plain Herman-Kluk SC-IVR spectrum, Eq. I(E)_SCIVR: each trajectory's
 *      summand C_t e^{iS_t} <chi|p_t q_t> <p0 q0|chi> times the importance weight
 *      of the density the initial conditions were drawn from, their mean over
 *      trajectories, and the Fourier transform folded onto t >= 0.
 *
 * Every number is IEEE double; transcendental functions come from libm.
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_TWO_PI 6.283185307179586476925286766559
#define OR_PI 3.141592653589793238462643383280

/* ------------------------------------------------------------------------ */
/* Potential: V(q) = sum_i diag_i(q_i) + sum_m c3_m q_i q_j q_k + sum_m c4_m q_i q_j q_k q_l */
/* ------------------------------------------------------------------------ */

/* Optional learned residual: a multilayer perceptron on x_i = s_in_i q_i,
 * z1 = W1 x + b1, a_l = silu(z_l), z_{l+1} = W_{l+1} a_l + b_{l+1} (l = 1, 2),
 * y = w4 . a3 + b4, V_mlp = s_out y.  W1: [H][F], W2, W3: [H][H], row-major. */
typedef struct {
    int32_t H;                /* hidden width */
    const double *s_in;       /* [F] */
    double s_out;
    const double *W1, *b1, *W2, *b2, *W3, *b3, *w4;
    double b4;
} or_mlp;

typedef struct {
    int32_t F;
    int32_t diag_kind;        /* 0: harmonic omega^2 q^2 / 2, 1: Morse D (1 - e^{-a q})^2 */
    const double *omega;      /* [F] */
    const double *D;          /* [F] */
    const double *a;          /* [F] */
    int32_t n3;
    const int32_t *idx3;      /* [n3 * 3] */
    const double *c3;         /* [n3] */
    int32_t n4;
    const int32_t *idx4;      /* [n4 * 4] */
    const double *c4;         /* [n4] */
    const or_mlp *mlp;        /* NULL: no learned residual */
    const struct or_cart_s *cart;   /* non-NULL: a Cartesian triatomic surface in its normal modes (F = 3) */
} or_pes;

/* ------------------------------------------------------------------------ */
/* Cartesian triatomic surface and its normal modes (Sec. III.A: the molecular */
/* surfaces are functions of Cartesian coordinates; the host driver builds the */
/* normal modes from the mass-weighted Hessian at the equilibrium geometry and */
/* converts between the two sets of coordinates).                             */
/* ------------------------------------------------------------------------ */

/* Atoms 0 and 2 bonded to the central atom 1.  V(x) = sum_b D_b (1 - e^{-a_b (r_b - re_b)})^2
 * + k/2 (cos theta - cos theta_e)^2, r_0 = |x0 - x1|, r_1 = |x2 - x1|, theta the angle 0-1-2.
 * x_eq, Lm fill the normal-mode map x = x_eq + Lm q (Lm[i][m] = L[i][m] / sqrt(mass of the
 * atom of coordinate i), L the orthonormal mass-weighted eigenvectors). */
typedef struct or_cart_s {
    double mass[3];
    double D[2], a[2], re[2];
    double k_bend, theta_e;
    double x_eq[9];
    double Lm[27];            /* [9][3] */
} or_cart;

/* V, gradient [9] and Hessian [9][9] of the Cartesian surface.  Derivatives written from
 * the dot products s = u.v, P = (u.u)(v.v) (u = x0 - x1, v = x2 - x1, cos theta = s P^{-1/2})
 * and r = (w.w)^{1/2} for each bond vector w: every intermediate is a polynomial in x or a
 * power of one, differentiated by the product and chain rules. */
double or_cart_eval(const or_cart *c, const double *x, double *g, double *H)
{
    double V = 0.0;
    if (g) memset(g, 0, 9 * sizeof(double));
    if (H) memset(H, 0, 81 * sizeof(double));
    /* bonds: atom pair (0, 1) and (2, 1) */
    for (int b = 0; b < 2; ++b) {
        const int ia = b == 0 ? 0 : 2, ib = 1;
        double w[3], ww = 0.0;
        for (int d = 0; d < 3; ++d) { w[d] = x[3 * ia + d] - x[3 * ib + d]; ww += w[d] * w[d]; }
        const double r = sqrt(ww);
        const double e = exp(-c->a[b] * (r - c->re[b]));
        V += c->D[b] * (1.0 - e) * (1.0 - e);
        const double f1 = 2.0 * c->D[b] * c->a[b] * e * (1.0 - e);                  /* dV/dr */
        const double f2 = 2.0 * c->D[b] * c->a[b] * c->a[b] * e * (2.0 * e - 1.0);  /* d2V/dr2 */
        /* dr/dw = w / r ; d2r/dw dw^T = (I - w w^T / r^2) / r */
        for (int d = 0; d < 3; ++d) {
            const double gd = f1 * w[d] / r;
            if (g) { g[3 * ia + d] += gd; g[3 * ib + d] -= gd; }
        }
        if (H)
            for (int d = 0; d < 3; ++d)
                for (int f = 0; f < 3; ++f) {
                    const double hw = f2 * w[d] * w[f] / ww + f1 * ((d == f ? 1.0 : 0.0) - w[d] * w[f] / ww) / r;
                    H[(3 * ia + d) * 9 + 3 * ia + f] += hw;
                    H[(3 * ib + d) * 9 + 3 * ib + f] += hw;
                    H[(3 * ia + d) * 9 + 3 * ib + f] -= hw;
                    H[(3 * ib + d) * 9 + 3 * ia + f] -= hw;
                }
    }
    /* bend: y = (u, v) in R^6, cos = s P^{-1/2} */
    {
        double y[6];
        for (int d = 0; d < 3; ++d) { y[d] = x[d] - x[3 + d]; y[3 + d] = x[6 + d] - x[3 + d]; }
        const double *u = y, *v = y + 3;
        double uu = 0.0, vv = 0.0, s = 0.0;
        for (int d = 0; d < 3; ++d) { uu += u[d] * u[d]; vv += v[d] * v[d]; s += u[d] * v[d]; }
        const double P = uu * vv;
        const double Pm12 = 1.0 / sqrt(P);
        const double cth = s * Pm12;
        const double dc = cth - cos(c->theta_e);
        V += 0.5 * c->k_bend * dc * dc;
        /* ds/dy = (v, u); dP/dy = (2 u vv, 2 v uu) */
        double ds[6], dP[6];
        for (int d = 0; d < 3; ++d) {
            ds[d] = v[d]; ds[3 + d] = u[d];
            dP[d] = 2.0 * u[d] * vv; dP[3 + d] = 2.0 * v[d] * uu;
        }
        /* dcos = ds P^{-1/2} - (1/2) s P^{-3/2} dP */
        double dcy[6];
        for (int i = 0; i < 6; ++i) dcy[i] = ds[i] * Pm12 - 0.5 * s * Pm12 * Pm12 * Pm12 * dP[i];
        double Hy[36];
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 6; ++j) {
                /* d2s: 1 where one index is in u and the other the same component in v */
                const double d2s = (i % 3 == j % 3 && (i < 3) != (j < 3)) ? 1.0 : 0.0;
                /* d2P: d/dy_j of (2 u vv, 2 v uu) */
                double d2P;
                if (i < 3 && j < 3) d2P = (i == j ? 2.0 * vv : 0.0);
                else if (i >= 3 && j >= 3) d2P = (i == j ? 2.0 * uu : 0.0);
                else if (i < 3) d2P = 4.0 * u[i] * v[j - 3];
                else d2P = 4.0 * v[i - 3] * u[j];
                const double P32 = Pm12 * Pm12 * Pm12, P52 = P32 * Pm12 * Pm12;
                const double d2c = d2s * Pm12 - 0.5 * P32 * (ds[i] * dP[j] + ds[j] * dP[i])
                                   - 0.5 * s * P32 * d2P + 0.75 * s * P52 * dP[i] * dP[j];
                Hy[i * 6 + j] = c->k_bend * (dcy[i] * dcy[j] + dc * d2c);
            }
        /* y = (x0 - x1, x2 - x1): dy/dx maps atom 0 -> u, atom 2 -> v, atom 1 -> -(u + v) */
        for (int i = 0; i < 6; ++i) {
            const double gi = c->k_bend * dc * dcy[i];
            const int atom = i < 3 ? 0 : 2, d = i % 3;
            if (g) { g[3 * atom + d] += gi; g[3 + d] -= gi; }
        }
        if (H)
            for (int i = 0; i < 6; ++i)
                for (int j = 0; j < 6; ++j) {
                    const int ai = i < 3 ? 0 : 2, di = i % 3, aj = j < 3 ? 0 : 2, dj = j % 3;
                    const double h = Hy[i * 6 + j];
                    H[(3 * ai + di) * 9 + 3 * aj + dj] += h;
                    H[(3 * ai + di) * 9 + 3 + dj] -= h;
                    H[(3 + di) * 9 + 3 * aj + dj] -= h;
                    H[(3 + di) * 9 + 3 + dj] += h;
                }
    }
    return V;
}

/* Equilibrium geometry (atom 1 at the origin, the molecule in the xy plane, the
 * bisector along y) and the normal modes: the eigenvectors of the mass-weighted
 * Hessian M^{-1/2} H M^{-1/2} by cyclic Jacobi rotations; the three largest
 * eigenvalues are omega^2 of the vibrations (the other six, translations and
 * rotations, vanish at the equilibrium).  Modes in increasing frequency; each
 * eigenvector's sign makes its first component of magnitude above 1e-3 positive.
 * Fills c->x_eq, c->Lm, omega[3]; returns the largest |eigenvalue| among the six
 * rigid-body modes (zero up to rounding). */
double or_normal_modes(or_cart *c, double *omega)
{
    const double h = 0.5 * c->theta_e;
    memset(c->x_eq, 0, sizeof(c->x_eq));
    c->x_eq[0] = -c->re[0] * sin(h); c->x_eq[1] = c->re[0] * cos(h);
    c->x_eq[6] = c->re[1] * sin(h);  c->x_eq[7] = c->re[1] * cos(h);
    double Hx[81], A[81], Vm[81];
    or_cart_eval(c, c->x_eq, NULL, Hx);
    for (int i = 0; i < 9; ++i)
        for (int j = 0; j < 9; ++j) {
            A[i * 9 + j] = Hx[i * 9 + j] / sqrt(c->mass[i / 3] * c->mass[j / 3]);
            Vm[i * 9 + j] = i == j ? 1.0 : 0.0;
        }
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < 9; ++i)
            for (int j = 0; j < 9; ++j) {
                tot += A[i * 9 + j] * A[i * 9 + j];
                if (i != j) off += A[i * 9 + j] * A[i * 9 + j];
            }
        if (off <= 1e-30 * tot) break;
        for (int p = 0; p < 8; ++p)
            for (int q = p + 1; q < 9; ++q) {
                const double apq = A[p * 9 + q];
                if (apq == 0.0) continue;
                /* rotation that zeroes A[p][q]: tan(2 phi) = 2 apq / (aqq - app) */
                const double theta = (A[q * 9 + q] - A[p * 9 + p]) / (2.0 * apq);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
                for (int k = 0; k < 9; ++k) {
                    const double akp = A[k * 9 + p], akq = A[k * 9 + q];
                    A[k * 9 + p] = cs * akp - sn * akq;
                    A[k * 9 + q] = sn * akp + cs * akq;
                }
                for (int k = 0; k < 9; ++k) {
                    const double apk = A[p * 9 + k], aqk = A[q * 9 + k];
                    A[p * 9 + k] = cs * apk - sn * aqk;
                    A[q * 9 + k] = sn * apk + cs * aqk;
                }
                for (int k = 0; k < 9; ++k) {
                    const double vkp = Vm[k * 9 + p], vkq = Vm[k * 9 + q];
                    Vm[k * 9 + p] = cs * vkp - sn * vkq;
                    Vm[k * 9 + q] = sn * vkp + cs * vkq;
                }
            }
    }
    /* order by eigenvalue: the three largest are the vibrations */
    int idx[9];
    for (int i = 0; i < 9; ++i) idx[i] = i;
    for (int i = 0; i < 9; ++i)
        for (int j = i + 1; j < 9; ++j)
            if (A[idx[j] * 9 + idx[j]] < A[idx[i] * 9 + idx[i]]) { int t = idx[i]; idx[i] = idx[j]; idx[j] = t; }
    double rigid = 0.0;
    for (int i = 0; i < 6; ++i) rigid = fmax(rigid, fabs(A[idx[i] * 9 + idx[i]]));
    for (int m = 0; m < 3; ++m) {
        const int col = idx[6 + m];
        omega[m] = sqrt(A[col * 9 + col]);
        double sgn = 1.0;
        for (int i = 0; i < 9; ++i)
            if (fabs(Vm[i * 9 + col]) > 1e-3) { sgn = Vm[i * 9 + col] > 0.0 ? 1.0 : -1.0; break; }
        for (int i = 0; i < 9; ++i) c->Lm[i * 3 + m] = sgn * Vm[i * 9 + col] / sqrt(c->mass[i / 3]);
    }
    return rigid;
}


static double or_sigmoid(double z) { return 1.0 / (1.0 + exp(-z)); }

/* silu(z) = z sigma(z) and its first two derivatives. */
static void or_silu(double z, double *f, double *f1, double *f2)
{
    double s = or_sigmoid(z);
    *f = z * s;
    *f1 = s * (1.0 + z * (1.0 - s));
    *f2 = s * (1.0 - s) * (2.0 + z * (1.0 - 2.0 * s));
}

/* V_mlp(q), its gradient (added into g) and Hessian (added into H).
 * The Hessian of a chain of affine maps and elementwise activations is
 * sum_l J_l^T diag(abar_l * silu''(z_l)) J_l with J_l = dz_l/dx and
 * abar_l = dy/da_l (second-order chain rule, written layer by layer). */
void or_mlp_eval(const or_mlp *m, int F, const double *q, double *V, double *g, double *Hm)
{
    const int Hd = m->H;
    double *x = malloc(sizeof(double) * F);
    double *z[3], *a[3], *d1[3], *d2[3], *abar[3], *J[3];
    for (int l = 0; l < 3; ++l) {
        z[l] = malloc(sizeof(double) * Hd); a[l] = malloc(sizeof(double) * Hd);
        d1[l] = malloc(sizeof(double) * Hd); d2[l] = malloc(sizeof(double) * Hd);
        abar[l] = malloc(sizeof(double) * Hd); J[l] = malloc(sizeof(double) * Hd * F);
    }
    const double *W[3] = {m->W1, m->W2, m->W3}, *b[3] = {m->b1, m->b2, m->b3};
    for (int i = 0; i < F; ++i) x[i] = m->s_in[i] * q[i];
    for (int l = 0; l < 3; ++l) {
        const int nin = l == 0 ? F : Hd;
        const double *in = l == 0 ? x : a[l - 1];
        for (int o = 0; o < Hd; ++o) {
            double acc = b[l][o];
            for (int i = 0; i < nin; ++i) acc += W[l][o * nin + i] * in[i];
            z[l][o] = acc;
            or_silu(acc, &a[l][o], &d1[l][o], &d2[l][o]);
        }
    }
    double y = m->b4;
    for (int o = 0; o < Hd; ++o) y += m->w4[o] * a[2][o];
    *V += m->s_out * y;
    /* backward: abar_3 = w4, abar_l = W_{l+1}^T (abar_{l+1} * silu'(z_{l+1})) */
    for (int o = 0; o < Hd; ++o) abar[2][o] = m->w4[o];
    for (int l = 1; l >= 0; --l)
        for (int i = 0; i < Hd; ++i) {
            double acc = 0.0;
            for (int o = 0; o < Hd; ++o) acc += W[l + 1][o * Hd + i] * abar[l + 1][o] * d1[l + 1][o];
            abar[l][i] = acc;
        }
    if (g) {
        for (int i = 0; i < F; ++i) {
            double acc = 0.0;
            for (int o = 0; o < Hd; ++o) acc += m->W1[o * F + i] * abar[0][o] * d1[0][o];
            g[i] += m->s_out * m->s_in[i] * acc;
        }
    }
    if (Hm) {
        /* J_1 = W1, J_{l+1} = W_{l+1} diag(silu'(z_l)) J_l */
        for (int o = 0; o < Hd; ++o)
            for (int k = 0; k < F; ++k) J[0][o * F + k] = m->W1[o * F + k];
        for (int l = 1; l < 3; ++l)
            for (int o = 0; o < Hd; ++o)
                for (int k = 0; k < F; ++k) {
                    double acc = 0.0;
                    for (int i = 0; i < Hd; ++i) acc += W[l][o * Hd + i] * d1[l - 1][i] * J[l - 1][i * F + k];
                    J[l][o * F + k] = acc;
                }
        for (int k = 0; k < F; ++k)
            for (int kk = 0; kk < F; ++kk) {
                double acc = 0.0;
                for (int l = 0; l < 3; ++l)
                    for (int o = 0; o < Hd; ++o) acc += abar[l][o] * d2[l][o] * J[l][o * F + k] * J[l][o * F + kk];
                Hm[k * F + kk] += m->s_out * m->s_in[k] * m->s_in[kk] * acc;
            }
    }
    free(x);
    for (int l = 0; l < 3; ++l) { free(z[l]); free(a[l]); free(d1[l]); free(d2[l]); free(abar[l]); free(J[l]); }
}

/* One monomial c * prod_s q[idx[s]] and its derivatives by the product rule
 * over index positions (repeated indices are handled automatically). */
static void or_monomial(int deg, const int32_t *idx, double c, const double *q, int F,
                        double *V, double *g, double *H)
{
    double v = c;
    for (int s = 0; s < deg; ++s) v *= q[idx[s]];
    *V += v;
    if (g) {
        for (int s = 0; s < deg; ++s) {
            double prod = c;
            for (int t = 0; t < deg; ++t)
                if (t != s) prod *= q[idx[t]];
            g[idx[s]] += prod;
        }
    }
    if (H) {
        for (int s = 0; s < deg; ++s)
            for (int t = 0; t < deg; ++t) {
                if (t == s) continue;
                double prod = c;
                for (int u = 0; u < deg; ++u)
                    if (u != s && u != t) prod *= q[idx[u]];
                H[idx[s] * F + idx[t]] += prod;
            }
    }
}

/* V(q); if g != NULL also the gradient [F]; if H != NULL also the Hessian [F*F] row-major. */
double or_pes_eval(const or_pes *pes, const double *q, double *g, double *H)
{
    const int F = pes->F;
    double V = 0.0;
    if (g) memset(g, 0, sizeof(double) * F);
    if (H) memset(H, 0, sizeof(double) * F * F);
    if (pes->cart) {
        /* V(q) = V_cart(x_eq + Lm q): g = Lm^T grad_x V, H = Lm^T H_x Lm (F = 3) */
        const or_cart *c = pes->cart;
        double x[9], gx[9], Hx[81];
        for (int i = 0; i < 9; ++i) {
            x[i] = c->x_eq[i];
            for (int m = 0; m < 3; ++m) x[i] += c->Lm[i * 3 + m] * q[m];
        }
        V = or_cart_eval(c, x, gx, Hx);
        for (int m = 0; m < 3; ++m) {
            if (g) {
                g[m] = 0.0;
                for (int i = 0; i < 9; ++i) g[m] += c->Lm[i * 3 + m] * gx[i];
            }
            if (H)
                for (int n = 0; n < 3; ++n) {
                    double acc = 0.0;
                    for (int i = 0; i < 9; ++i)
                        for (int j = 0; j < 9; ++j) acc += c->Lm[i * 3 + m] * Hx[i * 9 + j] * c->Lm[j * 3 + n];
                    H[m * 3 + n] = acc;
                }
        }
        return V;
    }
    for (int i = 0; i < F; ++i) {
        if (pes->diag_kind == 0) {
            double w2 = pes->omega[i] * pes->omega[i];
            V += 0.5 * w2 * q[i] * q[i];
            if (g) g[i] += w2 * q[i];
            if (H) H[i * F + i] += w2;
        } else {
            double Dm = pes->D[i], am = pes->a[i];
            double u = exp(-am * q[i]);
            V += Dm * (1.0 - u) * (1.0 - u);
            if (g) g[i] += 2.0 * Dm * am * u * (1.0 - u);
            if (H) H[i * F + i] += 2.0 * Dm * am * am * u * (2.0 * u - 1.0);
        }
    }
    for (int m = 0; m < pes->n3; ++m) or_monomial(3, pes->idx3 + 3 * m, pes->c3[m], q, F, &V, g, H);
    for (int m = 0; m < pes->n4; ++m) or_monomial(4, pes->idx4 + 4 * m, pes->c4[m], q, F, &V, g, H);
    if (pes->mlp) or_mlp_eval(pes->mlp, F, q, &V, g, H);
    return V;
}

/* ------------------------------------------------------------------------ */
/* Determinants by LU with partial pivoting (textbook Doolittle elimination) */
/* ------------------------------------------------------------------------ */

/* det of an n x n real matrix (row-major); A is destroyed. */
double or_det_real(int n, double *A)
{
    double det = 1.0;
    for (int k = 0; k < n; ++k) {
        int piv = k;
        double best = fabs(A[k * n + k]);
        for (int i = k + 1; i < n; ++i)
            if (fabs(A[i * n + k]) > best) { best = fabs(A[i * n + k]); piv = i; }
        if (piv != k) {
            for (int j = 0; j < n; ++j) {
                double t = A[k * n + j]; A[k * n + j] = A[piv * n + j]; A[piv * n + j] = t;
            }
            det = -det;
        }
        double akk = A[k * n + k];
        det *= akk;
        if (akk == 0.0) return 0.0;
        for (int i = k + 1; i < n; ++i) {
            double l = A[i * n + k] / akk;
            for (int j = k + 1; j < n; ++j) A[i * n + j] -= l * A[k * n + j];
        }
    }
    return det;
}

/* det of an n x n complex matrix (row-major); A is destroyed. */
double complex or_det_complex(int n, double complex *A)
{
    double complex det = 1.0;
    for (int k = 0; k < n; ++k) {
        int piv = k;
        double best = cabs(A[k * n + k]);
        for (int i = k + 1; i < n; ++i)
            if (cabs(A[i * n + k]) > best) { best = cabs(A[i * n + k]); piv = i; }
        if (piv != k) {
            for (int j = 0; j < n; ++j) {
                double complex t = A[k * n + j]; A[k * n + j] = A[piv * n + j]; A[piv * n + j] = t;
            }
            det = -det;
        }
        double complex akk = A[k * n + k];
        det *= akk;
        if (akk == 0.0) return 0.0;
        for (int i = k + 1; i < n; ++i) {
            double complex l = A[i * n + k] / akk;
            for (int j = k + 1; j < n; ++j) A[i * n + j] -= l * A[k * n + j];
        }
    }
    return det;
}

/* ------------------------------------------------------------------------ */
/* Coherent states (Eq. coherent_state, normalisation (gamma_i/pi)^{1/4} per mode) */
/* ------------------------------------------------------------------------ */

/* log <p1 q1 | p2 q2> for product coherent states of widths gamma:
 * sum_i [ -gamma_i/4 (q1-q2)^2 - (p1-p2)^2/(4 gamma_i) + (i/2)(p1+p2)(q1-q2) ]. */
double complex or_log_overlap(int F, const double *gamma, const double *p1, const double *q1,
                              const double *p2, const double *q2)
{
    double re = 0.0, im = 0.0;
    for (int i = 0; i < F; ++i) {
        double dq = q1[i] - q2[i], dp = p1[i] - p2[i];
        re += -0.25 * gamma[i] * dq * dq - dp * dp / (4.0 * gamma[i]);
        im += 0.5 * (p1[i] + p2[i]) * dq;
    }
    return re + I * im;
}

/* ------------------------------------------------------------------------ */
/* Propagation of one trajectory                                             */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t F;
    int32_t n_steps;
    double dt;
    double stab_tol;
    const double *gamma;   /* [F] */
    const double *p_eq;    /* [n_chi * F] */
    const double *q_eq;    /* [n_chi * F] */
    int32_t n_chi;
    int32_t amplitude;     /* 0: time-averaged (prefactor phase only), 1: Herman-Kluk (Eq. I(E)_SCIVR) */
} or_prop;

typedef struct {
    double *p, *q;          /* [F] at T */
    double *S, *theta;      /* action and unwrapped arg det A at T */
    double *detM;           /* det M at T */
    double complex *detA;   /* det A at T */
    double *M;              /* [2F * 2F] at T, rows (p, q), columns (p0, q0) */
    double *stab;           /* max over steps of |det(M)^2 - 1| (+inf once not finite) */
} or_final;

/* Yoshida (1990) fourth-order triple jump, written as position-Verlet
 * compositions: drifts c1..c4 and kicks d1..d3 (fractions of dt). */
static void or_yoshida(double c[4], double d[3])
{
    double cbrt2 = cbrt(2.0);
    double w1 = 1.0 / (2.0 - cbrt2);
    double w0 = -cbrt2 / (2.0 - cbrt2);
    c[0] = 0.5 * w1; c[1] = 0.5 * (w0 + w1); c[2] = c[1]; c[3] = c[0];
    d[0] = w1; d[1] = w0; d[2] = w1;
}

/* Drift by tau under T = p^2/2: q += tau p, S += tau p.p/2, dq-rows of M += tau dp-rows. */
static void or_drift(int F, double tau, double *q, const double *p, double *S, double *M)
{
    const int n = 2 * F;
    double kin = 0.0;
    for (int a = 0; a < F; ++a) kin += 0.5 * p[a] * p[a];
    *S += tau * kin;
    for (int a = 0; a < F; ++a) q[a] += tau * p[a];
    for (int a = 0; a < F; ++a)
        for (int col = 0; col < n; ++col) M[(F + a) * n + col] += tau * M[a * n + col];
}

/* Kick by tau under V(q): p -= tau grad V, S -= tau V, dp-rows of M -= tau H dq-rows. */
static void or_kick(const or_pes *pes, double tau, const double *q, double *p, double *S,
                    double *M, double *g, double *H)
{
    const int F = pes->F, n = 2 * F;
    double V = or_pes_eval(pes, q, g, H);
    *S -= tau * V;
    for (int a = 0; a < F; ++a) p[a] -= tau * g[a];
    for (int a = 0; a < F; ++a)
        for (int col = 0; col < n; ++col) {
            double hm = 0.0;
            for (int b = 0; b < F; ++b) hm += H[a * F + b] * M[(F + b) * n + col];
            M[a * n + col] -= tau * hm;
        }
}

/* Herman-Kluk prefactor matrix (Eq. prefactor), in the width-symmetric form
 * A = 1/2 [ G^{1/2} Mqq G^{-1/2} + G^{-1/2} Mpp G^{1/2}
 *           - i G^{1/2} Mqp G^{1/2} + i G^{-1/2} Mpq G^{-1/2} ],  G = diag(gamma),
 * with Mqq = dq_t/dq_0, Mpp = dp_t/dp_0, Mqp = dq_t/dp_0, Mpq = dp_t/dq_0. */
static void or_prefactor_matrix(int F, const double *gamma, const double *M, double complex *A)
{
    const int n = 2 * F;
    for (int a = 0; a < F; ++a)
        for (int b = 0; b < F; ++b) {
            double ga = sqrt(gamma[a]), gb = sqrt(gamma[b]);
            double Mpp = M[a * n + b];
            double Mpq = M[a * n + F + b];
            double Mqp = M[(F + a) * n + b];
            double Mqq = M[(F + a) * n + F + b];
            double re = ga / gb * Mqq + gb / ga * Mpp;
            double im = -ga * gb * Mqp + Mpq / (ga * gb);
            A[a * F + b] = 0.5 * (re + I * im);
        }
}

/* Continuous phase of det A.  The argument is unwrapped relative to the
 * reference rotation exp(-i sum_i gamma_i t): per step, the change of
 * arg(det A) + sum_i gamma_i t is taken as its principal value. */
static double or_unwrap(double theta, double arg_old, double arg_new, double ref_step)
{
    double d = arg_new - arg_old + ref_step;
    d -= OR_TWO_PI * nearbyint(d / OR_TWO_PI);
    return theta + d - ref_step;
}

/* Propagate one trajectory from (p0, q0) and write the amplitude series
 * amp[chi * amp_chi_stride + c], c = 0..n_steps, for every reference state chi.
 * The optional series (length n_steps+1, may be NULL) record S_c, theta_c,
 * det A_c and det M_c.  Returns 1 if the trajectory stayed good, else 0. */
int or_propagate_one(const or_pes *pes, const or_prop *prm, const double *p0, const double *q0,
                     double complex *amp, int64_t amp_chi_stride, or_final *fin,
                     double *S_series, double *theta_series, double complex *detA_series,
                     double *detM_series)
{
    const int F = pes->F, n = 2 * F;
    double c[4], d[3];
    or_yoshida(c, d);

    double *p = malloc(sizeof(double) * F), *q = malloc(sizeof(double) * F);
    double *M = malloc(sizeof(double) * n * n), *Mw = malloc(sizeof(double) * n * n);
    double *g = malloc(sizeof(double) * F), *H = malloc(sizeof(double) * F * F);
    double complex *A = malloc(sizeof(double complex) * F * F);

    memcpy(p, p0, sizeof(double) * F);
    memcpy(q, q0, sizeof(double) * F);
    for (int i = 0; i < n * n; ++i) M[i] = 0.0;
    for (int i = 0; i < n; ++i) M[i * n + i] = 1.0;
    double S = 0.0, theta = 0.0, arg_old = 0.0, detM = 1.0;
    double complex detA = 1.0;
    double ref_step = 0.0;
    for (int i = 0; i < F; ++i) ref_step += prm->gamma[i] * prm->dt;
    int good = 1;
    double stab = 0.0;

    for (int step = 0; step <= prm->n_steps; ++step) {
        if (step > 0) {
            const double dt = prm->dt;
            or_drift(F, c[0] * dt, q, p, &S, M);
            or_kick(pes, d[0] * dt, q, p, &S, M, g, H);
            or_drift(F, c[1] * dt, q, p, &S, M);
            or_kick(pes, d[1] * dt, q, p, &S, M, g, H);
            or_drift(F, c[2] * dt, q, p, &S, M);
            or_kick(pes, d[2] * dt, q, p, &S, M, g, H);
            or_drift(F, c[3] * dt, q, p, &S, M);

            /* stability monitor: |det(M^T M) - 1| = |det(M)^2 - 1| */
            memcpy(Mw, M, sizeof(double) * n * n);
            detM = or_det_real(n, Mw);
            double dev = isfinite(detM) ? fabs(detM * detM - 1.0) : INFINITY;
            if (dev > stab) stab = dev;
            if (dev > prm->stab_tol) good = 0;

            /* prefactor determinant and its continuous phase */
            or_prefactor_matrix(F, prm->gamma, M, A);
            detA = or_det_complex(F, A);
            double arg_new = carg(detA);
            theta = or_unwrap(theta, arg_old, arg_new, ref_step);
            arg_old = arg_new;
            if (!isfinite(S) || !isfinite(theta)) good = 0;
            for (int i = 0; i < F; ++i)
                if (!isfinite(p[i]) || !isfinite(q[i])) good = 0;
        }
        if (S_series) S_series[step] = S;
        if (theta_series) theta_series[step] = theta;
        if (detA_series) detA_series[step] = detA;
        if (detM_series) detM_series[step] = detM;
        if (amp) {
            for (int x = 0; x < prm->n_chi; ++x) {
                double complex lo = or_log_overlap(F, prm->gamma, prm->p_eq + x * F,
                                                   prm->q_eq + x * F, p, q);
                if (prm->amplitude == 1) {
                    /* Herman-Kluk summand of Eq. I(E)_SCIVR times the importance weight
                     * of the density the initial conditions were drawn from, the Husimi
                     * density of the first reference state:
                     *   C_t e^{i S_t} <chi_x|p_t q_t> <p0 q0|chi_x> w,  w = 1 / |<p0 q0|chi_0>|^2,
                     * with C_t = |det A|^{1/2} e^{i theta/2} (Eq. prefactor on the branch
                     * that theta follows).  Every reference state shares the trajectories,
                     * so every state takes the same w (for x = 0 the summand is
                     * C_t e^{i S_t} <chi|p_t q_t> / <chi|p0 q0>). */
                    double complex lo0 = or_log_overlap(F, prm->gamma, prm->p_eq + x * F,
                                                        prm->q_eq + x * F, p0, q0);
                    double complex lo00 = x == 0 ? lo0 : or_log_overlap(F, prm->gamma, prm->p_eq,
                                                                        prm->q_eq, p0, q0);
                    double complex Ct = sqrt(cabs(detA)) * cexp(0.5 * I * theta);
                    double complex ov0 = cexp(lo0);
                    double complex ov00 = cexp(lo00);
                    double w0 = 1.0 / (creal(ov00) * creal(ov00) + cimag(ov00) * cimag(ov00));
                    amp[x * amp_chi_stride + step] = Ct * cexp(I * S) * cexp(lo) * conj(ov0) * w0;
                } else {
                    double phase = cimag(lo) + S + 0.5 * theta;
                    amp[x * amp_chi_stride + step] = exp(creal(lo)) * (cos(phase) + I * sin(phase));
                }
            }
        }
    }
    if (fin) {
        if (fin->p) memcpy(fin->p, p, sizeof(double) * F);
        if (fin->q) memcpy(fin->q, q, sizeof(double) * F);
        if (fin->S) *fin->S = S;
        if (fin->theta) *fin->theta = theta;
        if (fin->detM) *fin->detM = detM;
        if (fin->detA) *fin->detA = detA;
        if (fin->M) memcpy(fin->M, M, sizeof(double) * n * n);
        if (fin->stab) *fin->stab = stab;
    }
    free(p); free(q); free(M); free(Mw); free(g); free(H); free(A);
    return good;
}

/* Batch propagation.  p0, q0: [F][n_traj] (variable-major).  amp: complex
 * [n_chi][n_traj][amp_ld], amp_ld >= n_steps + 1.  good: [n_traj].  Optional
 * final-state arrays (may be NULL): fin_p, fin_q [n_traj][F]; fin_S, fin_theta,
 * fin_detM, fin_stab [n_traj]; fin_detA [n_traj]; fin_M [n_traj][2F][2F]. */
int or_propagate(const or_pes *pes, const or_prop *prm, int64_t n_traj, const double *p0,
                 const double *q0, double complex *amp, int64_t amp_ld, uint8_t *good,
                 double *fin_p, double *fin_q, double *fin_S, double *fin_theta, double *fin_detM,
                 double complex *fin_detA, double *fin_M, double *fin_stab, int n_threads)
{
    const int F = pes->F, n = 2 * F;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 4)
#endif
    for (int64_t j = 0; j < n_traj; ++j) {
        double p_init[64], q_init[64];
        for (int i = 0; i < F; ++i) { p_init[i] = p0[i * n_traj + j]; q_init[i] = q0[i * n_traj + j]; }
        or_final fin = {
            fin_p ? fin_p + j * F : NULL, fin_q ? fin_q + j * F : NULL,
            fin_S ? fin_S + j : NULL, fin_theta ? fin_theta + j : NULL,
            fin_detM ? fin_detM + j : NULL, fin_detA ? fin_detA + j : NULL,
            fin_M ? fin_M + j * n * n : NULL, fin_stab ? fin_stab + j : NULL };
        int ok = or_propagate_one(pes, prm, p_init, q_init, amp ? amp + j * amp_ld : NULL,
                                  n_traj * amp_ld, &fin, NULL, NULL, NULL, NULL);
        if (good) good[j] = (uint8_t)ok;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Time-averaged spectrum, Eq. I(E)_discreto                                 */
/* ------------------------------------------------------------------------ */

/* I(E_k) = dt^2 / (2 pi T n_good) sum_{j good} w_j | sum_{c=0}^{n_steps} a_j(c) e^{i E_k c dt} |^2
 * with T = n_steps dt and E_k = E_min + k (E_max - E_min)/(n_E - 1).  The
 * paper's (2 pi)^{-F} is carried by the weights (w_j = 1/|<p0 q0|chi>|^2 for
 * Husimi samples).  amp: [n_traj][amp_ld]. */
int or_spectrum(const double complex *amp, int64_t amp_ld, const double *w, const uint8_t *good,
                int64_t n_traj, int32_t n_steps, double dt, double E_min, double E_max,
                int32_t n_E, double *I_out, int64_t *n_good_out, int n_threads)
{
    int64_t n_good = 0;
    for (int64_t j = 0; j < n_traj; ++j) n_good += good[j] ? 1 : 0;
    if (n_good_out) *n_good_out = n_good;
    const double T = n_steps * dt;
    const double norm = n_good > 0 ? dt * dt / (OR_TWO_PI * T * (double)n_good) : 0.0;
    const int K = n_steps + 1;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel
#endif
    {
        double complex *tw = malloc(sizeof(double complex) * K);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int k = 0; k < n_E; ++k) {
            double E = n_E > 1 ? E_min + k * ((E_max - E_min) / (n_E - 1)) : E_min;
            for (int c = 0; c < K; ++c) {
                double ang = E * (c * dt);
                tw[c] = cos(ang) + I * sin(ang);
            }
            double acc = 0.0;
            for (int64_t j = 0; j < n_traj; ++j) {
                if (!good[j]) continue;
                double complex X = 0.0;
                const double complex *a = amp + j * amp_ld;
                for (int c = 0; c < K; ++c) X += a[c] * tw[c];
                acc += w[j] * (creal(X) * creal(X) + cimag(X) * cimag(X));
            }
            I_out[k] = norm * acc;
        }
        free(tw);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Plain Herman-Kluk SC-IVR spectrum, Eq. I(E)_SCIVR                         */
/* ------------------------------------------------------------------------ */

/* The survival amplitude <chi|e^{-iHt}|chi> at t = c dt is the Monte Carlo mean
 * of the Herman-Kluk summands (propagation with amplitude = 1, which carries
 * the weights) over the good trajectories,
 *   C(c dt) = (1/n_good) sum_{j good} amp_j(c),
 * and I(E) = (1/2pi) int_{-T}^{T} C(t) e^{i E t} dt by the rectangle rule on the
 * symmetric grid c = -n_steps..n_steps, folded onto c >= 0 with C(-t) = conj C(t):
 *   I(E_k) = (dt/pi) Re[ C(0)/2 + sum_{c=1}^{n_steps} C(c dt) e^{i E_k c dt} ]. */
int or_spectrum_hk(const double complex *amp, int64_t amp_ld, const uint8_t *good, int64_t n_traj,
                   int32_t n_steps, double dt, double E_min, double E_max, int32_t n_E, double *I_out,
                   int64_t *n_good_out, double complex *C_out)
{
    int64_t n_good = 0;
    for (int64_t j = 0; j < n_traj; ++j) n_good += good[j] ? 1 : 0;
    if (n_good_out) *n_good_out = n_good;
    const int K = n_steps + 1;
    double complex *C = malloc(sizeof(double complex) * K);
    for (int c = 0; c < K; ++c) {
        double complex acc = 0.0;
        for (int64_t j = 0; j < n_traj; ++j)
            if (good[j]) acc += amp[j * amp_ld + c];
        C[c] = n_good > 0 ? acc / (double)n_good : 0.0;
        if (C_out) C_out[c] = C[c];
    }
    for (int k = 0; k < n_E; ++k) {
        double E = n_E > 1 ? E_min + k * ((E_max - E_min) / (n_E - 1)) : E_min;
        double complex acc = 0.5 * C[0];
        for (int c = 1; c < K; ++c) {
            double ang = E * (c * dt);
            acc += C[c] * (cos(ang) + I * sin(ang));
        }
        I_out[k] = dt / OR_PI * creal(acc);
    }
    free(C);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Husimi sampling with a counter-based generator                            */
/* ------------------------------------------------------------------------ */

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the
 * 4-word Philox S-box with multipliers 0xD2511F53, 0xCD9E8D57 and key
 * schedule increments 0x9E3779B9, 0xBB67AE85. */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t prod0 = (uint64_t)0xD2511F53u * x0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * x2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Standard normal number d (0 <= d < 2F) of trajectory j: Philox block d/4
 * with counter (j_lo, j_hi, d/4, 0) and key (seed_lo, seed_hi); words (0,1)
 * and (2,3) feed two Box-Muller pairs; uniforms are (u + 1/2) 2^-32. */
static double or_normal(uint64_t seed, int64_t j, int d)
{
    uint32_t ctr[4] = { (uint32_t)j, (uint32_t)((uint64_t)j >> 32), (uint32_t)(d / 4), 0u };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t u[4];
    or_philox4x32_10(ctr, key, u);
    int pair = (d % 4) / 2, second = d % 2;
    double u1 = ((double)u[2 * pair] + 0.5) * 0x1p-32;
    double u2 = ((double)u[2 * pair + 1] + 0.5) * 0x1p-32;
    double r = sqrt(-2.0 * log(u1));
    return second ? r * sin(OR_TWO_PI * u2) : r * cos(OR_TWO_PI * u2);
}

/* Husimi samples around chi = |p_eq, q_eq>: q0_i = q_eq_i + z_i / sqrt(gamma_i),
 * p0_i = p_eq_i + z_{F+i} sqrt(gamma_i), i.e. density |<p0 q0|chi>|^2 / (2 pi)^F,
 * and weights w = 1 / |<p0 q0|chi>|^2.  p0, q0: [F][n_traj]; w: [n_traj]. */
int or_sample_initial(int32_t F, const double *gamma, const double *p_eq, const double *q_eq,
                      int64_t n_traj, uint64_t seed, double *p0, double *q0, double *w)
{
    for (int64_t j = 0; j < n_traj; ++j) {
        double pj[64], qj[64];
        for (int i = 0; i < F; ++i) {
            qj[i] = q_eq[i] + or_normal(seed, j, i) / sqrt(gamma[i]);
            pj[i] = p_eq[i] + or_normal(seed, j, F + i) * sqrt(gamma[i]);
            q0[i * n_traj + j] = qj[i];
            p0[i * n_traj + j] = pj[i];
        }
        double complex lo = or_log_overlap(F, gamma, pj, qj, p_eq, q_eq);
        w[j] = exp(-2.0 * creal(lo));
    }
    return 0;
}

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Surrogate training objective and its parameter gradient                   */
/* ------------------------------------------------------------------------ */

/* Loss over n samples (rows of q [n][F], Vref [n], gref [n][F]) of the MLP
 * alone (its output V_mlp = s_out y and gradient):
 *   L = (1/n) sum_j [ alpha (V_mlp - Vref_j)^2 + beta |grad V_mlp - gref_j|^2 ].
 * Parameter gradients (same layout as the weights) are written to the d*
 * arrays.  The gradient-matching term is differentiated as the directional
 * derivative D_u V with u = dL/dgrad held fixed, propagated forward as a
 * tangent through the network and then back (second-order chain rule). */
double or_mlp_loss_grad(const or_mlp *m, int F, int64_t n, const double *q, const double *Vref,
                        const double *gref, double alpha, double beta,
                        double *dW1, double *db1, double *dW2, double *db2, double *dW3, double *db3,
                        double *dw4, double *db4)
{
    const int Hd = m->H;
    const double *W[3] = {m->W1, m->W2, m->W3}, *b[3] = {m->b1, m->b2, m->b3};
    double *dW[3] = {dW1, dW2, dW3}, *db[3] = {db1, db2, db3};
    memset(dW1, 0, sizeof(double) * Hd * F); memset(dW2, 0, sizeof(double) * Hd * Hd);
    memset(dW3, 0, sizeof(double) * Hd * Hd); memset(db1, 0, sizeof(double) * Hd);
    memset(db2, 0, sizeof(double) * Hd); memset(db3, 0, sizeof(double) * Hd);
    memset(dw4, 0, sizeof(double) * Hd); *db4 = 0.0;
    double *x = malloc(sizeof(double) * F), *u = malloc(sizeof(double) * F), *xt = malloc(sizeof(double) * F);
    double *z[3], *a[3], *f1[3], *f2[3], *zt[3], *at[3], *abar[3], *zb[3], *ztb[3], *ab[3], *atb[3];
    for (int l = 0; l < 3; ++l) {
        z[l] = malloc(sizeof(double) * Hd); a[l] = malloc(sizeof(double) * Hd);
        f1[l] = malloc(sizeof(double) * Hd); f2[l] = malloc(sizeof(double) * Hd);
        zt[l] = malloc(sizeof(double) * Hd); at[l] = malloc(sizeof(double) * Hd);
        abar[l] = malloc(sizeof(double) * Hd); zb[l] = malloc(sizeof(double) * Hd);
        ztb[l] = malloc(sizeof(double) * Hd); ab[l] = malloc(sizeof(double) * Hd);
        atb[l] = malloc(sizeof(double) * Hd);
    }
    double loss = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        const double *qj = q + j * F;
        for (int i = 0; i < F; ++i) x[i] = m->s_in[i] * qj[i];
        for (int l = 0; l < 3; ++l) {
            const int nin = l == 0 ? F : Hd;
            const double *in = l == 0 ? x : a[l - 1];
            for (int o = 0; o < Hd; ++o) {
                double acc = b[l][o];
                for (int i = 0; i < nin; ++i) acc += W[l][o * nin + i] * in[i];
                z[l][o] = acc;
                or_silu(acc, &a[l][o], &f1[l][o], &f2[l][o]);
            }
        }
        double y = m->b4;
        for (int o = 0; o < Hd; ++o) y += m->w4[o] * a[2][o];
        /* input gradient dy/dx via abar */
        for (int o = 0; o < Hd; ++o) abar[2][o] = m->w4[o];
        for (int l = 1; l >= 0; --l)
            for (int i = 0; i < Hd; ++i) {
                double acc = 0.0;
                for (int o = 0; o < Hd; ++o) acc += W[l + 1][o * Hd + i] * abar[l + 1][o] * f1[l + 1][o];
                abar[l][i] = acc;
            }
        double ev = m->s_out * y - Vref[j];
        loss += alpha * ev * ev;
        for (int i = 0; i < F; ++i) {
            double acc = 0.0;
            for (int o = 0; o < Hd; ++o) acc += m->W1[o * F + i] * abar[0][o] * f1[0][o];
            double gi = m->s_out * m->s_in[i] * acc;
            double e = gi - gref[j * F + i];
            loss += beta * e * e;
            u[i] = 2.0 * beta * e / (double)n;        /* dL/dgrad_i, held fixed */
        }
        /* tangent along u: D_u V = s_out * d/de y(x + e s_in u) */
        for (int i = 0; i < F; ++i) xt[i] = m->s_in[i] * u[i];
        for (int l = 0; l < 3; ++l) {
            const int nin = l == 0 ? F : Hd;
            const double *in = l == 0 ? xt : at[l - 1];
            for (int o = 0; o < Hd; ++o) {
                double acc = 0.0;
                for (int i = 0; i < nin; ++i) acc += W[l][o * nin + i] * in[i];
                zt[l][o] = acc;
                at[l][o] = f1[l][o] * acc;
            }
        }
        /* reverse pass of (y, y_t) with seeds ybar = 2 alpha ev s_out / n, ytbar = s_out */
        const double ybar = 2.0 * alpha * ev * m->s_out / (double)n, ytbar = m->s_out;
        *db4 += ybar;
        for (int o = 0; o < Hd; ++o) {
            dw4[o] += ybar * a[2][o] + ytbar * at[2][o];
            ab[2][o] = ybar * m->w4[o];
            atb[2][o] = ytbar * m->w4[o];
        }
        for (int l = 2; l >= 0; --l) {
            const int nin = l == 0 ? F : Hd;
            const double *in = l == 0 ? x : a[l - 1];
            const double *int_ = l == 0 ? xt : at[l - 1];
            for (int o = 0; o < Hd; ++o) {
                zb[l][o] = ab[l][o] * f1[l][o] + atb[l][o] * f2[l][o] * zt[l][o];
                ztb[l][o] = atb[l][o] * f1[l][o];
                db[l][o] += zb[l][o];
                for (int i = 0; i < nin; ++i) dW[l][o * nin + i] += zb[l][o] * in[i] + ztb[l][o] * int_[i];
            }
            if (l > 0)
                for (int i = 0; i < Hd; ++i) {
                    double s1 = 0.0, s2 = 0.0;
                    for (int o = 0; o < Hd; ++o) {
                        s1 += W[l][o * Hd + i] * zb[l][o];
                        s2 += W[l][o * Hd + i] * ztb[l][o];
                    }
                    ab[l - 1][i] = s1;
                    atb[l - 1][i] = s2;
                }
        }
    }
    free(x); free(u); free(xt);
    for (int l = 0; l < 3; ++l) {
        free(z[l]); free(a[l]); free(f1[l]); free(f2[l]); free(zt[l]); free(at[l]); free(abar[l]);
        free(zb[l]); free(ztb[l]); free(ab[l]); free(atb[l]);
    }
    return loss / (double)n;
}
