// Normal modes of a Cartesian triatomic surface and the potential handle that
// propagates on it (Sec. III.A of arXiv:1312.4698: the host driver turns the
// Cartesian surface into mass-weighted normal coordinates; the trajectories run
// in those).  Host code: the Hessian at the equilibrium geometry from the bond-
// vector derivatives of cartesian.cuh, its mass-weighted form diagonalised by
// Jacobi rotations (largest off-diagonal element first), and the affine map of
// the bond vectors to q that the kernels evaluate.
#include <cmath>
#include <cstring>
#include <vector>

#include "cartesian.cuh"
#include "scivr_internal.cuh"

namespace scivr {
namespace {

bool valid(const scivr_cart_triatomic *c)
{
    if (!c) return false;
    auto pos = [](double v) { return std::isfinite(v) && v > 0.0; };
    for (int i = 0; i < 3; ++i)
        if (!pos(c->mass[i])) return false;
    for (int b = 0; b < 2; ++b)
        if (!pos(c->D[b]) || !pos(c->a[b]) || !pos(c->re[b])) return false;
    return pos(c->k_bend) && std::isfinite(c->theta_e) && c->theta_e > 0.0 && c->theta_e < M_PI;
}

CartQ params(const scivr_cart_triatomic *c)
{
    CartQ p{};
    for (int b = 0; b < 2; ++b) {
        p.D[b] = c->D[b];
        p.a[b] = c->a[b];
        p.re[b] = c->re[b];
    }
    p.k = c->k_bend;
    p.cos_e = std::cos(c->theta_e);
    return p;
}

// Coefficient of atom i in bond vector b: w_0 = x0 - x1, w_1 = x2 - x1.
double bond_coef(int b, int atom)
{
    if (atom == 1) return -1.0;
    return (b == 0 ? atom == 0 : atom == 2) ? 1.0 : 0.0;
}

struct Modes {
    double omega[3];
    double x_eq[9];
    double Lm[9][3];
};

void normal_modes(const scivr_cart_triatomic *c, Modes &out)
{
    const double h = 0.5 * c->theta_e;
    double x[9] = {-c->re[0] * std::sin(h), c->re[0] * std::cos(h), 0.0, 0.0, 0.0, 0.0,
                   c->re[1] * std::sin(h), c->re[1] * std::cos(h), 0.0};
    std::memcpy(out.x_eq, x, sizeof(x));
    CartQ p = params(c);
    double w[2][3], gw[2][3], G[2][2][3][3];
    for (int d = 0; d < 3; ++d) {
        w[0][d] = x[d] - x[3 + d];
        w[1][d] = x[6 + d] - x[3 + d];
    }
    cart3_bond_terms(p, w, gw, G);
    // mass-weighted Cartesian Hessian: sum over bond pairs of P_b^T G P_b' / sqrt(m_i m_j)
    double A[9][9], V[9][9];
    for (int i = 0; i < 3; ++i)
        for (int d = 0; d < 3; ++d)
            for (int j = 0; j < 3; ++j)
                for (int f = 0; f < 3; ++f) {
                    double hx = 0.0;
                    for (int b = 0; b < 2; ++b)
                        for (int bb = 0; bb < 2; ++bb) hx += bond_coef(b, i) * bond_coef(bb, j) * G[b][bb][d][f];
                    A[3 * i + d][3 * j + f] = hx / std::sqrt(c->mass[i] * c->mass[j]);
                }
    for (int i = 0; i < 9; ++i)
        for (int j = 0; j < 9; ++j) V[i][j] = i == j ? 1.0 : 0.0;
    // Jacobi: rotate away the largest off-diagonal element until all are negligible
    double scale = 0.0;
    for (int i = 0; i < 9; ++i) scale = std::fmax(scale, std::fabs(A[i][i]));
    for (int it = 0; it < 2000; ++it) {
        int p0 = 0, q0 = 1;
        double big = 0.0;
        for (int i = 0; i < 9; ++i)
            for (int j = i + 1; j < 9; ++j)
                if (std::fabs(A[i][j]) > big) { big = std::fabs(A[i][j]); p0 = i; q0 = j; }
        if (big <= 1e-17 * scale) break;
        const double app = A[p0][p0], aqq = A[q0][q0], apq = A[p0][q0];
        const double phi = 0.5 * std::atan2(2.0 * apq, aqq - app);
        const double cs = std::cos(phi), sn = std::sin(phi);
        for (int k = 0; k < 9; ++k) {   // columns p0, q0
            const double akp = A[k][p0], akq = A[k][q0];
            A[k][p0] = cs * akp - sn * akq;
            A[k][q0] = sn * akp + cs * akq;
        }
        for (int k = 0; k < 9; ++k) {   // rows p0, q0
            const double apk = A[p0][k], aqk = A[q0][k];
            A[p0][k] = cs * apk - sn * aqk;
            A[q0][k] = sn * apk + cs * aqk;
        }
        for (int k = 0; k < 9; ++k) {
            const double vkp = V[k][p0], vkq = V[k][q0];
            V[k][p0] = cs * vkp - sn * vkq;
            V[k][q0] = sn * vkp + cs * vkq;
        }
    }
    // the three largest eigenvalues, in increasing order
    int order[9];
    for (int i = 0; i < 9; ++i) order[i] = i;
    for (int i = 1; i < 9; ++i)
        for (int j = i; j > 0 && A[order[j]][order[j]] < A[order[j - 1]][order[j - 1]]; --j) {
            const int t = order[j];
            order[j] = order[j - 1];
            order[j - 1] = t;
        }
    for (int m = 0; m < 3; ++m) {
        const int col = order[6 + m];
        out.omega[m] = std::sqrt(A[col][col]);
        double sgn = 1.0;
        for (int i = 0; i < 9; ++i)
            if (std::fabs(V[i][col]) > 1e-3) { sgn = V[i][col] > 0.0 ? 1.0 : -1.0; break; }
        for (int i = 0; i < 9; ++i) out.Lm[i][m] = sgn * V[i][col] / std::sqrt(c->mass[i / 3]);
    }
}

}  // namespace

}  // namespace scivr

using namespace scivr;

extern "C" int scivr_normal_modes(const scivr_cart_triatomic *c, double *omega, double *x_eq, double *Lm)
{
    if (!valid(c)) return set_error(SCIVR_EINVAL, "scivr_normal_modes: invalid triatomic parameters");
    Modes md;
    normal_modes(c, md);
    if (omega) std::memcpy(omega, md.omega, sizeof(md.omega));
    if (x_eq) std::memcpy(x_eq, md.x_eq, sizeof(md.x_eq));
    if (Lm) std::memcpy(Lm, md.Lm, sizeof(md.Lm));
    clear_error();
    return SCIVR_OK;
}

extern "C" int scivr_normal_to_cartesian(const scivr_cart_triatomic *c, int64_t n, const double *q, double *x)
{
    if (!valid(c)) return set_error(SCIVR_EINVAL, "scivr_normal_to_cartesian: invalid triatomic parameters");
    if (n < 0 || (n > 0 && (!q || !x))) return set_error(SCIVR_EINVAL, "scivr_normal_to_cartesian: bad arrays");
    Modes md;
    normal_modes(c, md);
    for (int64_t j = 0; j < n; ++j)
        for (int i = 0; i < 9; ++i)
            x[j * 9 + i] = md.x_eq[i] + md.Lm[i][0] * q[j * 3] + md.Lm[i][1] * q[j * 3 + 1] + md.Lm[i][2] * q[j * 3 + 2];
    clear_error();
    return SCIVR_OK;
}

extern "C" int scivr_cartesian_to_normal(const scivr_cart_triatomic *c, int64_t n, const double *x, double *q)
{
    if (!valid(c)) return set_error(SCIVR_EINVAL, "scivr_cartesian_to_normal: invalid triatomic parameters");
    if (n < 0 || (n > 0 && (!q || !x))) return set_error(SCIVR_EINVAL, "scivr_cartesian_to_normal: bad arrays");
    Modes md;
    normal_modes(c, md);
    for (int64_t j = 0; j < n; ++j)
        for (int m = 0; m < 3; ++m) {
            double acc = 0.0;
            for (int i = 0; i < 9; ++i) acc += md.Lm[i][m] * c->mass[i / 3] * (x[j * 9 + i] - md.x_eq[i]);
            q[j * 3 + m] = acc;
        }
    clear_error();
    return SCIVR_OK;
}

extern "C" int scivr_create_pes_cartesian(const scivr_cart_triatomic *c, scivr_pes *out)
{
    if (!out) return set_error(SCIVR_EINVAL, "scivr_create_pes_cartesian: NULL output");
    *out = nullptr;
    if (!valid(c)) return set_error(SCIVR_EINVAL, "scivr_create_pes_cartesian: invalid triatomic parameters");
    Modes md;
    normal_modes(c, md);
    CartQ p = params(c);
    for (int b = 0; b < 2; ++b) {
        const int ia = b == 0 ? 0 : 2;
        for (int d = 0; d < 3; ++d) {
            p.w_eq[b][d] = md.x_eq[3 * ia + d] - md.x_eq[3 + d];
            for (int m = 0; m < 3; ++m) p.J[b][d][m] = md.Lm[3 * ia + d][m] - md.Lm[3 + d][m];
        }
    }
    // device block: the CartQ record, then omega and zero D, a (the diagonal fields
    // of the polynomial kind, unused by this kind) in 256-byte slots
    const size_t bytes = 256 * ((sizeof(CartQ) + 255) / 256) + 3 * 256;
    void *blob = nullptr;
    cudaError_t e = cudaMalloc(&blob, bytes);
    if (e != cudaSuccess) return cuda_error(e, "scivr_create_pes_cartesian: cudaMalloc");
    std::vector<char> host(bytes, 0);
    std::memcpy(host.data(), &p, sizeof(CartQ));
    const size_t o_om = 256 * ((sizeof(CartQ) + 255) / 256);
    std::memcpy(host.data() + o_om, md.omega, sizeof(md.omega));
    e = cudaMemcpy(blob, host.data(), bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(blob);
        return cuda_error(e, "scivr_create_pes_cartesian: cudaMemcpy");
    }
    scivr_pes h = new scivr_pes_s{};
    h->blob = blob;
    h->mlp_blob = nullptr;
    PesDev &dv = h->dev;
    char *b = static_cast<char *>(blob);
    dv.F = 3;
    dv.P = 6;
    dv.kind = SCIVR_PES_CART3;
    dv.cart = reinterpret_cast<const CartQ *>(b);
    dv.diag_kind = SCIVR_DIAG_HARMONIC;
    dv.has3 = dv.has4 = 0;
    dv.omega = reinterpret_cast<const double *>(b + o_om);
    dv.D = reinterpret_cast<const double *>(b + o_om + 256);
    dv.a = reinterpret_cast<const double *>(b + o_om + 512);
    *out = h;
    clear_error();
    return SCIVR_OK;
}
