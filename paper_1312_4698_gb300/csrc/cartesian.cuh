// Cartesian triatomic surface in normal coordinates (Sec. III.A of arXiv:1312.4698:
// the molecular surfaces are functions of Cartesian coordinates, and the host
// builds the mass-weighted normal modes in which the trajectories run).
//
// The surface depends on x only through the two bond vectors w_0 = x0 - x1 and
// w_1 = x2 - x1 (atom 1 central): two Morse stretches of |w_b| and a bend
// (k/2)(cos theta - cos theta_e)^2 with cos theta = w_0.w_1 / (|w_0||w_1|).  In the
// normal coordinates q (x = x_eq + Lm q) each bond vector is affine in q,
// w_b = w_eq[b] + J[b] q with J[b] = d w_b / d q (3 x 3), so one force stage needs
// the bond-vector derivatives and two 3 x 3 chain-rule products per block:
//   grad_q V = sum_b J[b]^T dV/dw_b,   H_q = sum_{b,b'} J[b]^T d2V/dw_b dw_b' J[b'].
#pragma once

#include <cmath>

namespace scivr {

struct CartQ {
    double D[2], a[2], re[2];   // Morse stretches of bonds 0-1 and 2-1
    double k, cos_e;            // bend: k/2 (cos theta - cos_e)^2
    double w_eq[2][3];          // bond vectors at the equilibrium geometry
    double J[2][3][3];          // J[b][d][m] = d (w_b)_d / d q_m
};

// V, dV/dw [2][3] and d2V/dw dw [2][2][3][3] at bond vectors w.
// Bend derivatives in unit vectors u^ = w_0/|w_0|, v^ = w_1/|w_1|, c = u^.v^:
//   dc/dw_0 = (v^ - c u^)/|w_0|, dc/dw_1 = (u^ - c v^)/|w_1|,
//   d2c/dw_0 dw_0 = (3c u^u^T - c I - u^v^T - v^u^T)/|w_0|^2,
//   d2c/dw_0 dw_1 = (I - u^u^T - v^v^T + c u^v^T)/(|w_0||w_1|),
//   d2c/dw_1 dw_1 = (3c v^v^T - c I - u^v^T - v^u^T)/|w_1|^2.
__host__ __device__ inline double cart3_bond_terms(const CartQ &c, const double (&w)[2][3], double (&gw)[2][3],
                                                   double (&G)[2][2][3][3])
{
    double V = 0.0, r[2], e[2][3];
    for (int b = 0; b < 2; ++b) {
        r[b] = sqrt(w[b][0] * w[b][0] + w[b][1] * w[b][1] + w[b][2] * w[b][2]);
        for (int d = 0; d < 3; ++d) e[b][d] = w[b][d] / r[b];
    }
    for (int b = 0; b < 2; ++b)
        for (int bb = 0; bb < 2; ++bb)
            for (int d = 0; d < 3; ++d)
                for (int f = 0; f < 3; ++f) G[b][bb][d][f] = 0.0;
    // stretches: V_b(r), dr/dw = e, d2r/dw dw = (I - e e^T)/r
    for (int b = 0; b < 2; ++b) {
        const double ex = exp(-c.a[b] * (r[b] - c.re[b]));
        V += c.D[b] * (1.0 - ex) * (1.0 - ex);
        const double v1 = 2.0 * c.D[b] * c.a[b] * ex * (1.0 - ex);
        const double v2 = 2.0 * c.D[b] * c.a[b] * c.a[b] * ex * (2.0 * ex - 1.0);
        for (int d = 0; d < 3; ++d) {
            gw[b][d] = v1 * e[b][d];
            for (int f = 0; f < 3; ++f)
                G[b][b][d][f] = v2 * e[b][d] * e[b][f] + v1 * ((d == f ? 1.0 : 0.0) - e[b][d] * e[b][f]) / r[b];
        }
    }
    // bend
    const double cs = e[0][0] * e[1][0] + e[0][1] * e[1][1] + e[0][2] * e[1][2];
    const double dcs = cs - c.cos_e;
    V += 0.5 * c.k * dcs * dcs;
    double dc[2][3];
    for (int d = 0; d < 3; ++d) {
        dc[0][d] = (e[1][d] - cs * e[0][d]) / r[0];
        dc[1][d] = (e[0][d] - cs * e[1][d]) / r[1];
    }
    for (int b = 0; b < 2; ++b)
        for (int d = 0; d < 3; ++d) gw[b][d] += c.k * dcs * dc[b][d];
    for (int d = 0; d < 3; ++d)
        for (int f = 0; f < 3; ++f) {
            const double id = d == f ? 1.0 : 0.0;
            const double c00 = (3.0 * cs * e[0][d] * e[0][f] - cs * id - e[0][d] * e[1][f] - e[1][d] * e[0][f]) / (r[0] * r[0]);
            const double c11 = (3.0 * cs * e[1][d] * e[1][f] - cs * id - e[0][d] * e[1][f] - e[1][d] * e[0][f]) / (r[1] * r[1]);
            const double c01 = (id - e[0][d] * e[0][f] - e[1][d] * e[1][f] + cs * e[0][d] * e[1][f]) / (r[0] * r[1]);
            G[0][0][d][f] += c.k * (dc[0][d] * dc[0][f] + dcs * c00);
            G[1][1][d][f] += c.k * (dc[1][d] * dc[1][f] + dcs * c11);
            G[0][1][d][f] += c.k * (dc[0][d] * dc[1][f] + dcs * c01);
            G[1][0][f][d] += c.k * (dc[0][d] * dc[1][f] + dcs * c01);
        }
    return V;
}

// V, grad_q V [3] and the Hessian [3][3] in the normal coordinates q.
__host__ __device__ inline double cart3_eval_q(const CartQ &c, const double (&q)[3], double (&g)[3], double (&H)[3][3])
{
    double w[2][3], gw[2][3], G[2][2][3][3];
    for (int b = 0; b < 2; ++b)
        for (int d = 0; d < 3; ++d) w[b][d] = c.w_eq[b][d] + c.J[b][d][0] * q[0] + c.J[b][d][1] * q[1] + c.J[b][d][2] * q[2];
    const double V = cart3_bond_terms(c, w, gw, G);
    for (int m = 0; m < 3; ++m) {
        double acc = 0.0;
        for (int b = 0; b < 2; ++b)
            for (int d = 0; d < 3; ++d) acc += c.J[b][d][m] * gw[b][d];
        g[m] = acc;
    }
    // H = sum_{b,b'} J[b]^T G[b][b'] J[b']
    for (int m = 0; m < 3; ++m)
        for (int n = 0; n < 3; ++n) H[m][n] = 0.0;
    for (int b = 0; b < 2; ++b)
        for (int bb = 0; bb < 2; ++bb)
            for (int d = 0; d < 3; ++d) {
                double t[3];   // (G[b][bb] J[bb])[d][n]
                for (int n = 0; n < 3; ++n)
                    t[n] = G[b][bb][d][0] * c.J[bb][0][n] + G[b][bb][d][1] * c.J[bb][1][n] + G[b][bb][d][2] * c.J[bb][2][n];
                for (int m = 0; m < 3; ++m)
                    for (int n = 0; n < 3; ++n) H[m][n] += c.J[b][d][m] * t[n];
            }
    return V;
}

}  // namespace scivr
