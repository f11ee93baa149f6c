"""Closed forms and analysis helpers used by the tests (no dependency on either implementation).

Everything here is written from textbook mathematics, not from the oracle or
the library:

* Yoshida's fourth-order triple jump, composed as 2x2 matrices for a
  harmonic mode (exact for a linear flow);
* Glauber coherent-state algebra: <beta|alpha> = exp(-|a|^2/2 - |b|^2/2 + b* a),
  and the evolution |alpha> -> e^{-i theta/2} |alpha e^{-i theta}> under a
  harmonic step whose one-step map is a rotation by theta;
* the Dirichlet kernel sum_{c=0}^{K-1} e^{i c x};
* peak picking by 3-point parabolic interpolation.
"""
from __future__ import annotations

import math

import numpy as np


def yoshida_coefficients():
    """Drift fractions c1..c4 and kick fractions d1..d3 of the triple jump (Yoshida 1990)."""
    s = 2.0 ** (1.0 / 3.0)
    w1 = 1.0 / (2.0 - s)
    w0 = -s / (2.0 - s)
    return [w1 / 2, (w0 + w1) / 2, (w0 + w1) / 2, w1 / 2], [w1, w0, w1]


def harmonic_step_matrix(omega: float, dt: float) -> np.ndarray:
    """One triple-jump step for V = omega^2 q^2 / 2, acting on (q, p)."""
    c, d = yoshida_coefficients()
    R = np.eye(2)
    for k in range(4):
        R = np.array([[1.0, c[k] * dt], [0.0, 1.0]]) @ R
        if k < 3:
            R = np.array([[1.0, 0.0], [-d[k] * dt * omega * omega, 1.0]]) @ R
    return R


def harmonic_rotation(omega: float, dt: float):
    """(theta, gamma_tilde): the step is a rotation by theta in (sqrt(g) q, p / sqrt(g))."""
    R = harmonic_step_matrix(omega, dt)
    theta = math.acos(0.5 * (R[0, 0] + R[1, 1]))
    g = math.sqrt(-R[1, 0] / R[0, 1])
    return theta, g


def glauber_alpha(g, p, q):
    return (np.sqrt(g) * q + 1j * p / np.sqrt(g)) / np.sqrt(2.0)


def harmonic_amplitude(omegas, dt, n_steps, p0, q0, p_eq, q_eq):
    """Exact <chi| U^c |p0 q0> for uncoupled harmonic modes with widths gamma_tilde.

    |p, q> (Eq. coherent_state phase convention) equals e^{-i p q / 2} |alpha>.
    Returns (amp [K], thetas [F], gammas [F])."""
    c = np.arange(n_steps + 1)
    log_a = np.zeros(n_steps + 1, dtype=np.complex128)
    thetas, gammas = [], []
    for i, w in enumerate(np.atleast_1d(omegas)):
        th, g = harmonic_rotation(float(w), dt)
        thetas.append(th)
        gammas.append(g)
        a0 = glauber_alpha(g, p0[i], q0[i])
        ax = glauber_alpha(g, p_eq[i], q_eq[i])
        log_a += (0.5j * (p_eq[i] * q_eq[i] - p0[i] * q0[i]) - 0.5j * c * th
                  - 0.5 * abs(ax) ** 2 - 0.5 * abs(a0) ** 2
                  + np.conj(ax) * a0 * np.exp(-1j * c * th))
    return np.exp(log_a), np.array(thetas), np.array(gammas)


def dirichlet(x, K):
    """sum_{c=0}^{K-1} e^{i c x} in closed form (geometric series)."""
    x = np.asarray(x, dtype=np.float64)
    half = 0.5 * x
    s = np.sin(half)
    near = np.abs(s) < 1e-12
    safe = np.where(near, 1.0, s)
    val = np.exp(0.5j * (K - 1) * x) * np.sin(K * half) / safe
    # at x = 2 pi m the sum is K e^{i (K-1) pi m}
    lim = K * np.exp(0.5j * (K - 1) * x)
    return np.where(near, lim, val)


def harmonic_X_eigen(E, dt, K, theta, alpha_chi, alpha0, p_eq, q_eq, p0, q0, n_max=80):
    """X(E) = sum_c <chi|U^c|p0 q0> e^{i E c dt} for ONE mode via the eigen-expansion
    <chi|n><n|p0 q0> e^{-i (n + 1/2) theta c}; independent of any time-domain sum."""
    pref = np.exp(0.5j * (p_eq * q_eq - p0 * q0) - 0.5 * abs(alpha_chi) ** 2 - 0.5 * abs(alpha0) ** 2)
    z = np.conj(alpha_chi) * alpha0
    X = np.zeros_like(np.asarray(E, dtype=np.float64), dtype=np.complex128)
    term = 1.0 + 0j
    for n in range(n_max):
        if n > 0:
            term = term * z / n
        X = X + term * dirichlet(E * dt - (n + 0.5) * theta, K)
        if abs(term) < 1e-20 and n > 5:
            break
    return pref * X


def find_peaks(E, I, rel=0.01):
    """Grid local maxima >= rel * max(I), refined by a 3-point parabola.  Returns positions."""
    E = np.asarray(E)
    I = np.asarray(I)
    thr = rel * I.max()
    out = []
    for k in range(1, len(I) - 1):
        if I[k] >= thr and I[k] > I[k - 1] and I[k] >= I[k + 1]:
            y0, y1, y2 = I[k - 1], I[k], I[k + 1]
            den = y0 - 2 * y1 + y2
            off = 0.5 * (y0 - y2) / den if den != 0 else 0.0
            out.append(E[k] + off * (E[1] - E[0]))
    return np.array(out)


def match_peaks(ref, got):
    """Max |position error| over reference peaks, matching each to its nearest peak."""
    if len(ref) == 0:
        return 0.0
    if len(got) == 0:
        return float("inf")
    return float(max(np.min(np.abs(np.asarray(got) - r)) for r in ref))
