"""Pins of the oracle's time-averaged spectrum (Eq. I(E)_discreto) and of its sampler.

* A single-frequency amplitude gives the Dirichlet kernel in closed form.
* Discrete Parseval on the DFT frequency grid.
* Uncoupled harmonic modes: the whole pipeline (Husimi samples -> propagation
  -> spectrum) equals the eigen-expansion sum_n <chi|n><n|p0 q0> D_K(E - E_n)
  evaluated without any time-domain sum.
* 1D Morse: peaks at the closed-form levels omega (n+1/2) - omega^2 (n+1/2)^2 / (4D)
  within semiclassical accuracy.
* Philox4x32-10 known-answer vectors; Husimi moments; the weights' unbiasedness.
* The sum rule: a spectral density integrates to <chi|chi> = 1 (time-averaged and
  plain Herman-Kluk), which pins the normalisation independently of its formula.
"""
import os

import numpy as np
import pytest
import scipy.stats

import oracle
from paper_1312_4698_gb300 import workloads as wl
from tests import closed_forms as cf


def test_dirichlet_closed_form():
    dt, n_steps = 10.0, 777
    K = n_steps + 1
    E0 = 0.0123
    amp = np.exp(-1j * E0 * dt * np.arange(K))[None, :]
    n_E = 501
    E_min, E_max = 0.005, 0.02
    I, ng = oracle.spectrum(amp, [1.0], [1], n_steps, dt, E_min, E_max, n_E)
    E = np.linspace(E_min, E_max, n_E)
    ref = dt ** 2 / (2 * np.pi * n_steps * dt) * np.abs(cf.dirichlet((E - E0) * dt, K)) ** 2
    assert ng == 1
    assert np.max(np.abs(I - ref)) <= 1e-11 * np.max(ref)


def test_parseval_on_the_dft_grid():
    rng = np.random.default_rng(0)
    n, n_steps, dt = 5, 63, 7.0
    K = n_steps + 1
    amp = rng.normal(size=(n, K)) + 1j * rng.normal(size=(n, K))
    w = rng.uniform(0.5, 2.0, n)
    good = np.array([1, 1, 0, 1, 1], dtype=np.uint8)
    I, ng = oracle.spectrum(amp, w, good, n_steps, dt, 0.0, 2 * np.pi / dt * (K - 1) / K, K)
    T = n_steps * dt
    lhs = np.sum(I)
    rhs = dt ** 2 / (2 * np.pi * T * ng) * np.sum(w * good * K * np.sum(np.abs(amp) ** 2, axis=1))
    assert ng == 4
    assert abs(lhs - rhs) <= 1e-12 * rhs


def test_bad_trajectories_are_excluded_and_n_good_normalises():
    rng = np.random.default_rng(1)
    n, n_steps, dt = 6, 40, 5.0
    amp = rng.normal(size=(n, n_steps + 1)) + 1j * rng.normal(size=(n, n_steps + 1))
    amp[2, 7] = np.nan
    w = rng.uniform(0.5, 2.0, n)
    good = np.array([1, 0, 0, 1, 1, 0], dtype=np.uint8)
    I, ng = oracle.spectrum(amp, w, good, n_steps, dt, 0.01, 0.4, 33)
    sel = good.astype(bool)
    I2, ng2 = oracle.spectrum(amp[sel], w[sel], np.ones(3, np.uint8), n_steps, dt, 0.01, 0.4, 33)
    assert ng == 3 and ng2 == 3
    assert np.array_equal(I, I2)


@pytest.mark.parametrize("omegas", [[wl.cm1(1600.0)], wl.cm1([1600.0, 3650.0])])
def test_harmonic_pipeline_equals_eigen_expansion(omegas):
    omegas = np.atleast_1d(np.asarray(omegas, dtype=float))
    F = omegas.size
    dt, n_steps, N = 10.0, 1200, 48
    K = n_steps + 1
    rot = [cf.harmonic_rotation(w, dt) for w in omegas]
    th = np.array([r[0] for r in rot])
    gts = np.array([r[1] for r in rot])
    pes = wl.harmonic_pes(omegas)
    p_eq, q_eq = np.sqrt(gts), np.zeros(F)
    p0, q0, w = oracle.sample_initial(gts, p_eq, q_eq, N, 7)
    amp, good = oracle.propagate(pes, gts, p_eq, q_eq, dt, n_steps, p0, q0)
    assert good.all()
    E_min, E_max, n_E = 0.0, float(np.sum(omegas)) * 3.2, 400
    I, ng = oracle.spectrum(amp[0], w, good, n_steps, dt, E_min, E_max, n_E)
    E = np.linspace(E_min, E_max, n_E)
    # eigen-expansion: X(E) = prod over modes is NOT a product in E; do it for one mode
    # at a time with the other modes' energies folded in via the multi-index sum.
    acc = np.zeros(n_E)
    for j in range(N):
        if F == 1:
            X = cf.harmonic_X_eigen(E, dt, K, th[0], cf.glauber_alpha(gts[0], p_eq[0], q_eq[0]),
                                    cf.glauber_alpha(gts[0], p0[0, j], q0[0, j]),
                                    p_eq[0], q_eq[0], p0[0, j], q0[0, j])
        else:
            # two modes: sum over n1 of mode-1 coefficient times mode-2 expansion shifted by n1
            a1x = cf.glauber_alpha(gts[0], p_eq[0], q_eq[0])
            a10 = cf.glauber_alpha(gts[0], p0[0, j], q0[0, j])
            pref1 = np.exp(0.5j * (p_eq[0] * q_eq[0] - p0[0, j] * q0[0, j])
                           - 0.5 * abs(a1x) ** 2 - 0.5 * abs(a10) ** 2)
            z1 = np.conj(a1x) * a10
            X = np.zeros(n_E, dtype=np.complex128)
            term = 1.0 + 0j
            for n1 in range(60):
                if n1 > 0:
                    term = term * z1 / n1
                shifted = E - (n1 + 0.5) * th[0] / dt
                X += pref1 * term * cf.harmonic_X_eigen(
                    shifted, dt, K, th[1], cf.glauber_alpha(gts[1], p_eq[1], q_eq[1]),
                    cf.glauber_alpha(gts[1], p0[1, j], q0[1, j]), p_eq[1], q_eq[1],
                    p0[1, j], q0[1, j])
                if abs(term) < 1e-20 and n1 > 5:
                    break
        acc += w[j] * np.abs(X) ** 2
    ref = dt ** 2 / (2 * np.pi * n_steps * dt * N) * acc
    assert np.max(np.abs(I - ref)) <= 1e-9 * np.max(ref)


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_morse_levels_1d():
    """H2-like Morse oscillator: TA-SC-IVR peaks near the exact levels."""
    omega = float(wl.cm1(1600.0))
    D = 0.2
    pes = wl.morse_pes([omega], D)
    gamma = np.array([omega])
    p_eq, q_eq = np.sqrt(gamma), np.zeros(1)
    N, n_steps, dt = 800, 6000, 10.0
    p0, q0, w = oracle.sample_initial(gamma, p_eq, q_eq, N, 0)
    amp, good = oracle.propagate(pes, gamma, p_eq, q_eq, dt, n_steps, p0, q0)
    assert good.mean() > 0.99
    E = wl.cm1(np.linspace(400.0, 4400.0, 801))
    I, _ = oracle.spectrum(amp[0], w, good, n_steps, dt, E[0], E[-1], E.size)
    peaks = wl.to_cm1(cf.find_peaks(E, I, rel=0.02))
    n = np.arange(3) + 0.5
    exact = wl.to_cm1(omega * n - (omega * n) ** 2 / (4 * D))
    golden = np.loadtxt(os.path.join(GOLDEN, "morse_levels_h2like.txt"))[:, 1]
    assert np.allclose(exact, golden, atol=1e-3)
    # semiclassical + Monte Carlo accuracy: measured 1.2 and 3.4 cm^-1 for n = 0, 1
    # (N = 800, T = 60000 au); the bound is 5 cm^-1 per level
    assert cf.match_peaks(exact[:1], peaks) < 2.5, (peaks, exact)
    assert cf.match_peaks(exact[1:2], peaks) < 5.0, (peaks, exact)


def philox_kat():
    rows = []
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.strip() and not line.startswith("#"):
            v = [int(x, 16) for x in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_philox_known_answers():
    kat = philox_kat()
    assert len(kat) == 3
    for ctr, key, ref in kat:
        assert list(oracle.philox4x32_10(ctr, key)) == ref


def test_husimi_moments_and_normality():
    gamma = wl.cm1([1600.0, 3650.0, 3750.0])
    p_eq, q_eq = np.sqrt(gamma), np.array([0.5, 0.0, -0.5])
    N = 200000
    p0, q0, w = oracle.sample_initial(gamma, p_eq, q_eq, N, 42)
    zq = (q0 - q_eq[:, None]) * np.sqrt(gamma)[:, None]
    zp = (p0 - p_eq[:, None]) / np.sqrt(gamma)[:, None]
    for z in np.concatenate([zq, zp]):
        assert abs(z.mean()) < 5 / np.sqrt(N)
        assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0 / N)
        assert scipy.stats.kstest(z, "norm").pvalue > 1e-4
    # different draws are uncorrelated
    c = np.corrcoef(np.concatenate([zq, zp]))
    assert np.max(np.abs(c - np.eye(6))) < 5 / np.sqrt(N)


def test_weights_are_inverse_husimi_density():
    """E_rho[w |<p0 q0|chi'>|^2] = (2 pi)^-F int |<pq|chi'>|^2 dp dq = 1 for any chi'."""
    gamma = wl.cm1([1600.0, 3650.0])
    p_eq, q_eq = np.sqrt(gamma), np.zeros(2)
    N = 400000
    p0, q0, w = oracle.sample_initial(gamma, p_eq, q_eq, N, 3)
    # chi' displaced by half a width in q and in p
    q1 = q_eq + 0.5 / np.sqrt(gamma)
    p1 = p_eq - 0.5 * np.sqrt(gamma)
    f = np.exp(-0.5 * np.sum(gamma[:, None] * (q0 - q1[:, None]) ** 2
                             + (p0 - p1[:, None]) ** 2 / gamma[:, None], axis=0))
    est = np.mean(w * f)
    err = np.std(w * f) / np.sqrt(N)
    assert abs(est - 1.0) < 5 * err
    # and exactly: w |<p0 q0|chi>|^2 = 1 sample by sample
    f0 = np.exp(-0.5 * np.sum(gamma[:, None] * (q0 - q_eq[:, None]) ** 2
                              + (p0 - p_eq[:, None]) ** 2 / gamma[:, None], axis=0))
    assert np.max(np.abs(w * f0 - 1.0)) < 1e-12


def test_spectra_obey_the_sum_rule():
    """A spectral density integrates to <chi|chi> = 1.  Over one period 2 pi / dt, on the
    grid of K = n_steps + 1 points where the sum is exact:
    * time-averaged: for the harmonic ground state (gamma = the integrator's modified
      frequency, chi at the origin) every trajectory has w |a(c)|^2 = 1, so the integral
      is (1/T) dt (n_steps + 1) = (n_steps + 1) / n_steps, the rectangle rule's value;
      a lost factor dt or 2 pi in the normalisation would be visible at once;
    * plain Herman-Kluk: only the c = 0 term survives the integration, so the integral
      is Re C(0) = 1 on any surface."""
    omegas = wl.cm1([1600.0, 3650.0])
    dt, n_steps = 10.0, 400
    K = n_steps + 1
    gts = np.array([cf.harmonic_rotation(w, dt)[1] for w in omegas])
    z = np.zeros(2)
    p0, q0, w = oracle.sample_initial(gts, z, z, 64, 3)
    amp, good = oracle.propagate(wl.harmonic_pes(omegas), gts, z[None], z[None], dt, n_steps, p0, q0)
    assert np.max(np.abs(w[:, None] * np.abs(amp[0]) ** 2 - 1.0)) < 1e-12
    period = 2.0 * np.pi / dt
    I, ng = oracle.spectrum(amp[0], w, good, n_steps, dt, 0.0, period * (K - 1) / K, K)
    assert abs(I.sum() * period / K - K / n_steps) < 1e-12

    w8 = wl.config_f3(n_traj=64, n_steps=n_steps)
    p0, q0, w = oracle.sample_initial(w8.gamma, w8.p_eq, w8.q_eq, 64, 1)
    ah, gh = oracle.propagate(w8.pes, w8.gamma, w8.p_eq, w8.q_eq, dt, n_steps, p0, q0, amplitude=oracle.AMP_HK)
    Ih, ngh, C = oracle.spectrum_hk(ah[0], gh, n_steps, dt, 0.0, period * (K - 1) / K, K)
    assert ngh > 0 and C[0] == 1.0
    assert abs(Ih.sum() * period / K - 1.0) < 1e-12
