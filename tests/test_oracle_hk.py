"""Pins of the oracle's plain Herman-Kluk SC-IVR spectrum (Eq. I(E)_SCIVR).

Each trajectory contributes C_t e^{iS_t} <chi|p_t q_t> <p0 q0|chi> w (Eq.
SCTime_evolution between coherent states, sampling weight included); their
mean is the survival amplitude <chi|e^{-iHt}|chi>.  The pins use what the
mathematics fixes:

* A harmonic mode with chi at the origin (the ground state for gamma = omega):
  for the exact flow every single trajectory's summand equals e^{-i omega t/2}
  (the action cancels the overlap phase, |C_t| = 1), so the oracle's summands
  must approach it at the integrator's fourth order in dt.
* A displaced coherent state chi = |alpha>: the Monte Carlo mean must match the
  exact autocorrelation e^{-i omega t/2} exp(|alpha|^2 (e^{-i omega t} - 1))
  within five standard errors.  The same holds for a second reference state on
  trajectories drawn around the first, whose summands carry the sampling
  density's importance weight.
* Widths unequal to the frequency (gamma = omega/4, 2 omega): |det A| leaves 1, and
  the mean must match the exact survival amplitude of a sinc-DVR diagonalisation,
  which pins the prefactor's modulus |det A|^{1/2}.
* The folded transform: for C(t) = e^{-i E0 t} the symmetric rectangle rule gives the
  Dirichlet kernel (dt/pi) sin((n+1/2) x) / (2 sin(x/2)), x = (E - E0) dt.
* A 1D Morse oscillator: the peaks sit near the closed-form levels.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1312_4698_gb300 import workloads as wl
from tests import closed_forms as cf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _hk_amp(pes, gamma, p_eq, q_eq, dt, n_steps, N, seed, sample_center=None):
    c_p, c_q = (p_eq, q_eq) if sample_center is None else sample_center
    p0, q0, w = oracle.sample_initial(gamma, c_p, c_q, N, seed)
    amp, good = oracle.propagate(pes, gamma, p_eq, q_eq, dt, n_steps, p0, q0, amplitude=oracle.AMP_HK)
    return amp[0], good


def test_harmonic_ground_state_every_summand_is_the_exact_phase():
    omega = wl.cm1([1600.0, 3000.0])
    pes = wl.harmonic_pes(omega)
    zero = np.zeros(2)
    T = 2000.0
    errs = []
    for dt in (10.0, 5.0):
        n_steps = int(round(T / dt))
        amp, good = _hk_amp(pes, omega, zero, zero, dt, n_steps, 64, 3)
        assert good.all()
        t = dt * np.arange(n_steps + 1)
        exact = np.exp(-0.5j * omega.sum() * t)
        assert np.max(np.abs(amp[:, 0] - 1.0)) < 1e-14       # t = 0: C = 1, S = 0, the overlaps cancel
        errs.append(np.max(np.abs(amp - exact[None, :])))
    print("max |summand - e^{-i E0 t}|:", errs)
    assert errs[1] < 2e-3
    assert errs[0] / errs[1] > 12.0                         # fourth order: 16 for halving dt


def test_displaced_coherent_state_autocorrelation():
    omega = np.array([float(wl.cm1(1600.0))])
    pes = wl.harmonic_pes(omega)
    p_eq, q_eq = np.sqrt(omega), np.zeros(1)
    alpha2 = 0.5 * (omega[0] * q_eq[0] ** 2 + p_eq[0] ** 2 / omega[0])
    dt, n_steps, N = 5.0, 400, 20000
    amp, good = _hk_amp(pes, omega, p_eq, q_eq, dt, n_steps, N, 11)
    assert good.all()
    t = dt * np.arange(n_steps + 1)
    exact = np.exp(-0.5j * omega[0] * t) * np.exp(alpha2 * (np.exp(-1j * omega[0] * t) - 1.0))
    mean = amp.mean(axis=0)
    se = np.sqrt(amp.real.var(axis=0) + amp.imag.var(axis=0)) / np.sqrt(N)
    z = np.abs(mean - exact) / np.maximum(se, 1e-15)
    print("max deviation in standard errors:", z.max())
    assert np.all(z[1:] < 5.0)
    assert abs(mean[0] - 1.0) < 1e-14


@pytest.mark.parametrize("g_over_omega", [0.25, 2.0])
def test_widths_unequal_to_the_frequency_exercise_the_prefactor_modulus(g_over_omega):
    """Herman-Kluk is exact for a harmonic oscillator with any coherent-state width, but
    only with gamma != omega does |det A| leave 1 (here up to 1.25), so only then is the
    modulus |det A|^{1/2} of the prefactor tested.  The Monte Carlo mean of the summands
    must match the exact survival amplitude sum_n |<n|chi>|^2 e^{-i E_n t} (a sinc-DVR
    diagonalisation) within five standard errors; dropping the modulus, or taking
    |det A| instead of its square root, misses by 9 to 39 standard errors."""
    om = float(wl.cm1(1600.0))
    g = g_over_omega * om
    gamma, p_eq, q_eq = np.array([g]), np.array([0.8 * np.sqrt(g)]), np.array([0.3 / np.sqrt(g)])
    n = 400
    x = np.linspace(-1.0, 1.0, n) * 14.0 / np.sqrt(min(g, om))
    h = x[1] - x[0]
    i = np.arange(n)
    d = i[:, None] - i[None, :]
    H = np.where(d == 0, np.pi ** 2 / 3.0, 2.0 * (-1.0) ** d / np.where(d == 0, 1, d) ** 2) / (2.0 * h * h)
    H[np.diag_indices(n)] += 0.5 * om * om * x * x
    E, U = np.linalg.eigh(H)
    chi = (g / np.pi) ** 0.25 * np.exp(-0.5 * g * (x - q_eq[0]) ** 2 + 1j * p_eq[0] * (x - q_eq[0]))
    weights = np.abs((np.sqrt(h) * chi).conj() @ U) ** 2
    assert abs(weights.sum() - 1.0) < 1e-9
    dt, n_steps, N = 5.0, 400, 20000
    t = dt * np.arange(n_steps + 1)
    exact = (weights[None, :] * np.exp(-1j * np.outer(t, E))).sum(axis=1)
    amp, good = _hk_amp(wl.harmonic_pes(np.array([om])), gamma, p_eq, q_eq, dt, n_steps, N, 11)
    assert good.all()
    mean = amp.mean(axis=0)
    se = np.sqrt(amp.real.var(axis=0) + amp.imag.var(axis=0)) / np.sqrt(N)
    z = np.abs(mean - exact) / np.maximum(se, 1e-15)
    print(f"gamma/omega = {g_over_omega}: max deviation in standard errors {z[1:].max():.2f}")
    assert np.all(z[1:] < 5.0)


@pytest.mark.parametrize("dq,dp", [(0.5, 0.0), (0.0, 0.5), (0.7, -0.7)])
def test_reference_states_share_trajectories_sampled_around_the_first(dq, dp):
    """Two reference states on one set of trajectories drawn from the first state's
    Husimi density: the importance weight is that density's, so the mean of the second
    state's summands must still be its own exact autocorrelation (chi_1 displaced from
    chi_0 by dq, dp widths).  Weighting by the second state's own density instead
    misses it by 50 to 100 standard errors."""
    omega = np.array([float(wl.cm1(1600.0))])
    pes = wl.harmonic_pes(omega)
    om = omega[0]
    p_eq = np.array([[np.sqrt(om)], [np.sqrt(om) * (1.0 + dp)]])
    q_eq = np.array([[0.0], [dq / np.sqrt(om)]])
    dt, n_steps, N = 5.0, 400, 20000
    p0, q0, w = oracle.sample_initial(omega, p_eq[0], q_eq[0], N, 11)
    amp, good = oracle.propagate(pes, omega, p_eq, q_eq, dt, n_steps, p0, q0, amplitude=oracle.AMP_HK)
    assert good.all()
    t = dt * np.arange(n_steps + 1)
    for x in (0, 1):
        alpha2 = 0.5 * (om * q_eq[x, 0] ** 2 + p_eq[x, 0] ** 2 / om)
        exact = np.exp(-0.5j * om * t) * np.exp(alpha2 * (np.exp(-1j * om * t) - 1.0))
        mean = amp[x].mean(axis=0)
        se = np.sqrt(amp[x].real.var(axis=0) + amp[x].imag.var(axis=0)) / np.sqrt(N)
        z = np.abs(mean - exact) / np.maximum(se, 1e-15)
        print(f"chi {x}: max deviation in standard errors {z[1:].max():.2f}")
        assert np.all(z[1:] < 5.0), x
    # t = 0: the first state's summands are 1; the second's are the density ratio
    r = np.exp([2 * (oracle.log_overlap(omega, p_eq[1], q_eq[1], p0[:, j], q0[:, j]).real
                     - oracle.log_overlap(omega, p_eq[0], q_eq[0], p0[:, j], q0[:, j]).real) for j in range(8)])
    assert np.max(np.abs(amp[0][:, 0] - 1.0)) < 1e-14
    assert np.max(np.abs(amp[1][:8, 0] - r)) < 1e-12 * np.max(r)


def test_one_sided_transform_is_the_dirichlet_kernel():
    dt, n_steps, n = 10.0, 300, 7
    E0 = float(wl.cm1(2000.0))
    t = dt * np.arange(n_steps + 1)
    amp = np.tile(np.exp(-1j * E0 * t), (n, 1))
    good = np.ones(n, np.uint8)
    good[3] = 0
    amp[3] = np.nan                                       # excluded rows never reach the sum
    E = np.linspace(float(wl.cm1(1000.0)), float(wl.cm1(3000.0)), 401)
    I, ng, C = oracle.spectrum_hk(amp, good, n_steps, dt, E[0], E[-1], E.size)
    assert ng == n - 1
    assert np.allclose(C, np.exp(-1j * E0 * t), rtol=0, atol=1e-14)
    x = (E - E0) * dt
    with np.errstate(invalid="ignore", divide="ignore"):
        ref = dt / np.pi * np.where(np.abs(np.sin(x / 2)) > 1e-12,
                                    np.sin((n_steps + 0.5) * x) / (2 * np.sin(x / 2)), n_steps + 0.5)
    assert np.max(np.abs(I - ref)) <= 1e-10 * np.max(np.abs(ref))


def test_morse_levels_1d_plain_scivr():
    """H2-like Morse oscillator: the plain HK SC-IVR spectrum peaks near the exact levels."""
    omega = float(wl.cm1(1600.0))
    D = 0.2
    pes = wl.morse_pes([omega], D)
    gamma = np.array([omega])
    p_eq, q_eq = np.sqrt(gamma), np.zeros(1)
    N, n_steps, dt = 4000, 6000, 10.0
    amp, good = _hk_amp(pes, gamma, p_eq, q_eq, dt, n_steps, N, 0)
    assert good.mean() > 0.99
    E = wl.cm1(np.linspace(400.0, 4400.0, 801))
    I, _, _ = oracle.spectrum_hk(amp, good, n_steps, dt, E[0], E[-1], E.size)
    n = np.arange(3) + 0.5
    exact = wl.to_cm1(omega * n - (omega * n) ** 2 / (4 * D))
    golden = np.loadtxt(os.path.join(GOLDEN, "morse_levels_h2like.txt"))[:, 1]
    assert np.allclose(exact, golden, atol=1e-3)
    # the hard cut of C(t) at T puts side lobes every 2 pi / T (~23 cm^-1) around each
    # line: take the strongest maximum within 60 cm^-1 of each level
    Ec = wl.to_cm1(E)
    for lev in exact[:2]:
        win = np.flatnonzero(np.abs(Ec - lev) < 60.0)
        k = win[np.argmax(I[win])]
        y0, y1, y2 = I[k - 1], I[k], I[k + 1]
        pos = Ec[k] + 0.5 * (y0 - y2) / (y0 - 2 * y1 + y2) * (Ec[1] - Ec[0])
        print(f"level {lev:.2f}: strongest peak {pos:.2f} cm^-1")
        assert abs(pos - lev) < 5.0
