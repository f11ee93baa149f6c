"""Pins of the oracle's propagation: integrator, monodromy, action, prefactor phase, amplitude.

* Harmonic modes: the triple-jump step is a rotation by theta in coordinates
  scaled by gamma_tilde, so Herman-Kluk with widths gamma_tilde is exact and
  <chi|U^c|p0 q0> has a closed form in Glauber coherent-state algebra.  The
  oracle's amplitude series (overlap, action, prefactor phase and its
  unwrapping) must equal it to rounding.
* Anharmonic surfaces: symplecticity M^T J M = J, energy conservation of
  order dt^4, time reversal, finite-difference monodromy, order-4 convergence
  and the generating-function identity dS = p_t dq_t - p_0 dq_0.
"""
import numpy as np
import pytest

import oracle
from paper_1312_4698_gb300 import workloads as wl
from tests import closed_forms as cf


def _J(F):
    Z, I = np.zeros((F, F)), np.eye(F)
    # ordering (p, q): dp/dt = -dH/dq, dq/dt = dH/dp
    return np.block([[Z, -I], [I, Z]])


@pytest.mark.parametrize("omegas", [[wl.cm1(1600.0)], wl.cm1([1600.0, 3650.0, 3750.0])])
def test_harmonic_amplitude_closed_form(omegas):
    omegas = np.atleast_1d(np.asarray(omegas, dtype=float))
    F = omegas.size
    dt, n_steps = 10.0, 1500
    thetas, gts = zip(*[cf.harmonic_rotation(w, dt) for w in omegas])
    gts = np.array(gts)
    pes = wl.harmonic_pes(omegas)
    p_eq, q_eq = np.sqrt(gts), np.zeros(F)
    rng = np.random.default_rng(5)
    for _ in range(4):
        q0 = rng.normal(0, 1, F) / np.sqrt(gts)
        p0 = p_eq + rng.normal(0, 1, F) * np.sqrt(gts)
        r = oracle.propagate_one(pes, gts, p_eq, q_eq, dt, n_steps, p0, q0)
        ref, th, _ = cf.harmonic_amplitude(omegas, dt, n_steps, p0, q0, p_eq, q_eq)
        assert r["good"]
        err = np.max(np.abs(r["amp"][0] - ref))
        assert err < 1e-10, err
        c = np.arange(n_steps + 1)
        # continuous phase: theta_c = arg det A = -c sum_i theta_i, |det A| = 1
        assert np.max(np.abs(r["theta"] - (-c * np.sum(th)))) < 1e-9
        assert np.max(np.abs(np.abs(r["detA"]) - 1.0)) < 1e-12
        assert np.max(np.abs(r["detM"] - 1.0)) < 1e-12
        # action of a quadratic flow: S = (p q - p0 q0) / 2
        assert abs(r["S"][-1] - 0.5 * np.sum(r["p"] * r["q"] - p0 * q0)) < 1e-10


def test_phase_unwrapping_when_arg_det_A_turns_more_than_pi_per_step():
    """24 harmonic modes at 2900-3900 cm^-1 with dt = 10 au turn arg det A by 3.7 rad
    per step, so a principal-value unwrapping of the bare increments loses whole turns.
    The oracle unwraps relative to the reference rotation exp(-i sum_i gamma_i t) and
    must still give the closed-form theta_c = -c sum_i theta_i and amplitude series."""
    omegas = wl.cm1(np.linspace(2900.0, 3900.0, 24))
    F, dt, n_steps = omegas.size, 10.0, 600
    thetas, gts = zip(*[cf.harmonic_rotation(w, dt) for w in omegas])
    gts = np.array(gts)
    assert np.sum(thetas) > np.pi
    pes = wl.harmonic_pes(omegas)
    p_eq, q_eq = np.sqrt(gts), np.zeros(F)
    rng = np.random.default_rng(5)
    q0 = rng.normal(0, 1, F) / np.sqrt(gts)
    p0 = p_eq + rng.normal(0, 1, F) * np.sqrt(gts)
    r = oracle.propagate_one(pes, gts, p_eq, q_eq, dt, n_steps, p0, q0)
    ref, th, _ = cf.harmonic_amplitude(omegas, dt, n_steps, p0, q0, p_eq, q_eq)
    c = np.arange(n_steps + 1)
    exact = -c * np.sum(th)
    assert r["good"]
    assert np.max(np.abs(r["amp"][0] - ref)) < 1e-10
    assert np.max(np.abs(r["theta"] - exact)) < 1e-9
    bare = np.angle(r["detA"])
    naive = np.concatenate([[0.0], np.cumsum(np.angle(np.exp(1j * np.diff(bare))))])
    assert np.max(np.abs(naive - exact)) > 1.0       # the case the reference rotation exists for


def test_recipe_surface_with_24_modes_stays_symplectic():
    """The F = 24 surface of the synthetic recipe (2576 cubic and 17526 quartic
    couplings): along a Husimi trajectory M^T J M = J and det M = 1 to rounding."""
    w8 = wl.config_generic(24, 0, 1, 300)
    assert (w8.pes.c3.size, w8.pes.c4.size) == (2576, 17526)
    p0, q0, _ = oracle.sample_initial(w8.gamma, w8.p_eq[0], w8.q_eq[0], 1, 0)
    r = oracle.propagate_one(w8.pes, w8.gamma, w8.p_eq[0], w8.q_eq[0], w8.dt, w8.n_steps, p0[:, 0], q0[:, 0])
    M = r["M"]
    J = _J(24)
    assert r["good"]
    assert np.max(np.abs(M.T @ J @ M - J)) / max(1.0, np.max(np.abs(M)) ** 2) < 1e-12
    assert abs(r["detM"][-1] - 1.0) < 1e-9


def test_harmonic_prefactor_limits_with_frequency_widths():
    """With gamma = omega: |C_t| -> 1 and phi_t -> -sum omega t / 2 as dt -> 0 (O((omega dt)^4))."""
    omegas = wl.cm1([1600.0, 3650.0])
    pes = wl.harmonic_pes(omegas)
    T = 4000.0
    errs = []
    for dt in (10.0, 5.0):
        n = int(T / dt)
        r = oracle.propagate_one(pes, omegas, np.sqrt(omegas), np.zeros(2), dt, n,
                                 np.sqrt(omegas) + 0.01, np.array([1.0, -2.0]))
        phi = 0.5 * r["theta"][-1]
        errs.append((abs(abs(r["detA"][-1]) - 1.0), abs(phi + 0.5 * np.sum(omegas) * T)))
    # fourth order: halving dt divides the modulus defect and the phase drift by ~16
    assert errs[0][0] / errs[1][0] > 12
    assert errs[0][1] / errs[1][1] > 12
    assert errs[0][0] < 1e-3


def _anharmonic(F=3, seed=1):
    return wl.recipe_pes(F, np.random.default_rng(seed), sigma3=3e-8, sigma4=3e-9)


def _start(pes, seed=2):
    """A typical Husimi-like starting point (about one sigma from chi) for the surface's modes."""
    rng = np.random.default_rng(seed)
    om = pes.omega
    z = rng.uniform(-1.0, 1.0, (2, pes.F))
    return np.sqrt(om) * (1.0 + z[0]), z[1] / np.sqrt(om), om


@pytest.mark.parametrize("F", [2, 3, 6])
def test_monodromy_is_symplectic(F):
    pes = _anharmonic(F)
    p0, q0, om = _start(pes)
    r = oracle.propagate_one(pes, om, np.sqrt(om), np.zeros(F), 10.0, 3000, p0, q0)
    M = r["M"]
    J = _J(F)
    defect = np.max(np.abs(M.T @ J @ M - J)) / max(1.0, np.max(np.abs(M)) ** 2)
    assert defect < 1e-10, defect
    assert abs(r["detM"][-1] - 1.0) < 1e-9


def test_prefactor_matrix_is_the_analytic_block_of_the_monodromy():
    """The Herman-Kluk matrix with unequal widths on a coupled surface (reading of the
    garbled Gamma ordering).  In z = (Gamma^1/2 q + i Gamma^-1/2 p)/sqrt 2 a linear
    symplectic map is z' = A z + B z* with
      A = (G Mqq G^-1 + G^-1 Mpp G - i G Mqp G + i G^-1 Mpq G^-1) / 2,
      B = (G Mqq G^-1 - G^-1 Mpp G + i G Mqp G + i G^-1 Mpq G^-1) / 2   (G = Gamma^1/2),
    and symplecticity is A A^+ - B B^+ = I, A B^T = B A^T.  Both identities hold for
    the oracle's monodromy, and its det A is the determinant of that A; the transposed
    width ordering of the diagonal blocks breaks the identities by 2e-2 to 0.5 and
    changes det A by up to 26 %."""
    F = 3
    pes = _anharmonic(F)
    om = pes.omega
    G, Gi = np.diag(np.sqrt(om)), np.diag(1.0 / np.sqrt(om))
    rng = np.random.default_rng(2)
    for _ in range(5):
        z = rng.uniform(-1.0, 1.0, (2, F))
        p0, q0 = np.sqrt(om) * (1.0 + z[0]), z[1] / np.sqrt(om)
        r = oracle.propagate_one(pes, om, np.sqrt(om), np.zeros(F), 10.0, 1500, p0, q0)
        assert r["good"]
        M = r["M"]
        Mpp, Mpq, Mqp, Mqq = M[:F, :F], M[:F, F:], M[F:, :F], M[F:, F:]
        A = 0.5 * (G @ Mqq @ Gi + Gi @ Mpp @ G - 1j * G @ Mqp @ G + 1j * Gi @ Mpq @ Gi)
        B = 0.5 * (G @ Mqq @ Gi - Gi @ Mpp @ G + 1j * G @ Mqp @ G + 1j * Gi @ Mpq @ Gi)
        s = np.max(np.abs(A)) ** 2
        assert np.max(np.abs(A @ A.conj().T - B @ B.conj().T - np.eye(F))) < 1e-12 * s
        assert np.max(np.abs(A @ B.T - B @ A.T)) < 1e-12 * s
        dA = np.linalg.det(A)
        assert abs(dA - r["detA"][-1]) < 1e-12 * abs(dA)
        assert abs(dA) >= 1.0                       # singular values of A are >= 1


def _energy(pes, p, q):
    return 0.5 * np.sum(p * p) + oracle.pes_eval(pes, q)[0]


def test_energy_conservation_is_fourth_order():
    F = 3
    pes = _anharmonic(F)
    p0, q0, om = _start(pes)
    E0 = _energy(pes, p0, q0)
    T = 20000.0
    errs = []
    for dt in (20.0, 10.0):
        r = oracle.propagate_one(pes, om, np.sqrt(om), np.zeros(F), dt, int(T / dt), p0, q0)
        errs.append(abs(_energy(pes, r["p"], r["q"]) - E0) / abs(E0))
    assert errs[1] < 1e-5
    assert errs[0] / errs[1] > 10.0, errs


def test_time_reversal():
    F = 3
    pes = _anharmonic(F)
    p0, q0, om = _start(pes)
    chi = (np.sqrt(om), np.zeros(F))
    fw = oracle.propagate_one(pes, om, *chi, 10.0, 2000, p0, q0)
    bw = oracle.propagate_one(pes, om, *chi, 10.0, 2000, -fw["p"], fw["q"])
    assert np.allclose(bw["q"], q0, rtol=0, atol=1e-9 * np.max(np.abs(q0)))
    assert np.allclose(-bw["p"], p0, rtol=0, atol=1e-9 * np.max(np.abs(p0)))
    assert abs(bw["S"][-1] - fw["S"][-1]) < 1e-9 * max(1.0, abs(fw["S"][-1]))


def test_monodromy_matches_finite_differences():
    F = 3
    pes = _anharmonic(F)
    p0, q0, om = _start(pes)
    chi = (np.sqrt(om), np.zeros(F))
    n = 800
    r = oracle.propagate_one(pes, om, *chi, 10.0, n, p0, q0)
    M_fd = np.zeros((2 * F, 2 * F))
    for col in range(2 * F):
        h = 1e-5 * (np.sqrt(om[col % F]) if col < F else 1.0 / np.sqrt(om[col % F]))
        dp = np.zeros(F); dq = np.zeros(F)
        (dp if col < F else dq)[col % F] = h
        a = oracle.propagate_one(pes, om, *chi, 10.0, n, p0 + dp, q0 + dq)
        b = oracle.propagate_one(pes, om, *chi, 10.0, n, p0 - dp, q0 - dq)
        M_fd[:, col] = np.concatenate([a["p"] - b["p"], a["q"] - b["q"]]) / (2 * h)
    rel = np.max(np.abs(M_fd - r["M"])) / np.max(np.abs(r["M"]))
    assert rel < 1e-7, rel


def test_fourth_order_convergence_of_the_flow():
    F = 3
    pes = _anharmonic(F)
    p0, q0, om = _start(pes)
    chi = (np.sqrt(om), np.zeros(F))
    T = 3000.0
    sols = []
    for dt in (20.0, 10.0, 5.0):
        r = oracle.propagate_one(pes, om, *chi, dt, int(round(T / dt)), p0, q0)
        sols.append(np.concatenate([r["p"], r["q"]]))
    e1 = np.max(np.abs(sols[0] - sols[1]))
    e2 = np.max(np.abs(sols[1] - sols[2]))
    assert 12.0 < e1 / e2 < 20.0, e1 / e2


def test_action_is_a_generating_function():
    """dS_T = p_T . dq_T - p_0 . dq_0 (holds exactly for compositions of exact sub-flows)."""
    F = 3
    pes = _anharmonic(F)
    p0, q0, om = _start(pes)
    chi = (np.sqrt(om), np.zeros(F))
    n = 600
    r = oracle.propagate_one(pes, om, *chi, 10.0, n, p0, q0)
    M = r["M"]
    Mqp, Mqq = M[F:, :F], M[F:, F:]
    dS_dp0 = r["p"] @ Mqp
    dS_dq0 = r["p"] @ Mqq - p0
    for i in range(F):
        for which, ref in (("p", dS_dp0[i]), ("q", dS_dq0[i])):
            h = 1e-5 * (np.sqrt(om[i]) if which == "p" else 1 / np.sqrt(om[i]))
            d = np.zeros(F); d[i] = h
            if which == "p":
                a = oracle.propagate_one(pes, om, *chi, 10.0, n, p0 + d, q0)
                b = oracle.propagate_one(pes, om, *chi, 10.0, n, p0 - d, q0)
            else:
                a = oracle.propagate_one(pes, om, *chi, 10.0, n, p0, q0 + d)
                b = oracle.propagate_one(pes, om, *chi, 10.0, n, p0, q0 - d)
            fd = (a["S"][-1] - b["S"][-1]) / (2 * h)
            assert abs(fd - ref) < 1e-6 * max(1.0, abs(ref)), (which, i, fd, ref)


def test_stability_threshold_direction():
    F = 3
    pes = _anharmonic(F)
    p0, q0, om = _start(pes)
    chi = (np.sqrt(om), np.zeros(F))
    assert oracle.propagate_one(pes, om, *chi, 10.0, 300, p0, q0, stab_tol=1.0)["good"]
    # rounding alone moves det M off 1 by more than 1e-300
    assert not oracle.propagate_one(pes, om, *chi, 10.0, 300, p0, q0, stab_tol=1e-300)["good"]


def test_stability_quantity_is_det_squared_minus_one():
    """The monitored quantity is |det(M^T M) - 1| = |det(M)^2 - 1| (reading of Sec. II),
    tested every step and sticky: with D its largest value along the trajectory (from the
    det M series, itself pinned against LAPACK), a tolerance of 0.75 D flags the
    trajectory bad and 1.25 D keeps it good.  Monitoring |det M - 1|, about D / 2,
    would keep it good at 0.75 D."""
    F = 3
    pes = _anharmonic(F)
    p0, q0, om = _start(pes)
    chi = (np.sqrt(om), np.zeros(F))
    r = oracle.propagate_one(pes, om, *chi, 10.0, 2000, p0, q0, stab_tol=1.0)
    D = np.max(np.abs(r["detM"][1:] ** 2 - 1.0))
    assert D > 1e-14
    assert not oracle.propagate_one(pes, om, *chi, 10.0, 2000, p0, q0, stab_tol=0.75 * D)["good"]
    assert oracle.propagate_one(pes, om, *chi, 10.0, 2000, p0, q0, stab_tol=1.25 * D)["good"]


def test_runaway_trajectory_is_flagged_bad():
    # a strongly negative quartic coupling makes large-amplitude motion escape to infinity
    F = 2
    om = wl.cm1([1500.0, 2500.0])
    pes = wl.morse_pes(om, 0.2, idx4=np.array([[0, 0, 1, 1]]), c4=np.array([-1e-3]))
    r = oracle.propagate_one(pes, om, np.sqrt(om), np.zeros(F), 10.0, 400,
                             np.array([2.0, 2.0]), np.array([5.0, 5.0]))
    assert not r["good"]


def test_non_finite_initial_condition_is_flagged_and_excluded():
    """A NaN or infinite starting coordinate gives a bad trajectory (never a crash), and
    the spectrum over the set equals the spectrum of the set without that trajectory."""
    w8 = wl.config_f3(n_traj=12, n_steps=200, n_E=120)
    p0, q0, w = oracle.sample_initial(w8.gamma, w8.p_eq, w8.q_eq, w8.n_traj, 4)
    p0[1, 3] = np.nan
    q0[2, 7] = np.inf
    amp, good = oracle.propagate(w8.pes, w8.gamma, w8.p_eq, w8.q_eq, w8.dt, w8.n_steps, p0, q0)
    assert good[3] == 0 and good[7] == 0 and good.sum() == w8.n_traj - 2
    I, ng = oracle.spectrum(amp[0], w, good, w8.n_steps, w8.dt, w8.E_min, w8.E_max, w8.n_E)
    keep = np.setdiff1d(np.arange(w8.n_traj), [3, 7])
    I2, ng2 = oracle.spectrum(np.ascontiguousarray(amp[0][keep]), w[keep], good[keep], w8.n_steps, w8.dt,
                              w8.E_min, w8.E_max, w8.n_E)
    assert ng == ng2 == w8.n_traj - 2
    assert np.all(np.isfinite(I))
    assert np.max(np.abs(I - I2)) <= 1e-14 * np.max(np.abs(I2))


def test_batch_matches_single_and_chi_layout():
    F = 3
    pes = _anharmonic(F)
    om = wl.cm1([1600.0, 3650.0, 3750.0])
    p_eq = np.stack([np.sqrt(om), np.sqrt(3 * om)])
    q_eq = np.zeros((2, F))
    p0, q0, w = oracle.sample_initial(om, p_eq[0], q_eq[0], 7, 1)
    amp, good = oracle.propagate(pes, om, p_eq, q_eq, 10.0, 50, p0, q0)
    assert amp.shape == (2, 7, 51)
    for j in range(7):
        r = oracle.propagate_one(pes, om, p_eq, q_eq, 10.0, 50, p0[:, j], q0[:, j])
        assert np.array_equal(r["amp"], amp[:, j, :], equal_nan=True)
        assert r["good"] == bool(good[j])


@pytest.mark.parametrize("sigma", [(3e-8, 3e-9), (5e-8, 5e-9)])
def test_chunk_end_stability_cadence_selects_the_per_step_good_set(sigma):
    """The mixed-precision kernels test det M every C = 16 steps (and at the last step)
    instead of every step (Sec. II, Sec. III.A: a trajectory is discarded as
    soon as |det(M^T M) - 1| exceeds the tolerance; the flag is sticky and the whole
    trajectory is dropped).  On the oracle's own per-step det M series, over surfaces
    where about half the trajectories go bad (couplings on mass-weighted q), the
    chunk-end test with C = 8 and 16 must keep exactly the trajectories the per-step
    test keeps, at the FP64 threshold and at the mixed path's FP32 one."""
    rng = np.random.default_rng(3)
    pes = wl.recipe_pes(6, rng, sigma3=sigma[0], sigma4=sigma[1], units=wl.COUPLING_MASS_WEIGHTED)
    p_eq, q_eq = wl.ground_chi(pes.omega)
    n, n_steps = 96, 600
    p0, q0, _ = oracle.sample_initial(pes.omega, p_eq, q_eq, n, 5)
    dev = np.empty((n, n_steps))
    for j in range(n):
        r = oracle.propagate_one(pes, pes.omega, p_eq, q_eq, 10.0, n_steps, p0[:, j], q0[:, j])
        d = r["detM"][1:]
        dev[j] = np.where(np.isfinite(d), np.abs(d * d - 1.0), np.inf)
    for tol in (1e-6, 1e-6 * 2.0 ** 29):
        every = ~(dev > tol).any(axis=1)
        assert 0 < every.sum() < n
        for C in (8, 16):
            ends = np.r_[np.arange(C - 1, n_steps, C), n_steps - 1]
            chunk = ~(dev[:, ends] > tol).any(axis=1)
            assert np.array_equal(every, chunk), (tol, C, np.flatnonzero(every != chunk))
