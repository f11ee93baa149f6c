"""Plain Herman-Kluk SC-IVR on the GPU (Eq. I(E)_SCIVR): the per-trajectory
summands C_t e^{iS_t} <chi|p_t q_t> / <chi|p0 q0> that scivr_propagate records
with SCIVR_AMP_HK (a further reference state chi_x on the same trajectories:
C_t e^{iS_t} <chi_x|p_t q_t> <p0 q0|chi_x> / |<p0 q0|chi_0>|^2), and the survival-amplitude spectrum of scivr_spectrum_hk,
against the FP64 oracle element by element and against closed forms.

Tolerances follow those of the time-averaged path: FP64 summands to 1e-9 of a
trajectory's largest summand (rounding order differs between the two
implementations; errors grow along the trajectory), mixed precision to 5e-2;
the spectrum step alone on identical inputs to 1e-12 relative (a sum of K
FP64 terms, each with one rounding of the phase E c dt).
"""
import numpy as np
import pytest

import oracle
from paper_1312_4698_gb300 import workloads as wl
from tests.test_gpu_parity import MIXED_STAB_TOL, amp_err, check_flags

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    from paper_1312_4698_gb300 import scivr
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return scivr


def _t(x, dtype=None):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda", dtype=dtype)


def hk_propagate(G, w8, p0, q0, precision=0, kernel=0, stab_tol=None, fin=False):
    import torch
    F, n = p0.shape
    K = w8.n_steps + 1
    pes = G.scivr_create_pes(w8.pes)
    amp = torch.empty((w8.n_chi, n, K, 2), dtype=torch.float64, device="cuda")
    good = torch.empty(n, dtype=torch.uint8, device="cuda")
    fd = dict(stab=torch.empty(n, dtype=torch.float64, device="cuda")) if fin else None
    tol = w8.stab_tol if stab_tol is None else stab_tol
    G.scivr_propagate(pes, w8.dt, w8.n_steps, w8.gamma, w8.p_eq, w8.q_eq, n, _t(p0), _t(q0), amp, K, good,
                      precision=precision, stab_tol=tol, kernel=kernel, fin=fd, amplitude=G.SCIVR_AMP_HK)
    torch.cuda.synchronize()
    assert G.scivr_check_status() == G.SCIVR_OK
    a = amp.cpu().numpy()
    out = dict(amp=np.ascontiguousarray(a).view(np.complex128)[..., 0], good=good.cpu().numpy(), dev_amp=amp, dev_good=good)
    if fin:
        out["stab"] = fd["stab"].cpu().numpy()
    return out


def hk_spectrum(G, amp, good, n_steps, dt, E_min, E_max, n_E):
    """amp: device [n, K, 2] float64 or a complex numpy array."""
    import torch
    if isinstance(amp, np.ndarray):
        amp = _t(np.stack([amp.real, amp.imag], axis=-1))
    if isinstance(good, np.ndarray):
        good = _t(good.astype(np.uint8))
    n, K = amp.shape[0], amp.shape[1]
    I = torch.empty(n_E, dtype=torch.float64, device="cuda")
    C = torch.empty((K, 2), dtype=torch.float64, device="cuda")
    ng = torch.zeros(1, dtype=torch.int64, device="cuda")
    G.scivr_spectrum_hk(amp, K, good, n, n_steps, dt, E_min, E_max, n_E, I, C, ng)
    torch.cuda.synchronize()
    c = C.cpu().numpy()
    return I.cpu().numpy(), int(ng.cpu().item()), c[:, 0] + 1j * c[:, 1]


@pytest.mark.parametrize("F,kernel", [(1, 1), (3, 1), (6, 1), (9, 1), (1, 2), (3, 2), (6, 2), (9, 2)])
def test_hk_summands_match_oracle(G, F, kernel):
    """FP64, both schedules: 70 trajectories (ragged for every block shape) and
    301 steps (not a multiple of any chunk length)."""
    w8 = wl.config_f3(n_traj=70, n_steps=301) if F == 3 else wl.config_generic(F, seed=F, n_traj=70, n_steps=301)
    p0, q0, w = oracle.sample_initial(w8.gamma, w8.p_eq, w8.q_eq, w8.n_traj, 11)
    ra, rg, rf = oracle.propagate(w8.pes, w8.gamma, w8.p_eq, w8.q_eq, w8.dt, w8.n_steps, p0, q0, final=True,
                                  amplitude=oracle.AMP_HK)
    g = hk_propagate(G, w8, p0, q0, kernel=kernel, fin=True)
    check_flags(g["good"], g["stab"], rg, rf["stab"])
    sel = g["good"].astype(bool) & rg.astype(bool)
    assert np.all(g["amp"][:, :, 0] == 1.0)                     # t = 0: exactly 1 on every row
    assert amp_err(g["amp"][:, sel], ra[:, sel], np.ones(sel.sum(), np.uint8)) < 1e-9


def test_hk_summands_several_reference_states(G):
    w8 = wl.config_f3(n_traj=33, n_steps=200)
    om = w8.gamma
    w8 = w8.with_(p_eq=np.stack([np.sqrt(om), np.sqrt(3 * om), -np.sqrt(om)]),
                  q_eq=np.stack([np.zeros(3), np.zeros(3), np.array([1.0, -2.0, 0.5])]))
    p0, q0, w = oracle.sample_initial(w8.gamma, w8.p_eq[0], w8.q_eq[0], w8.n_traj, 5)
    ra, rg = oracle.propagate(w8.pes, w8.gamma, w8.p_eq, w8.q_eq, w8.dt, w8.n_steps, p0, q0,
                              amplitude=oracle.AMP_HK)
    for kernel in (1, 2):
        g = hk_propagate(G, w8, p0, q0, kernel=kernel)
        assert g["amp"].shape == (3, 33, 201)
        assert amp_err(g["amp"], ra, rg) < 1e-9


@pytest.mark.parametrize("F", [3, 6, 9])
def test_hk_summands_mixed_precision(G, F):
    w8 = wl.config_f3(n_traj=64, n_steps=400) if F == 3 else wl.config_generic(F, seed=F, n_traj=64, n_steps=400)
    p0, q0, w = oracle.sample_initial(w8.gamma, w8.p_eq, w8.q_eq, w8.n_traj, 3)
    ra, rg = oracle.propagate(w8.pes, w8.gamma, w8.p_eq, w8.q_eq, w8.dt, w8.n_steps, p0, q0,
                              amplitude=oracle.AMP_HK)
    g = hk_propagate(G, w8, p0, q0, precision=1, stab_tol=MIXED_STAB_TOL)
    sel = rg.astype(bool) & g["good"].astype(bool)
    assert sel.sum() >= 0.95 * rg.sum()
    assert amp_err(g["amp"][:, sel], ra[:, sel], np.ones(sel.sum(), np.uint8)) < 5e-2


def test_hk_summands_harmonic_ground_state_closed_form(G):
    """chi = the ground state of a harmonic surface (gamma = omega, chi at the
    origin): every exact summand is e^{-i E0 t}, E0 = sum omega / 2; the
    fourth-order integrator at dt = 5 stays within 2e-3 over 400 steps.  GPU
    against the closed form directly, both schedules."""
    omega = wl.cm1([1600.0, 3000.0])
    zero = np.zeros((1, 2))
    w8 = wl.Workload("harm", wl.harmonic_pes(omega), omega, zero, zero, 64, 400, 5.0, 0.0, 0.1, 10, 0)
    p0, q0, w = oracle.sample_initial(omega, zero[0], zero[0], 64, 3)
    t = w8.dt * np.arange(w8.n_steps + 1)
    exact = np.exp(-0.5j * omega.sum() * t)
    for kernel in (1, 2):
        g = hk_propagate(G, w8, p0, q0, kernel=kernel)
        assert g["good"].all()
        assert np.max(np.abs(g["amp"][0] - exact[None, :])) < 2e-3


def test_hk_surrogate_path_matches_oracle(G):
    """The learned-residual split-step path records the same summand."""
    from tests.test_gpu_mlp import _diag_only
    F, n = 3, 64
    w8 = wl.config_f3(n_traj=n, n_steps=300)
    pes = _diag_only(w8.pes)
    m = wl.init_mlp(F, 256, 3, s_in=np.sqrt(w8.gamma), s_out=2e-4)
    pes.mlp = m
    w8.pes = pes
    p0, q0, w = oracle.sample_initial(w8.gamma, w8.p_eq[0], w8.q_eq[0], n, 0)
    ta, tg = oracle.propagate(pes, w8.gamma, w8.p_eq, w8.q_eq, w8.dt, w8.n_steps, p0, q0)
    ra, rg = oracle.propagate(pes, w8.gamma, w8.p_eq, w8.q_eq, w8.dt, w8.n_steps, p0, q0, amplitude=oracle.AMP_HK)
    g = hk_propagate(G, w8, p0, q0, precision=1, stab_tol=MIXED_STAB_TOL)
    assert rg.all() and g["good"].all()
    e = amp_err(g["amp"], ra, rg)
    print(f"surrogate HK summands: max error {e:.2e}")
    # same bound as the time-averaged integrand of this surface (BF16 network, FP32 monodromy)
    assert e < 5e-2


@pytest.mark.parametrize("n,n_steps,n_E", [(1, 1, 2), (130, 50, 77), (4096, 255, 64), (9001, 600, 301)])
def test_hk_spectrum_matches_oracle(G, n, n_steps, n_E):
    """Random summands with excluded rows holding NaN: the row count spans
    several 4096-row slices with a ragged tail, K several 256-column blocks."""
    rng = np.random.default_rng(n + n_steps)
    K = n_steps + 1
    amp = (rng.normal(size=(n, K)) + 1j * rng.normal(size=(n, K))) * 0.3
    good = (rng.uniform(size=n) > 0.2).astype(np.uint8)
    good[0] = 1
    amp[good == 0] = np.nan
    dt, E_min, E_max = 10.0, float(wl.cm1(500.0)), float(wl.cm1(4500.0))
    rI, rng_, rC = oracle.spectrum_hk(amp, good, n_steps, dt, E_min, E_max, n_E)
    gI, gng, gC = hk_spectrum(G, amp, good, n_steps, dt, E_min, E_max, n_E)
    assert gng == rng_ == int(good.sum())
    assert np.max(np.abs(gC - rC)) <= 1e-13 * max(np.max(np.abs(rC)), 1e-300)
    assert np.max(np.abs(gI - rI)) <= 1e-12 * max(np.max(np.abs(rI)), 1e-300)


def test_hk_spectrum_no_good_rows_is_zero(G):
    n, n_steps = 5, 20
    amp = np.full((n, n_steps + 1), np.nan + 1j * np.nan)
    good = np.zeros(n, np.uint8)
    I, ng, C = hk_spectrum(G, amp, good, n_steps, 10.0, 0.0, 0.02, 16)
    assert ng == 0 and np.all(C == 0) and np.all(I == 0)


def test_hk_spectrum_dirichlet_closed_form(G):
    """C(t) = e^{-i E0 t} on every row: the folded rectangle-rule transform is the
    Dirichlet kernel (dt/pi) sin((n+1/2) x) / (2 sin(x/2)), x = (E - E0) dt."""
    dt, n_steps, n = 10.0, 300, 7
    E0 = float(wl.cm1(2000.0))
    t = dt * np.arange(n_steps + 1)
    amp = np.tile(np.exp(-1j * E0 * t), (n, 1))
    E_min, E_max, n_E = float(wl.cm1(1000.0)), float(wl.cm1(3000.0)), 400
    I, ng, C = hk_spectrum(G, amp, np.ones(n, np.uint8), n_steps, dt, E_min, E_max, n_E)
    E = E_min + np.arange(n_E) * ((E_max - E_min) / (n_E - 1))
    x = (E - E0) * dt
    ref = dt / np.pi * np.sin((n_steps + 0.5) * x) / (2 * np.sin(x / 2))
    assert ng == n
    assert np.max(np.abs(I - ref)) <= 1e-10 * np.max(np.abs(ref))


def test_hk_f3_workload_spectrum_peaks_match_oracle(G):
    """The F = 3 workload end to end on the GPU (FP64 propagation, then the HK
    spectrum step on device-resident summands) against the oracle: every peak
    within 0.1 cm^-1 and the spectra within 1e-8 in the max norm."""
    from tests import closed_forms as cf
    w8 = wl.config_f3(n_traj=2048)
    p0, q0, w = oracle.sample_initial(w8.gamma, w8.p_eq, w8.q_eq, w8.n_traj, w8.seed)
    ra, rg = oracle.propagate(w8.pes, w8.gamma, w8.p_eq, w8.q_eq, w8.dt, w8.n_steps, p0, q0,
                              amplitude=oracle.AMP_HK)
    rI, rng_, _ = oracle.spectrum_hk(ra[0], rg, w8.n_steps, w8.dt, w8.E_min, w8.E_max, w8.n_E)
    g = hk_propagate(G, w8, p0, q0)
    # the oracle's good set on both sides: flags that flip sit at the threshold by rounding
    gI, gng, _ = hk_spectrum(G, g["dev_amp"][0], _t(rg), w8.n_steps, w8.dt, w8.E_min, w8.E_max, w8.n_E)
    assert gng == rng_
    E = w8.energies()
    pr = wl.to_cm1(cf.find_peaks(E, rI))
    pg = wl.to_cm1(cf.find_peaks(E, gI))
    print(f"{len(pr)} peaks; max shift {np.max(np.abs(pr - pg)) if len(pr) == len(pg) else float('nan'):.2e} cm^-1")
    assert len(pr) > 0 and len(pr) == len(pg)
    assert np.max(np.abs(pr - pg)) <= 0.1
    assert np.max(np.abs(gI - rI)) <= 1e-8 * np.max(np.abs(rI))


def test_hk_default_workload_full_size_sampled(G):
    """The plain HK configuration bench.py times (--amplitude hk) at its full size and
    launch shape: F = 6, 16384 trajectories x 4000 steps, mixed propagation.  24 sampled
    summand rows (the ragged last one included) against the FP64 oracle within the mixed
    bound, and the HK spectrum of that sample (oracle flags as the good mask) against
    the oracle's: within 3e-2 of its maximum, every oracle peak above 10 % matched
    within 1 cm^-1."""
    import torch
    from tests import closed_forms as cf
    from tests.test_gpu_parity import MIXED_STAB_TOL as TOL
    w8 = wl.config_f6()
    n, K = w8.n_traj, w8.n_steps + 1
    p0, q0, w = oracle.sample_initial(w8.gamma, w8.p_eq, w8.q_eq, n, w8.seed)
    g = hk_propagate(G, w8, p0, q0, precision=1, stab_tol=TOL)
    idx = np.sort(np.random.default_rng(2).choice(n, 24, replace=False))
    idx[-1] = n - 1
    ra, rg = oracle.propagate(w8.pes, w8.gamma, w8.p_eq, w8.q_eq, w8.dt, w8.n_steps, p0[:, idx], q0[:, idx],
                              amplitude=oracle.AMP_HK)
    sel = rg.astype(bool) & g["good"][idx].astype(bool)
    assert sel.sum() >= 22
    e_amp = amp_err(g["amp"][:, idx][:, sel], ra[:, sel], np.ones(sel.sum(), np.uint8))
    print(f"sampled HK rows: max error {e_amp:.2e}")
    assert e_amp < 5e-2
    mask = torch.zeros(n, dtype=torch.uint8, device="cuda")
    mask[torch.as_tensor(idx, device="cuda")] = _t(rg)
    gI, gng, _ = hk_spectrum(G, g["dev_amp"][0], mask, w8.n_steps, w8.dt, w8.E_min, w8.E_max, w8.n_E)
    rI, rng_, _ = oracle.spectrum_hk(ra[0], rg, w8.n_steps, w8.dt, w8.E_min, w8.E_max, w8.n_E)
    assert gng == rng_
    e_s = np.max(np.abs(gI - rI)) / np.max(np.abs(rI))
    E = w8.energies()
    pr = wl.to_cm1(cf.find_peaks(E, rI, 0.1))
    pg = wl.to_cm1(cf.find_peaks(E, gI, 0.02))
    shift = np.array([np.min(np.abs(pg - x)) for x in pr])
    print(f"sample HK spectrum: rel err {e_s:.2e}; {len(pr)} peaks, max shift {shift.max():.3f} cm^-1")
    assert e_s <= 3e-2
    assert len(pr) > 0 and shift.max() <= 1.0
