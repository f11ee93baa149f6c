"""GPU path (through the C ABI) against the FP64 CPU oracle, element by element.

Inputs come from the oracle's sampler or from numpy; nothing the oracle
consumes or is compared with comes from the CUDA path.

Tolerances (FP64 path): rounding differs between the two implementations
(fused multiply-adds, summation order, libm vs CUDA transcendental
functions, reciprocal-multiply instead of division in the LU), so values are
compared with bounds derived from error growth along a trajectory:
amplitudes to 1e-9 of the trajectory's largest amplitude, spectra to 1e-9
relative in the max norm, peak positions to 0.1 cm^-1.
"""
import numpy as np
import pytest

import oracle
from paper_1312_4698_gb300 import workloads as wl
from tests import closed_forms as cf

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


MIXED_STAB_TOL = 1e-6 * 2.0 ** 29   # the FP64 threshold scaled by eps32 / eps64


def gpu_propagate(G, w8, p0, q0, precision=0, fin=False, kernel=0, stab_tol=None):
    import torch
    F, n = p0.shape
    K = w8.n_steps + 1
    pes = G.scivr_create_pes(w8.pes)
    amp = torch.empty((w8.n_chi, n, K, 2), dtype=torch.float64, device="cuda")
    good = torch.empty(n, dtype=torch.uint8, device="cuda")
    fd = None
    if fin:
        fd = dict(p=torch.empty((F, n), dtype=torch.float64, device="cuda"),
                  q=torch.empty((F, n), dtype=torch.float64, device="cuda"),
                  S=torch.empty(n, dtype=torch.float64, device="cuda"),
                  theta=torch.empty(n, dtype=torch.float64, device="cuda"),
                  detM=torch.empty(n, dtype=torch.float64, device="cuda"),
                  detA=torch.empty((n, 2), dtype=torch.float64, device="cuda"),
                  M=torch.empty((n, 2 * F, 2 * F), dtype=torch.float64, device="cuda"),
                  stab=torch.empty(n, dtype=torch.float64, device="cuda"))
    tol = w8.stab_tol if stab_tol is None else stab_tol
    G.scivr_propagate(pes, w8.dt, w8.n_steps, w8.gamma, w8.p_eq, w8.q_eq, n, _t(p0), _t(q0), amp, K,
                      good, precision=precision, stab_tol=tol, fin=fd, kernel=kernel)
    torch.cuda.synchronize()
    a = amp.cpu().numpy()
    a = np.ascontiguousarray(a).view(np.complex128)[..., 0]
    out = dict(amp=a, good=good.cpu().numpy())
    if fin:
        out.update({k: v.cpu().numpy() for k, v in fd.items()})
    return out


def gpu_spectrum(G, amp, w, good, n_steps, dt, E_min, E_max, n_E):
    import torch
    n, K = amp.shape
    a = np.stack([amp.real, amp.imag], axis=-1)
    I = torch.empty(n_E, dtype=torch.float64, device="cuda")
    ng = torch.zeros(1, dtype=torch.int64, device="cuda")
    G.scivr_spectrum(_t(a), K, _t(w), _t(good.astype(np.uint8)), n, n_steps, dt, E_min, E_max, n_E, I, ng)
    torch.cuda.synchronize()
    return I.cpu().numpy(), int(ng.cpu().item())


STAB_BAND = 10.0


def check_flags(g_good, g_stab, r_good, r_stab, tol=1e-6):
    """Good flags must agree except for trajectories whose stability measure
    max |det(M)^2 - 1| sits within a factor STAB_BAND of the threshold on BOTH
    sides: there the measure is accumulated rounding error, which differs
    between any two FP64 implementations (summation order, FMA contraction).
    Returns the indices of the flipped trajectories."""
    flips = np.flatnonzero(np.asarray(g_good).astype(bool) != np.asarray(r_good).astype(bool))
    for j in flips:
        assert tol / STAB_BAND <= r_stab[j] <= tol * STAB_BAND, (j, r_stab[j])
        assert tol / STAB_BAND <= g_stab[j] <= tol * STAB_BAND, (j, g_stab[j])
    assert len(flips) <= max(1, len(r_good) // 100)
    return flips


def amp_err(a, b, good):
    """Max over good trajectories of |a - b| / max_c |b|."""
    sel = good.astype(bool)
    if not sel.any():
        return 0.0
    scale = np.max(np.abs(b[..., sel, :]), axis=-1, keepdims=True)
    return float(np.max(np.abs(a[..., sel, :] - b[..., sel, :]) / scale))


def test_sampler_matches_oracle(G):
    import torch
    w8 = wl.config_f6(n_traj=1000)
    n = 1000
    pes = G.scivr_create_pes(w8.pes)
    p0 = torch.empty((6, n), dtype=torch.float64, device="cuda")
    q0 = torch.empty_like(p0)
    w = torch.empty(n, dtype=torch.float64, device="cuda")
    G.scivr_sample_initial(pes, w8.gamma, w8.p_eq[0], w8.q_eq[0], n, 12345, p0, q0, w)
    torch.cuda.synchronize()
    rp, rq, rw = oracle.sample_initial(w8.gamma, w8.p_eq[0], w8.q_eq[0], n, 12345)
    assert np.allclose(p0.cpu().numpy(), rp, rtol=1e-13, atol=1e-15)
    assert np.allclose(q0.cpu().numpy(), rq, rtol=1e-13, atol=1e-13)
    assert np.allclose(w.cpu().numpy(), rw, rtol=1e-12)


@pytest.mark.parametrize("F,kernel", [(F, 1) for F in range(1, 10)] + [(F, 2) for F in range(1, 10)])
def test_propagate_matches_oracle_small(G, F, kernel):
    """FP64 path, both schedules (1 = thread per trajectory, 2 = lane group),
    every supported F; 70 trajectories (ragged w.r.t. any block size) and a
    step count that is not a multiple of the group's chunk length."""
    if F == 3:
        w8 = wl.config_f3(n_traj=70, n_steps=301)
    else:
        w8 = wl.config_generic(F, seed=F, n_traj=70, n_steps=301)
    p0, q0, w = oracle.sample_initial(w8.gamma, w8.p_eq, w8.q_eq, w8.n_traj, 11)
    ra, rg, rf = oracle.propagate(w8.pes, w8.gamma, w8.p_eq, w8.q_eq, w8.dt, w8.n_steps, p0, q0,
                                  final=True)
    g = gpu_propagate(G, w8, p0, q0, fin=True, kernel=kernel)
    check_flags(g["good"], g["stab"], rg, rf["stab"])
    assert amp_err(g["amp"], ra, rg) < 1e-9
    sel = rg.astype(bool)
    assert np.allclose(g["p"][:, sel], rf["p"].T[:, sel], rtol=1e-9, atol=1e-12)
    assert np.allclose(g["q"][:, sel], rf["q"].T[:, sel], rtol=1e-9, atol=1e-9)
    assert np.allclose(g["S"][sel], rf["S"][sel], rtol=1e-9, atol=1e-9)
    assert np.allclose(g["theta"][sel], rf["theta"][sel], rtol=1e-9, atol=1e-9)
    assert np.allclose(g["M"][sel], rf["M"][sel], rtol=1e-8, atol=1e-8 * np.max(np.abs(rf["M"][sel])))
    dA = g["detA"][:, 0] + 1j * g["detA"][:, 1]
    assert np.allclose(dA[sel], rf["detA"][sel], rtol=1e-9)
    assert np.allclose(g["detM"][sel], rf["detM"][sel], rtol=0, atol=1e-9)


def test_propagate_several_reference_states(G):
    w8 = wl.config_f3(n_traj=33, n_steps=200)
    om = w8.gamma
    w8 = w8.with_(p_eq=np.stack([np.sqrt(om), np.sqrt(3 * om), -np.sqrt(om)]),
                  q_eq=np.stack([np.zeros(3), np.zeros(3), np.array([1.0, -2.0, 0.5])]))
    p0, q0, w = oracle.sample_initial(w8.gamma, w8.p_eq[0], w8.q_eq[0], w8.n_traj, 5)
    ra, rg = oracle.propagate(w8.pes, w8.gamma, w8.p_eq, w8.q_eq, w8.dt, w8.n_steps, p0, q0)
    g = gpu_propagate(G, w8, p0, q0)
    assert g["amp"].shape == (3, 33, 201)
    assert amp_err(g["amp"], ra, rg) < 1e-9


def test_propagate_harmonic_closed_form(G):
    """GPU amplitudes against the Glauber closed form directly (not via the oracle)."""
    omegas = wl.cm1([1600.0, 3650.0, 3750.0])
    dt, n_steps = 10.0, 800
    gts = np.array([cf.harmonic_rotation(w, dt)[1] for w in omegas])
    w8 = wl.Workload("harm", wl.harmonic_pes(omegas), gts, np.sqrt(gts)[None], np.zeros((1, 3)),
                     5, n_steps, dt, 0.0, 0.1, 10, 0)
    rng = np.random.default_rng(9)
    q0 = rng.normal(0, 1, (3, 5)) / np.sqrt(gts)[:, None]
    p0 = np.sqrt(gts)[:, None] * (1 + rng.normal(0, 1, (3, 5)))
    g = gpu_propagate(G, w8, p0, q0)
    assert g["good"].all()
    for j in range(5):
        ref, _, _ = cf.harmonic_amplitude(omegas, dt, n_steps, p0[:, j], q0[:, j], np.sqrt(gts), np.zeros(3))
        assert np.max(np.abs(g["amp"][0, j] - ref)) < 1e-10


def test_bad_trajectories_flagged_like_the_oracle(G):
    """Strong couplings: a mix of escaping (non-finite) and stable trajectories."""
    w8 = wl.config_generic(6, seed=1, n_traj=96, n_steps=500)
    rng = np.random.default_rng(1)
    w8.pes = wl.recipe_pes(6, rng, sigma3=1e-7, sigma4=1e-8)   # mass-weighted: many escape
    p0, q0, w = oracle.sample_initial(w8.gamma, w8.p_eq, w8.q_eq, w8.n_traj, 2)
    p0[0, 5] = np.nan    # injected non-finite initial condition -> bad, not a fault
    ra, rg, rf = oracle.propagate(w8.pes, w8.gamma, w8.p_eq, w8.q_eq, w8.dt, w8.n_steps, p0, q0,
                                  final=True)
    g = gpu_propagate(G, w8, p0, q0, fin=True)
    assert 0 < rg.sum() < rg.size
    assert g["good"][5] == 0 and rg[5] == 0
    assert np.isinf(g["stab"][5]) and np.isinf(rf["stab"][5])
    check_flags(g["good"], g["stab"], rg, rf["stab"])
    assert amp_err(g["amp"], ra, rg) < 1e-9


@pytest.mark.parametrize("n,n_steps,n_E", [(1, 1, 2), (130, 50, 77), (64, 15, 64), (257, 100, 130)])
def test_spectrum_matches_oracle_random_amplitudes(G, n, n_steps, n_E):
    rng = np.random.default_rng(n + n_steps)
    K = n_steps + 1
    amp = (rng.normal(size=(n, K)) + 1j * rng.normal(size=(n, K))) * 0.3
    w = rng.uniform(0.2, 5.0, n)
    good = (rng.uniform(size=n) > 0.2).astype(np.uint8)
    good[0] = 1
    bad = np.flatnonzero(good == 0)
    if bad.size:
        amp[bad[0], 3 % K] = np.nan          # bad rows must not leak NaN
    dt, E_min, E_max = 10.0, 0.001, 0.06
    ri, rng_ = oracle.spectrum(amp, w, good, n_steps, dt, E_min, E_max, n_E)
    gi, gng = gpu_spectrum(G, amp, w, good, n_steps, dt, E_min, E_max, n_E)
    assert gng == rng_
    assert np.max(np.abs(gi - ri)) <= 1e-12 * np.max(np.abs(ri))


def test_spectrum_all_bad_is_zero(G):
    amp = np.ones((5, 11), dtype=complex)
    gi, ng = gpu_spectrum(G, amp, np.ones(5), np.zeros(5, np.uint8), 10, 10.0, 0.0, 0.1, 9)
    assert ng == 0 and np.all(gi == 0.0)


def _full_path(G, w8, p0, q0, w, stab=False):
    import torch
    n = p0.shape[1]
    K = w8.n_steps + 1
    pes = G.scivr_create_pes(w8.pes)
    bufs = G.alloc_buffers(w8, n_traj=n)
    bufs.p0.copy_(_t(p0))
    bufs.q0.copy_(_t(q0))
    bufs.w.copy_(_t(w))
    st = torch.empty(n, dtype=torch.float64, device="cuda")
    G.scivr_propagate(pes, w8.dt, w8.n_steps, w8.gamma, w8.p_eq, w8.q_eq, n, bufs.p0, bufs.q0,
                      bufs.amp, K, bufs.good, stab_tol=w8.stab_tol, fin=dict(stab=st))
    for x in range(w8.n_chi):
        G.scivr_spectrum(bufs.amp[x], K, bufs.w, bufs.good, n, w8.n_steps, w8.dt, w8.E_min,
                         w8.E_max, w8.n_E, bufs.I[x], bufs.n_good)
    torch.cuda.synchronize()
    bufs.stab = st.cpu().numpy()
    return bufs


def test_config_f3_full_spectrum_matches_oracle(G):
    """F=3 workload at its full size: 1024 trajectories, 3000 steps, 2000 energies.

    Flags are compared with check_flags; the spectra are compared on the
    oracle's good set (the oracle's flags feed the GPU spectrum, never the
    other way round), to 1e-9 relative and 0.1 cm^-1 per peak."""
    import torch
    w8 = wl.config_f3()
    p0, q0, w = oracle.sample_initial(w8.gamma, w8.p_eq, w8.q_eq, w8.n_traj, w8.seed)
    ra, rg, rf = oracle.propagate(w8.pes, w8.gamma, w8.p_eq, w8.q_eq, w8.dt, w8.n_steps, p0, q0,
                                  final=True)
    ri, rng_ = oracle.spectrum(ra[0], w, rg, w8.n_steps, w8.dt, w8.E_min, w8.E_max, w8.n_E)
    bufs = _full_path(G, w8, p0, q0, w)
    gg = bufs.good.cpu().numpy()
    flips = check_flags(gg, bufs.stab, rg, rf["stab"])
    assert int(bufs.n_good.item()) == rng_ + int(np.sum(gg[flips])) - int(np.sum(rg[flips]))
    I = torch.empty(w8.n_E, dtype=torch.float64, device="cuda")
    ng = torch.zeros(1, dtype=torch.int64, device="cuda")
    G.scivr_spectrum(bufs.amp[0], w8.n_steps + 1, bufs.w, _t(rg), w8.n_traj, w8.n_steps, w8.dt,
                     w8.E_min, w8.E_max, w8.n_E, I, ng)
    torch.cuda.synchronize()
    gi = I.cpu().numpy()
    assert int(ng.item()) == rng_
    rel = np.max(np.abs(gi - ri)) / np.max(np.abs(ri))
    assert rel <= 1e-9, rel
    E = w8.energies()
    pr = wl.to_cm1(cf.find_peaks(E, ri))
    pg = wl.to_cm1(cf.find_peaks(E, gi))
    assert len(pr) == len(pg) and len(pr) > 0
    assert np.max(np.abs(pr - pg)) <= 0.1
    # the product spectrum (GPU flags) differs from it only through flipped trajectories
    raw = bufs.I[0].cpu().numpy()
    if len(flips) == 0:
        assert np.max(np.abs(raw - ri)) <= 1e-9 * np.max(ri)


def test_config_f6_full_size_sampled(G):
    """F=6 workload at its full size and launch shape (16384 trajectories, 4000
    steps, 4000 energies): amplitude rows of sampled trajectories against the
    oracle, and the spectrum of that sample (selected through the good mask)."""
    import torch
    w8 = wl.config_f6()
    p0, q0, w = oracle.sample_initial(w8.gamma, w8.p_eq, w8.q_eq, w8.n_traj, w8.seed)
    bufs = _full_path(G, w8, p0, q0, w)
    idx = np.sort(np.random.default_rng(0).choice(w8.n_traj, 24, replace=False))
    idx[-1] = w8.n_traj - 1   # the ragged last block
    ra, rg, rf = oracle.propagate(w8.pes, w8.gamma, w8.p_eq, w8.q_eq, w8.dt, w8.n_steps,
                                  p0[:, idx], q0[:, idx], final=True)
    ga = bufs.amp[0, torch.as_tensor(idx, device="cuda")].cpu().numpy()
    ga = ga[..., 0] + 1j * ga[..., 1]
    gg = bufs.good.cpu().numpy()
    check_flags(gg[idx], bufs.stab[idx], rg, rf["stab"])
    assert amp_err(ga[None], ra, rg) < 1e-9
    # spectrum of the sampled trajectories only (oracle flags), through the full-size launch
    mask = torch.zeros(w8.n_traj, dtype=torch.uint8, device="cuda")
    mask[torch.as_tensor(idx, device="cuda")] = _t(rg)
    sub_good = mask
    I = torch.empty(w8.n_E, dtype=torch.float64, device="cuda")
    ng = torch.zeros(1, dtype=torch.int64, device="cuda")
    G.scivr_spectrum(bufs.amp[0], w8.n_steps + 1, bufs.w, sub_good, w8.n_traj, w8.n_steps, w8.dt,
                     w8.E_min, w8.E_max, w8.n_E, I, ng)
    torch.cuda.synchronize()
    ri, rng_ = oracle.spectrum(ra[0], w[idx], rg, w8.n_steps, w8.dt, w8.E_min, w8.E_max, w8.n_E)
    assert int(ng.item()) == rng_
    gi = I.cpu().numpy()
    assert np.max(np.abs(gi - ri)) <= 1e-9 * np.max(np.abs(ri))
    # the whole-set spectrum is the n_good-weighted mean of the two halves' spectra
    half = torch.zeros_like(mask)
    half[: w8.n_traj // 2] = 1
    parts = []
    for msk in (half, 1 - half):
        Ih = torch.empty_like(I)
        ngh = torch.zeros_like(ng)
        G.scivr_spectrum(bufs.amp[0], w8.n_steps + 1, bufs.w, bufs.good * msk, w8.n_traj,
                         w8.n_steps, w8.dt, w8.E_min, w8.E_max, w8.n_E, Ih, ngh)
        parts.append((Ih, ngh))
    torch.cuda.synchronize()
    comb = sum(Ih.cpu().numpy() * int(ngh.item()) for Ih, ngh in parts) / int(bufs.n_good.item())
    full = bufs.I[0].cpu().numpy()
    assert np.max(np.abs(comb - full)) <= 1e-12 * np.max(full)


@pytest.mark.parametrize("kernel", [1, 2])
def test_propagate_several_reference_states_both_schedules(G, kernel):
    w8 = wl.config_f6(n_traj=37, n_steps=77)
    om = w8.gamma
    w8 = w8.with_(p_eq=np.stack([np.sqrt(om), np.sqrt(3 * om)]), q_eq=np.zeros((2, 6)))
    p0, q0, w = oracle.sample_initial(w8.gamma, w8.p_eq[0], w8.q_eq[0], w8.n_traj, 4)
    ra, rg = oracle.propagate(w8.pes, w8.gamma, w8.p_eq, w8.q_eq, w8.dt, w8.n_steps, p0, q0)
    g = gpu_propagate(G, w8, p0, q0, kernel=kernel)
    assert amp_err(g["amp"], ra, rg) < 1e-9


# ---------------------------------------------------------------------------
# Mixed precision (FP32 monodromy / potential / det M / det A elimination;
# FP64 p, q, S, continuous phase).  Bounds: amplitudes within 5e-2 of the trajectory's largest
# amplitude (FP32 rounding of the force and of M perturbs the trajectory and
# the prefactor phase; measured 3e-3 typical, 2.3e-2 worst over 16384
# trajectories of the F=6 workload); spectra within 1 cm^-1 per peak.
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("F", [2, 3, 6, 8, 9])
def test_mixed_propagate_close_to_oracle(G, F):
    w8 = wl.config_f3(n_traj=64, n_steps=400) if F == 3 else wl.config_generic(F, seed=F, n_traj=64, n_steps=400)
    p0, q0, w = oracle.sample_initial(w8.gamma, w8.p_eq, w8.q_eq, w8.n_traj, 3)
    ra, rg = oracle.propagate(w8.pes, w8.gamma, w8.p_eq, w8.q_eq, w8.dt, w8.n_steps, p0, q0)
    g = gpu_propagate(G, w8, p0, q0, precision=1, stab_tol=MIXED_STAB_TOL, fin=True)
    sel = rg.astype(bool) & g["good"].astype(bool)
    assert sel.sum() >= 0.95 * rg.sum()
    assert amp_err(g["amp"][:, sel], ra[:, sel], np.ones(sel.sum(), np.uint8)) < 5e-2
    # det M of the FP32 monodromy at the last step: its deviation from the FP64 value is the
    # FP32 rounding accumulated in M (the quantity the mixed stability test thresholds);
    # measured 5e-5 (F = 2) to 1.8e-3 (F = 3) over 400 steps
    rf = oracle.propagate(w8.pes, w8.gamma, w8.p_eq, w8.q_eq, w8.dt, w8.n_steps, p0, q0, final=True)[2]
    e_det = np.max(np.abs(g["detM"][sel] - rf["detM"][sel]))
    print(f"F={F}: max |det M (mixed) - det M (FP64)| = {e_det:.2e}")
    assert e_det < 1e-2
    # final positions and momenta (FP64 state driven by FP32 forces), in the
    # dimensionless units sqrt(gamma) q and p / sqrt(gamma); measured 8e-6 (F = 2) to
    # 1.1e-4 (F = 3) over 400 steps
    rg_ = np.sqrt(w8.gamma)[:, None]
    e_q = np.max(np.abs((g["q"] - rf["q"].T) * rg_)[:, sel])
    e_p = np.max(np.abs((g["p"] - rf["p"].T) / rg_)[:, sel])
    print(f"F={F}: max final-state deviation q {e_q:.2e}, p {e_p:.2e}")
    assert e_q < 1e-3 and e_p < 1e-3
    # det A: FP32 elimination of the A formed from the FP32 monodromy; measured 5.7e-6
    # (F = 2) to 3.1e-5 (F = 9) relative over 400 steps, below the monodromy's own FP32
    # error (the det M deviation above)
    dA = g["detA"][:, 0] + 1j * g["detA"][:, 1]
    e_dA = np.max(np.abs(dA[sel] - rf["detA"][sel]) / np.abs(rf["detA"][sel]))
    print(f"F={F}: max relative |det A (mixed) - det A (FP64)| = {e_dA:.2e}")
    assert e_dA < 1e-3


def test_mixed_spectrum_peaks_within_1cm(G):
    """F=3 workload at full size, mixed propagation + FP64 Fourier step, against the
    FP64 oracle on the oracle's good set: every peak within 1 cm^-1."""
    import torch
    w8 = wl.config_f3()
    p0, q0, w = oracle.sample_initial(w8.gamma, w8.p_eq, w8.q_eq, w8.n_traj, w8.seed)
    ra, rg = oracle.propagate(w8.pes, w8.gamma, w8.p_eq, w8.q_eq, w8.dt, w8.n_steps, p0, q0)
    ri, rng_ = oracle.spectrum(ra[0], w, rg, w8.n_steps, w8.dt, w8.E_min, w8.E_max, w8.n_E)
    n, K = w8.n_traj, w8.n_steps + 1
    pes = G.scivr_create_pes(w8.pes)
    amp = torch.empty((1, n, K, 2), dtype=torch.float64, device="cuda")
    good = torch.empty(n, dtype=torch.uint8, device="cuda")
    G.scivr_propagate(pes, w8.dt, w8.n_steps, w8.gamma, w8.p_eq, w8.q_eq, n, _t(p0), _t(q0), amp, K,
                      good, precision=1, stab_tol=MIXED_STAB_TOL)
    I = torch.empty(w8.n_E, dtype=torch.float64, device="cuda")
    G.scivr_spectrum(amp[0], K, _t(w), _t(rg), n, w8.n_steps, w8.dt, w8.E_min, w8.E_max, w8.n_E, I)
    torch.cuda.synchronize()
    gi = I.cpu().numpy()
    gg = good.cpu().numpy()
    flips = int(np.sum(gg.astype(bool) != rg.astype(bool)))
    assert flips <= n // 100, flips
    E = w8.energies()
    pr = wl.to_cm1(cf.find_peaks(E, ri))
    pg = wl.to_cm1(cf.find_peaks(E, gi))
    assert len(pr) > 0 and len(pr) == len(pg)
    assert np.max(np.abs(pr - pg)) <= 1.0
    assert np.max(np.abs(gi - ri)) <= 2e-2 * np.max(ri)


def test_default_configuration_full_size_sampled(G):
    """The configuration bench.py times by default, at its full size and launch shape:
    F=6 workload (16384 trajectories, 4000 steps, 4000 energies), mixed propagation,
    tensor-core bf16x3 Fourier step.

    * 24 sampled amplitude rows (the ragged last one included) against the FP64 oracle,
      to the mixed bound of 5e-2 of each row's largest amplitude;
    * the full-set spectrum of the tensor-core step against the FP64 Fourier step on
      the same device amplitudes (itself parity-tested to 1e-9), to the bf16x3 bound;
    * the sample's spectrum (oracle flags as the good mask) against the oracle's: within
      3e-2 of its maximum, and every oracle peak above 10 % of the maximum has a GPU peak
      within 1 cm^-1 (24 trajectories give small side peaks near any count threshold, so
      peaks are matched rather than counted)."""
    import torch
    from tests.test_gpu_tc import TOL
    w8 = wl.config_f6()
    n, K = w8.n_traj, w8.n_steps + 1
    p0, q0, w = oracle.sample_initial(w8.gamma, w8.p_eq, w8.q_eq, n, w8.seed)
    pes = G.scivr_create_pes(w8.pes)
    bufs = G.alloc_buffers(w8, n_traj=n)
    bufs.p0.copy_(_t(p0))
    bufs.q0.copy_(_t(q0))
    bufs.w.copy_(_t(w))
    G.scivr_propagate(pes, w8.dt, w8.n_steps, w8.gamma, w8.p_eq, w8.q_eq, n, bufs.p0, bufs.q0, bufs.amp, K,
                      bufs.good, precision=G.SCIVR_MIXED, stab_tol=MIXED_STAB_TOL)
    I_tc = torch.empty(w8.n_E, dtype=torch.float64, device="cuda")
    I_64 = torch.empty_like(I_tc)
    ng = torch.zeros(1, dtype=torch.int64, device="cuda")
    G.scivr_spectrum(bufs.amp[0], K, bufs.w, bufs.good, n, w8.n_steps, w8.dt, w8.E_min, w8.E_max, w8.n_E, I_tc,
                     ng, ft_mode=G.SCIVR_FT_TC_BF16X3)
    G.scivr_spectrum(bufs.amp[0], K, bufs.w, bufs.good, n, w8.n_steps, w8.dt, w8.E_min, w8.E_max, w8.n_E, I_64,
                     ng)
    torch.cuda.synchronize()
    assert G.scivr_check_status() == G.SCIVR_OK
    gg = bufs.good.cpu().numpy()
    assert gg.mean() > 0.99
    e_tc = np.max(np.abs(I_tc.cpu().numpy() - I_64.cpu().numpy())) / np.max(np.abs(I_64.cpu().numpy()))
    print(f"full set: bf16x3 vs FP64 Fourier step rel err {e_tc:.2e}")
    assert e_tc <= TOL[2]
    idx = np.sort(np.random.default_rng(1).choice(n, 24, replace=False))
    idx[-1] = n - 1
    ra, rg = oracle.propagate(w8.pes, w8.gamma, w8.p_eq, w8.q_eq, w8.dt, w8.n_steps, p0[:, idx], q0[:, idx])
    ga = bufs.amp[0, torch.as_tensor(idx, device="cuda")].cpu().numpy()
    ga = ga[..., 0] + 1j * ga[..., 1]
    sel = rg.astype(bool) & gg[idx].astype(bool)
    assert sel.sum() >= 22
    e_amp = amp_err(ga[None][:, sel], ra[:, sel], np.ones(sel.sum(), np.uint8))
    print(f"sampled rows: mixed vs FP64 oracle max error {e_amp:.2e}")
    assert e_amp < 5e-2
    mask = torch.zeros(n, dtype=torch.uint8, device="cuda")
    mask[torch.as_tensor(idx, device="cuda")] = _t(rg)
    I_s = torch.empty_like(I_tc)
    G.scivr_spectrum(bufs.amp[0], K, bufs.w, mask, n, w8.n_steps, w8.dt, w8.E_min, w8.E_max, w8.n_E, I_s, ng,
                     ft_mode=G.SCIVR_FT_TC_BF16X3)
    torch.cuda.synchronize()
    ri, _ = oracle.spectrum(ra[0], w[idx], rg, w8.n_steps, w8.dt, w8.E_min, w8.E_max, w8.n_E)
    gs = I_s.cpu().numpy()
    e_s = np.max(np.abs(gs - ri)) / np.max(ri)
    E = w8.energies()
    pr = wl.to_cm1(cf.find_peaks(E, ri, 0.1))
    pg = wl.to_cm1(cf.find_peaks(E, gs, 0.02))
    shift = np.array([np.min(np.abs(pg - x)) for x in pr])
    print(f"sample spectrum: rel err {e_s:.2e}; {len(pr)} peaks, max shift {shift.max():.3f} cm^-1")
    assert e_s <= 3e-2
    assert len(pr) > 0 and shift.max() <= 1.0


# ---------------------------------------------------------------------------
# Wide groups (F = 10..16, one trajectory per warp, mixed precision only).
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("F", [10, 12, 15, 16])
def test_wide_group_mixed_close_to_oracle(G, F):
    """Mixed path for F > 9 against the FP64 oracle: 67 trajectories (ragged for two
    trajectories per CTA) and 301 steps (not a multiple of the 8-step chunk); F = 16
    fills all 32 lanes with monodromy columns.  Bounds as for F <= 9."""
    w8 = wl.config_generic(F, seed=F, n_traj=67, n_steps=301)
    p0, q0, w = oracle.sample_initial(w8.gamma, w8.p_eq, w8.q_eq, w8.n_traj, 3)
    ra, rg, rf = oracle.propagate(w8.pes, w8.gamma, w8.p_eq, w8.q_eq, w8.dt, w8.n_steps, p0, q0, final=True)
    g = gpu_propagate(G, w8, p0, q0, precision=1, stab_tol=MIXED_STAB_TOL, fin=True)
    assert G.scivr_check_status() == G.SCIVR_OK
    sel = rg.astype(bool) & g["good"].astype(bool)
    assert sel.sum() >= 0.9 * rg.sum() and sel.sum() > 0
    e_amp = amp_err(g["amp"][:, sel], ra[:, sel], np.ones(sel.sum(), np.uint8))
    e_det = np.max(np.abs(g["detM"][sel] - rf["detM"][sel]))
    dA = g["detA"][:, 0] + 1j * g["detA"][:, 1]
    e_dA = np.max(np.abs(dA[sel] - rf["detA"][sel]) / np.abs(rf["detA"][sel]))
    rg_ = np.sqrt(w8.gamma)[:, None]
    e_q = np.max(np.abs((g["q"] - rf["q"].T) * rg_)[:, sel])
    e_S = np.max(np.abs(g["S"][sel] - rf["S"][sel]))
    print(f"F={F}: {sel.sum()} of {rg.sum()} good; amp {e_amp:.2e} det M {e_det:.2e} det A {e_dA:.2e} "
          f"q {e_q:.2e} S {e_S:.2e}")
    assert e_amp < 5e-2 and e_det < 1e-2 and e_dA < 1e-3 and e_q < 1e-3


@pytest.mark.parametrize("F", [17, 20, 24])
def test_two_column_groups_mixed_close_to_oracle(G, F):
    """Mixed path above F = 16 (two monodromy columns per lane, coupling tensors read from
    L2, det M in shared memory, 2-step chunks) against the FP64 oracle: 35 trajectories
    (ragged for four trajectories per CTA) and 61 steps (odd: a 1-step tail chunk).  The
    F = 24 surface is the batch recipe's (300 x 300 quartic Hessian tensor).  Bounds as for
    F <= 16."""
    w8 = wl.config_generic(F, seed=F, n_traj=35, n_steps=61)
    p0, q0, w = oracle.sample_initial(w8.gamma, w8.p_eq, w8.q_eq, w8.n_traj, 3)
    ra, rg, rf = oracle.propagate(w8.pes, w8.gamma, w8.p_eq, w8.q_eq, w8.dt, w8.n_steps, p0, q0, final=True)
    g = gpu_propagate(G, w8, p0, q0, precision=1, stab_tol=MIXED_STAB_TOL, fin=True)
    assert G.scivr_check_status() == G.SCIVR_OK
    sel = rg.astype(bool) & g["good"].astype(bool)
    print(f"F={F}: oracle good {rg.sum()}, GPU good {g['good'].sum()}, both {sel.sum()}")
    assert sel.sum() >= 0.9 * rg.sum() and sel.sum() > 0
    e_amp = amp_err(g["amp"][:, sel], ra[:, sel], np.ones(sel.sum(), np.uint8))
    e_det = np.max(np.abs(g["detM"][sel] - rf["detM"][sel]))
    dA = g["detA"][:, 0] + 1j * g["detA"][:, 1]
    e_dA = np.max(np.abs(dA[sel] - rf["detA"][sel]) / np.abs(rf["detA"][sel]))
    rg_ = np.sqrt(w8.gamma)[:, None]
    e_q = np.max(np.abs((g["q"] - rf["q"].T) * rg_)[:, sel])
    e_M = np.max(np.abs(g["M"][sel] - rf["M"][sel])) / max(1.0, np.max(np.abs(rf["M"][sel])))
    print(f"F={F}: {sel.sum()} of {rg.sum()} good; amp {e_amp:.2e} det M {e_det:.2e} det A {e_dA:.2e} "
          f"q {e_q:.2e} M {e_M:.2e}")
    assert e_amp < 5e-2 and e_det < 1e-1 and e_dA < 1e-3 and e_q < 1e-3 and e_M < 1e-3


def test_wide_group_several_reference_states_and_hk(G):
    """F = 12: two reference states, time-averaged and Herman-Kluk summands."""
    from tests.test_gpu_hk import hk_propagate
    w8 = wl.config_generic(12, seed=5, n_traj=40, n_steps=120)
    om = w8.gamma
    w8 = w8.with_(p_eq=np.stack([np.sqrt(om), np.sqrt(3 * om)]), q_eq=np.zeros((2, 12)))
    p0, q0, w = oracle.sample_initial(w8.gamma, w8.p_eq[0], w8.q_eq[0], w8.n_traj, 4)
    ra, rg = oracle.propagate(w8.pes, w8.gamma, w8.p_eq, w8.q_eq, w8.dt, w8.n_steps, p0, q0)
    g = gpu_propagate(G, w8, p0, q0, precision=1, stab_tol=MIXED_STAB_TOL)
    sel = rg.astype(bool) & g["good"].astype(bool)
    assert amp_err(g["amp"][:, sel], ra[:, sel], np.ones(sel.sum(), np.uint8)) < 5e-2
    rh, rgh = oracle.propagate(w8.pes, w8.gamma, w8.p_eq, w8.q_eq, w8.dt, w8.n_steps, p0, q0,
                               amplitude=oracle.AMP_HK)
    gh = hk_propagate(G, w8, p0, q0, precision=1, stab_tol=MIXED_STAB_TOL)
    sel = rgh.astype(bool) & gh["good"].astype(bool)
    # t = 0: 1 for the sampling state, the density ratio |<chi_1|p0 q0>|^2 / |<chi_0|p0 q0>|^2 for the other
    assert np.all(gh["amp"][0, :, 0] == 1.0)
    assert np.max(np.abs(gh["amp"][1, :, 0] - rh[1, :, 0]) / np.abs(rh[1, :, 0])) < 1e-12
    assert amp_err(gh["amp"][:, sel], rh[:, sel], np.ones(sel.sum(), np.uint8)) < 5e-2


def test_wide_group_fp64_is_unsupported(G):
    import torch
    w8 = wl.config_generic(12, seed=1, n_traj=4, n_steps=5)
    p0, q0, w = oracle.sample_initial(w8.gamma, w8.p_eq, w8.q_eq, 4, 0)
    pes = G.scivr_create_pes(w8.pes)
    amp = torch.empty((1, 4, 6, 2), dtype=torch.float64, device="cuda")
    good = torch.empty(4, dtype=torch.uint8, device="cuda")
    with pytest.raises(G.ScivrError) as ei:
        G.scivr_propagate(pes, w8.dt, 5, w8.gamma, w8.p_eq, w8.q_eq, 4, _t(p0), _t(q0), amp, 6, good)
    assert ei.value.code == G.SCIVR_EUNSUPPORTED
