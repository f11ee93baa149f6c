"""Mixed-precision lane-group path against the FP64 oracle where the chunked
schedule has a ragged end, and the F = 9 methane-sized workload at full size.

The lane-group kernels process steps in chunks (mixed path: 8 steps up to
F = 12); the prefactor determinants, the phase scan and the amplitude records
run once per chunk, and the mixed path tests det M every 16 steps and at the
last step.
Step counts 301 and 405 end on a partial chunk (301 = 37*8 + 5, 405 = 50*8 + 5;
also partial for 16-step chunks: 18*16 + 13, 25*16 + 5), and 67 trajectories
leave the last CTA partly empty.  The discrete sum of Eq. 11
(I(E)_discreto) runs over every step up to T, so the tail chunk's samples
enter every spectrum.

Bounds are those of the mixed path elsewhere: amplitudes within 5e-2 of each
row's largest amplitude, det M within 1e-1, det A within 1e-3 relative, final
q and p within 1e-3 in the units sqrt(gamma) q and p / sqrt(gamma), and the
action within 1e-3 (FP64 accumulation of FP32 increments).
"""
import numpy as np
import pytest

import oracle
from paper_1312_4698_gb300 import workloads as wl
from tests import closed_forms as cf
from tests.test_gpu_parity import MIXED_STAB_TOL, _t, amp_err, gpu_propagate

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    from paper_1312_4698_gb300 import scivr
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return scivr


def tail_err(a, b, sel, tail):
    """Max over the selected rows of |a - b| on the last `tail` samples, relative to the
    row's largest |b| over all samples (a trajectory that leaves the reference state has a
    summand that underflows to zero late in the run)."""
    scale = np.max(np.abs(b[..., sel, :]), axis=-1)
    return float(np.max(np.max(np.abs(a[..., sel, -tail:] - b[..., sel, -tail:]), axis=-1) / scale))


def _workload(F, n_traj, n_steps):
    if F == 3:
        return wl.config_f3(n_traj=n_traj, n_steps=n_steps)
    return wl.config_generic(F, seed=F, n_traj=n_traj, n_steps=n_steps)


@pytest.mark.parametrize("n_steps", [301, 405])
@pytest.mark.parametrize("F", [2, 3, 6, 8, 9])
def test_mixed_ragged_tail_chunk_time_averaged(G, F, n_steps):
    w8 = _workload(F, 67, n_steps)
    p0, q0, w = oracle.sample_initial(w8.gamma, w8.p_eq, w8.q_eq, w8.n_traj, 11)
    ra, rg, rf = oracle.propagate(w8.pes, w8.gamma, w8.p_eq, w8.q_eq, w8.dt, w8.n_steps, p0, q0, final=True)
    g = gpu_propagate(G, w8, p0, q0, precision=1, stab_tol=MIXED_STAB_TOL, fin=True)
    assert G.scivr_check_status() == G.SCIVR_OK
    sel = rg.astype(bool) & g["good"].astype(bool)
    assert sel.sum() >= 0.95 * rg.sum() and sel.sum() > 0
    e_amp = amp_err(g["amp"][:, sel], ra[:, sel], np.ones(sel.sum(), np.uint8))
    # the last chunk's samples alone (the ragged tail)
    tail = n_steps % 8
    e_tail = tail_err(g["amp"], ra, sel, tail)
    e_det = np.max(np.abs(g["detM"][sel] - rf["detM"][sel]))
    dA = g["detA"][:, 0] + 1j * g["detA"][:, 1]
    e_dA = np.max(np.abs(dA[sel] - rf["detA"][sel]) / np.abs(rf["detA"][sel]))
    rg_ = np.sqrt(w8.gamma)[:, None]
    e_q = np.max(np.abs((g["q"] - rf["q"].T) * rg_)[:, sel])
    e_p = np.max(np.abs((g["p"] - rf["p"].T) / rg_)[:, sel])
    e_S = np.max(np.abs(g["S"][sel] - rf["S"][sel]))
    e_th = np.max(np.abs(g["theta"][sel] - rf["theta"][sel]))
    print(f"F={F} n_steps={n_steps}: {sel.sum()}/{rg.sum()} good; amp {e_amp:.2e} (tail {e_tail:.2e}) "
          f"det M {e_det:.2e} det A {e_dA:.2e} q {e_q:.2e} p {e_p:.2e} S {e_S:.2e} theta {e_th:.2e}")
    assert e_amp < 5e-2 and e_tail < 5e-2
    # det M of the FP32 monodromy is FP32 rounding of a determinant whose entries grow along
    # the trajectory (measured up to 2.4e-2 at F = 9); it only feeds the stability test, whose
    # FP32 threshold is 537
    assert e_det < 1e-1 and e_dA < 1e-3
    assert e_q < 1e-3 and e_p < 1e-3 and e_S < 1e-3
    # the continuous phase lands on the oracle's branch (no lost or extra turn)
    assert e_th < 1e-2


@pytest.mark.parametrize("n_steps", [301, 405])
@pytest.mark.parametrize("F", [2, 3, 6, 8, 9])
def test_mixed_ragged_tail_chunk_herman_kluk(G, F, n_steps):
    from tests.test_gpu_hk import hk_propagate
    w8 = _workload(F, 67, n_steps)
    om = w8.gamma
    w8 = w8.with_(p_eq=np.stack([np.sqrt(om), np.sqrt(3 * om)]), q_eq=np.zeros((2, F)))
    p0, q0, w = oracle.sample_initial(w8.gamma, w8.p_eq[0], w8.q_eq[0], w8.n_traj, 12)
    rh, rgh = oracle.propagate(w8.pes, w8.gamma, w8.p_eq, w8.q_eq, w8.dt, w8.n_steps, p0, q0,
                               stab_tol=MIXED_STAB_TOL, amplitude=oracle.AMP_HK)
    gh = hk_propagate(G, w8, p0, q0, precision=1, stab_tol=MIXED_STAB_TOL)
    sel = rgh.astype(bool) & gh["good"].astype(bool)
    assert sel.sum() >= 0.95 * rgh.sum() and sel.sum() > 0
    assert np.all(gh["amp"][0, :, 0] == 1.0)
    e = amp_err(gh["amp"][:, sel], rh[:, sel], np.ones(sel.sum(), np.uint8))
    tail = n_steps % 8
    e_tail = tail_err(gh["amp"], rh, sel, tail)
    print(f"F={F} n_steps={n_steps}: HK summands {e:.2e} (tail {e_tail:.2e})")
    assert e < 5e-2 and e_tail < 5e-2


def test_mixed_chunk_end_stability_test_flags(G):
    """Flags of the mixed path (FP32 det M tested every 16 steps) against the oracle's
    (FP64 det M tested every step) at the same threshold, on a surface where most
    trajectories go bad: F = 6 with the recipe's couplings on mass-weighted q (the
    literal reading, under which trajectories escape), 128 trajectories, 600 steps.
    The flipped trajectories are reported; at most 2 % may differ."""
    rng = np.random.default_rng(3)
    pes = wl.recipe_pes(6, rng, sigma3=3e-8, sigma4=3e-9, units=wl.COUPLING_MASS_WEIGHTED)
    p_eq, q_eq = wl.ground_chi(pes.omega)
    lo, hi = wl.grid_window(pes.omega)
    w8 = wl.Workload("f6_unstable", pes, pes.omega.copy(), p_eq[None], q_eq[None], 128, 600, 10.0, lo, hi,
                     400, 3)
    p0, q0, w = oracle.sample_initial(w8.gamma, w8.p_eq, w8.q_eq, w8.n_traj, 5)
    ra, rg = oracle.propagate(w8.pes, w8.gamma, w8.p_eq, w8.q_eq, w8.dt, w8.n_steps, p0, q0,
                              stab_tol=MIXED_STAB_TOL)
    g = gpu_propagate(G, w8, p0, q0, precision=1, stab_tol=MIXED_STAB_TOL)
    flips = np.flatnonzero(g["good"].astype(bool) != rg.astype(bool))
    print(f"oracle good {int(rg.sum())}/{w8.n_traj}, mixed good {int(g['good'].sum())}; flips {flips.tolist()}")
    assert 0 < rg.sum() < w8.n_traj          # the surface exercises the test both ways
    assert len(flips) <= max(1, w8.n_traj // 50)


def test_config_f9_full_size_sampled(G):
    """The methane-sized workload (F = 9, 65536 trajectories, 5000 steps, 4000
    energies) at its full size and launch shape: mixed propagation with FP32
    amplitude storage and the tensor-core bf16x3 Fourier step.  (5000 steps are
    whole 4-step chunks here, and the det M test falls every 16 steps and at the
    last step; the tests above cover the ragged tail.)

    * 24 sampled amplitude rows, the last trajectory included, against the FP64
      oracle within the mixed bound;
    * the full-set tensor-core spectrum against the FP64 Fourier step on the same
      device amplitudes (itself parity-tested to 1e-9), within the bf16x3 bound;
    * the sample's spectrum (oracle flags as the good mask) against the oracle's,
      every oracle peak above 10 % of the maximum matched within 1 cm^-1."""
    import torch
    from tests.test_gpu_tc import TOL
    w8 = wl.config_f9()
    n, K = w8.n_traj, w8.n_steps + 1
    p0, q0, w = oracle.sample_initial(w8.gamma, w8.p_eq, w8.q_eq, n, w8.seed)
    pes = G.scivr_create_pes(w8.pes)
    bufs = G.alloc_buffers(w8, n_traj=n, amp_f32=True)
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
    print(f"good {gg.sum()}/{n}")
    assert gg.mean() > 0.99
    e_tc = np.max(np.abs(I_tc.cpu().numpy() - I_64.cpu().numpy())) / np.max(np.abs(I_64.cpu().numpy()))
    print(f"full set: bf16x3 vs FP64 Fourier step rel err {e_tc:.2e}")
    assert e_tc <= TOL[2]
    idx = np.sort(np.random.default_rng(2).choice(n, 24, replace=False))
    idx[-1] = n - 1
    ra, rg = oracle.propagate(w8.pes, w8.gamma, w8.p_eq, w8.q_eq, w8.dt, w8.n_steps, p0[:, idx], q0[:, idx])
    ga = bufs.amp[0, torch.as_tensor(idx, device="cuda")].cpu().numpy().astype(np.float64)
    ga = ga[..., 0] + 1j * ga[..., 1]
    sel = rg.astype(bool) & gg[idx].astype(bool)
    assert sel.sum() >= 22
    e_amp = amp_err(ga[None][:, sel], ra[:, sel], np.ones(sel.sum(), np.uint8))
    e_tail = tail_err(ga[None], ra, sel, 8)
    print(f"sampled rows: mixed vs FP64 oracle max error {e_amp:.2e} (8-step tail {e_tail:.2e})")
    assert e_amp < 5e-2 and e_tail < 5e-2
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
