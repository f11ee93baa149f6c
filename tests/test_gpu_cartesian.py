"""Propagation through the Cartesian-surface interface (Sec. III.A) on the GPU against
the FP64 oracle.

The library builds the normal modes of a Cartesian triatomic itself
(scivr_create_pes_cartesian) and its FP64 propagation kernel evaluates the surface through
the bond vectors and the chain rule at every force stage; the oracle uses its own normal
modes and evaluates the full 9 x 9 Cartesian Hessian.  Initial conditions come from the
oracle's sampler with the oracle's frequencies as widths (gamma = omega, chi at q = 0,
p = sqrt(omega)).  Bounds as for the FP64 polynomial surfaces: amplitudes within 1e-9 of
each row's largest amplitude, spectra within 1e-9 relative, peaks within 0.1 cm^-1."""
import numpy as np
import pytest

import oracle
from paper_1312_4698_gb300 import workloads as wl
from tests import closed_forms as cf
from tests.test_gpu_parity import _t, amp_err, gpu_propagate, gpu_spectrum

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    from paper_1312_4698_gb300 import scivr
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return scivr


def _workload(c, n_traj, n_steps, n_E=1500):
    om = oracle.normal_modes(c)[0]
    p_eq, q_eq = wl.ground_chi(om)
    return wl.Workload("cart_triatomic", wl.CartPes(c), om.copy(), p_eq[None], q_eq[None], n_traj, n_steps,
                       10.0, 0.0, float(wl.cm1(12000.0)), n_E, 0)


def test_cartesian_surface_values_match_the_oracle(G):
    import torch
    c = wl.water_like_triatomic()
    pes = G.scivr_create_pes_cartesian(c)
    om = oracle.normal_modes(c)[0]
    q = np.random.default_rng(4).normal(size=(257, 3)) / np.sqrt(om) * 1.5
    V = torch.empty(257, dtype=torch.float64, device="cuda")
    g = torch.empty((257, 3), dtype=torch.float64, device="cuda")
    H = torch.empty((257, 3, 3), dtype=torch.float64, device="cuda")
    G.scivr_pes_eval(pes, 257, _t(q), 0, V, g, H)
    torch.cuda.synchronize()
    for j in range(0, 257, 16):
        rV, rg, rH = oracle.pes_eval(wl.CartPes(c), q[j])
        assert abs(V[j].item() - rV) <= 1e-12 * max(abs(rV), 1e-3)
        assert np.max(np.abs(g[j].cpu().numpy() - rg)) <= 1e-11 * max(np.max(np.abs(rg)), 1e-3)
        assert np.max(np.abs(H[j].cpu().numpy() - rH)) <= 1e-11 * np.max(np.abs(rH))


def test_cartesian_propagation_and_spectrum_match_the_oracle(G):
    c = wl.water_like_triatomic()
    w8 = _workload(c, 200, 1500)
    p0, q0, w = oracle.sample_initial(w8.gamma, w8.p_eq, w8.q_eq, w8.n_traj, 21)
    ra, rg, rf = oracle.propagate(w8.pes, w8.gamma, w8.p_eq, w8.q_eq, w8.dt, w8.n_steps, p0, q0, final=True)
    g = gpu_propagate(G, w8, p0, q0, precision=0, fin=True)
    assert G.scivr_check_status() == G.SCIVR_OK
    assert np.array_equal(g["good"], rg)
    e_amp = amp_err(g["amp"], ra, rg)
    sel = rg.astype(bool)        # bad (chaotic) trajectories' final M and det A are not compared
    e_M = np.max(np.abs(g["M"][sel] - rf["M"][sel])) / max(1.0, np.max(np.abs(rf["M"][sel])))
    dA = g["detA"][:, 0] + 1j * g["detA"][:, 1]
    e_dA = np.max(np.abs(dA[sel] - rf["detA"][sel]) / np.abs(rf["detA"][sel]))
    print(f"amp {e_amp:.2e} M {e_M:.2e} det A {e_dA:.2e} good {rg.sum()}/{w8.n_traj}")
    assert e_amp < 1e-9 and e_M < 1e-8 and e_dA < 1e-9
    ri, rng_ = oracle.spectrum(ra[0], w, rg, w8.n_steps, w8.dt, w8.E_min, w8.E_max, w8.n_E)
    gi, ng = gpu_spectrum(G, g["amp"][0], w, rg, w8.n_steps, w8.dt, w8.E_min, w8.E_max, w8.n_E)
    assert ng == rng_
    assert np.max(np.abs(gi - ri)) <= 1e-9 * np.max(np.abs(ri))
    E = w8.energies()
    pr, pg = wl.to_cm1(cf.find_peaks(E, ri)), wl.to_cm1(cf.find_peaks(E, gi))
    assert len(pr) > 0 and len(pr) == len(pg) and np.max(np.abs(pr - pg)) <= 0.1
    # the zero-point peak sits near the harmonic ZPE of the normal modes
    zpe = wl.to_cm1(0.5 * np.sum(w8.gamma))
    print(f"peaks (cm^-1): {np.round(pr[:6], 1)}; harmonic ZPE {zpe:.1f}")
    assert np.min(np.abs(pr - zpe)) < 100.0


def test_cartesian_surface_needs_fp64_thread_schedule(G):
    import torch
    c = wl.water_like_triatomic()
    w8 = _workload(c, 8, 5)
    p0, q0, _ = oracle.sample_initial(w8.gamma, w8.p_eq, w8.q_eq, 8, 0)
    pes = G.scivr_create_pes_cartesian(c)
    amp = torch.empty((1, 8, 6, 2), dtype=torch.float64, device="cuda")
    good = torch.empty(8, dtype=torch.uint8, device="cuda")
    for prec, kern in ((G.SCIVR_MIXED, G.SCIVR_KERNEL_AUTO), (G.SCIVR_FP64, G.SCIVR_KERNEL_GROUP)):
        with pytest.raises(G.ScivrError) as ei:
            G.scivr_propagate(pes, w8.dt, 5, w8.gamma, w8.p_eq, w8.q_eq, 8, _t(p0), _t(q0), amp, 6, good,
                              precision=prec, kernel=kern)
        assert ei.value.code == G.SCIVR_EUNSUPPORTED
