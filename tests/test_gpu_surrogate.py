"""The learned residual end to end on the GPU: training data from trajectories,
training by the library's own loss-gradient and AdamW kernels, and what the
trained network gains over the method without it.

The network learns the coupling polynomial of the F = 6 surface (cubic and
quartic terms) on top of its Morse diagonal.  "Without it" is the same
TA-SC-IVR run on the diagonal alone; both are measured against the FP64 oracle
on the full analytic surface.
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
    assert torch.cuda.is_available()
    return scivr


@pytest.fixture(scope="module")
def trained(G):
    import torch
    from paper_1312_4698_gb300 import surrogate as su
    w8 = wl.config_f6()
    full = G.scivr_create_pes(w8.pes)
    q = su.trajectory_points(full, w8, n_traj=8192, n_seg=8, seg_steps=60, seed=3)
    V, g = su.coupling_targets(full, q)
    net = su.initial_network(w8, V, seed=0)
    P = G.scivr_create_pes(su.surrogate_pes(w8, net))
    res = su.train(P, q, V, g, epochs=300, batch=4096, lr=3e-3)
    theta = torch.zeros(G.scivr_mlp_param_count(w8.F), device="cuda")
    G.scivr_mlp_get_params(P, theta)
    torch.cuda.synchronize()
    m = net.with_flat(theta.cpu().double().numpy())
    return dict(w8=w8, P=P, res=res, mlp=m)


def test_training_fits_the_coupling_residual(G, trained):
    import torch
    res, P, w8 = trained["res"], trained["P"], trained["w8"]
    L = np.array(res.losses)
    print(f"{res.steps} steps in {res.seconds:.2f} s: loss {L[0]:.3e} -> {L[-1]:.3e}")
    assert np.all(np.isfinite(L))
    assert L[-8:].mean() < L[:8].mean() / 1000
    # held-out points, expected values from the oracle's analytic surface
    F = w8.F
    rng = np.random.default_rng(42)
    qt = rng.normal(0.0, 1.0, (400, F)) * np.sqrt(1.0 / w8.pes.omega)
    diag = wl.PesDesc(F, w8.pes.diag_kind, w8.pes.omega, w8.pes.D, w8.pes.a, np.zeros((0, 3)), np.zeros(0),
                      np.zeros((0, 4)), np.zeros(0))
    Vc = np.array([oracle.pes_eval(w8.pes, x)[0] - oracle.pes_eval(diag, x)[0] for x in qt])
    gc = np.array([oracle.pes_eval(w8.pes, x)[1] - oracle.pes_eval(diag, x)[1] for x in qt])
    V = torch.zeros(400, device="cuda")
    g = torch.zeros(400, F, device="cuda")
    G.scivr_mlp_eval(P, 400, torch.as_tensor(qt, dtype=torch.float32, device="cuda"), V, g, None)
    torch.cuda.synchronize()
    eV = np.linalg.norm(V.cpu().double().numpy() - Vc) / np.linalg.norm(Vc)
    eg = np.linalg.norm(g.cpu().double().numpy() - gc) / np.linalg.norm(gc)
    print(f"held-out relative error: V {eV:.3e}, grad V {eg:.3e}")
    assert eV < 0.03 and eg < 0.05


def test_trained_network_gain_over_the_method_without_it(G, trained):
    """Spectra on 512 trajectories x 1500 steps of the F = 6 surface.  Truth:
    the oracle on the full analytic surface.  Without the learned term: the
    oracle on the Morse diagonal alone.  With it: the GPU surrogate path
    (diagonal + trained network).  Every peak of the surrogate spectrum lies
    within 1 cm^-1 of the truth, and its max-norm error is at least 10 times
    smaller than that of the run without the network."""
    import torch
    from tests.test_gpu_parity import gpu_propagate, gpu_spectrum, MIXED_STAB_TOL
    base = trained["w8"]
    n, steps = 512, 1500
    w8 = base.with_(n_traj=n, n_steps=steps, n_E=2000)
    p0, q0, w = oracle.sample_initial(w8.gamma, w8.p_eq[0], w8.q_eq[0], n, 0)
    ra, rg = oracle.propagate(w8.pes, w8.gamma, w8.p_eq, w8.q_eq, w8.dt, steps, p0, q0)
    I_true, _ = oracle.spectrum(ra[0], w, rg, steps, w8.dt, w8.E_min, w8.E_max, w8.n_E)
    diag = wl.PesDesc(6, w8.pes.diag_kind, w8.pes.omega, w8.pes.D, w8.pes.a, np.zeros((0, 3)), np.zeros(0),
                      np.zeros((0, 4)), np.zeros(0))
    da, dg = oracle.propagate(diag, w8.gamma, w8.p_eq, w8.q_eq, w8.dt, steps, p0, q0)
    I_diag, _ = oracle.spectrum(da[0], w, dg, steps, w8.dt, w8.E_min, w8.E_max, w8.n_E)
    sur = diag
    sur.mlp = trained["mlp"]
    ws = w8.with_(pes=sur)
    go = gpu_propagate(G, ws, p0, q0, precision=G.SCIVR_MIXED, stab_tol=MIXED_STAB_TOL)
    assert G.scivr_check_status() == G.SCIVR_OK
    I_s, _ = gpu_spectrum(G, go["amp"][0], w, go["good"], steps, w8.dt, w8.E_min, w8.E_max, w8.n_E)
    scale = np.max(I_true)
    e_s = np.max(np.abs(I_s - I_true)) / scale
    e_d = np.max(np.abs(I_diag - I_true)) / scale
    E = w8.energies()
    pt = wl.to_cm1(cf.find_peaks(E, I_true))
    ps = wl.to_cm1(cf.find_peaks(E, I_s))
    print(f"max-norm error: surrogate {e_s:.3e}, without the network {e_d:.3e} (gain {e_d / e_s:.1f}x); "
          f"{len(pt)} peaks, max shift {np.max(np.abs(pt - ps)) if len(pt) == len(ps) else float('nan'):.3f} cm^-1")
    assert len(pt) == len(ps) and len(pt) > 0
    assert np.max(np.abs(pt - ps)) <= 1.0
    assert e_s * 10 <= e_d
