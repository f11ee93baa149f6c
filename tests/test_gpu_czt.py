"""FP64 chirp-z Fourier step (SCIVR_FT_CZT64) against the oracle's direct sum of
Eq. I(E)_discreto.

The mode evaluates the same sums through Bluestein's identity and FP64 FFTs, so it is
held to FP64-level agreement with the direct sum: 1e-12 relative on random amplitudes
(rounding of the transform grows with log2 of its length, 13), the Dirichlet kernel of a
single-frequency amplitude in closed form, several energy blocks when n_steps + 1 +
n_E - 1 exceeds the transform length, and the plain F = 6 path end to end (FP64
propagation + this step) within 1e-9 of the oracle with every peak within 0.1 cm^-1."""
import numpy as np
import pytest

import oracle
from paper_1312_4698_gb300 import workloads as wl
from tests import closed_forms as cf
from tests.test_gpu_parity import _t

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    from paper_1312_4698_gb300 import scivr
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return scivr


def _czt(G, amp, w, good, n_steps, dt, E_min, E_max, n_E, mode=None):
    import torch
    n, K = amp.shape
    a = np.stack([amp.real, amp.imag], axis=-1)
    I = torch.empty(n_E, dtype=torch.float64, device="cuda")
    ng = torch.zeros(1, dtype=torch.int64, device="cuda")
    G.scivr_spectrum(_t(a), K, _t(w), _t(good.astype(np.uint8)), n, n_steps, dt, E_min, E_max, n_E, I, ng,
                     ft_mode=G.SCIVR_FT_CZT64 if mode is None else mode)
    torch.cuda.synchronize()
    return I.cpu().numpy(), int(ng.cpu().item())


@pytest.mark.parametrize("n,n_steps,n_E,E_min,E_max", [
    (70, 333, 2001, 0.002, 0.055),       # one energy block
    (5, 1, 2, 0.0, 0.1),                 # the smallest shapes
    (37, 6000, 3000, 0.01, 0.07),        # 8193 - 6001 = 2192 energies per block: two blocks
    (200, 4000, 4000, 0.0, 0.0547),      # the F = 6 workload's shape (one block)
])
def test_czt_matches_the_direct_sum(G, n, n_steps, n_E, E_min, E_max):
    rng = np.random.default_rng(n + n_steps)
    K = n_steps + 1
    amp = (rng.normal(size=(n, K)) + 1j * rng.normal(size=(n, K))) * np.exp(-np.arange(K) / (3.0 * K))
    w = rng.uniform(0.2, 5.0, n)
    good = (rng.uniform(size=n) > 0.2).astype(np.uint8)
    good[0] = 1
    bad = np.flatnonzero(good == 0)
    if bad.size:
        amp[bad[0], K // 2] = np.nan        # excluded rows never reach the sum
    ref, rng_ = oracle.spectrum(amp, w, good, n_steps, 10.0, E_min, E_max, n_E)
    got, ng = _czt(G, amp, w, good, n_steps, 10.0, E_min, E_max, n_E)
    assert ng == rng_
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    print(f"n={n} K={K} n_E={n_E}: max rel err {err:.2e}")
    assert err <= 1e-12


def test_czt_dirichlet_closed_form(G):
    """a(c) = exp(-i E0 c dt): I(E) = dt^2/(2 pi T) sin^2(K x/2)/sin^2(x/2), x = (E - E0) dt."""
    n_steps, dt, n_E = 3000, 10.0, 2500
    E0 = 0.0237
    K = n_steps + 1
    amp = np.exp(-1j * E0 * np.arange(K) * dt)[None, :]
    E_min, E_max = 0.01, 0.04
    got, _ = _czt(G, amp, np.ones(1), np.ones(1, np.uint8), n_steps, dt, E_min, E_max, n_E)
    E = np.linspace(E_min, E_max, n_E)
    ref = dt * dt / (2 * np.pi * n_steps * dt) * np.abs(cf.dirichlet((E - E0) * dt, K)) ** 2
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(ref)


def test_plain_fp64_path_with_czt_matches_the_oracle(G):
    """F = 6 workload (1024 trajectories, 4000 steps, 4000 energies): FP64 propagation and
    the chirp-z step against the oracle end to end."""
    from tests.test_gpu_parity import gpu_propagate
    w8 = wl.config_f6(n_traj=1024)
    p0, q0, w = oracle.sample_initial(w8.gamma, w8.p_eq, w8.q_eq, w8.n_traj, w8.seed)
    ra, rg = oracle.propagate(w8.pes, w8.gamma, w8.p_eq, w8.q_eq, w8.dt, w8.n_steps, p0, q0)
    ri, rng_ = oracle.spectrum(ra[0], w, rg, w8.n_steps, w8.dt, w8.E_min, w8.E_max, w8.n_E)
    g = gpu_propagate(G, w8, p0, q0, precision=0)
    gi, ng = _czt(G, g["amp"][0], w, rg, w8.n_steps, w8.dt, w8.E_min, w8.E_max, w8.n_E)
    assert ng == rng_
    err = np.max(np.abs(gi - ri)) / np.max(ri)
    E = w8.energies()
    pr, pg = wl.to_cm1(cf.find_peaks(E, ri)), wl.to_cm1(cf.find_peaks(E, gi))
    print(f"rel err {err:.2e}; {len(pr)} peaks, max shift {np.max(np.abs(pr - pg)) if len(pr) == len(pg) else -1:.2e}")
    assert err <= 1e-9
    assert len(pr) > 0 and len(pr) == len(pg) and np.max(np.abs(pr - pg)) <= 0.1


def test_czt_rejects_shapes_beyond_its_transform(G):
    import torch
    amp = torch.zeros((2, 7170, 2), dtype=torch.float64, device="cuda")
    w = torch.ones(2, dtype=torch.float64, device="cuda")
    good = torch.ones(2, dtype=torch.uint8, device="cuda")
    I = torch.zeros(100, dtype=torch.float64, device="cuda")
    with pytest.raises(G.ScivrError) as ei:
        G.scivr_spectrum(amp, 7170, w, good, 2, 7169, 10.0, 0.0, 0.1, 100, I, ft_mode=G.SCIVR_FT_CZT64)
    assert ei.value.code == G.SCIVR_EUNSUPPORTED
