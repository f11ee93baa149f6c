"""FP32 amplitude storage of the mixed path (scivr_prop_params.amp_prec =
SCIVR_MIXED): complex-float rows, half the bytes of complex-double rows.

The mixed kernels form every amplitude sample c >= 1 in FP32 (overlap exponent and
phase, FP32 sine, cosine and exponential), so the float rows hold exactly the values
the double rows hold; only the c = 0 sample, formed in FP64, is rounded.  Every Fourier
mode of scivr_spectrum reads the float rows (the FP64 modes widen them on load).

Against the same propagation stored as complex doubles (held to the FP64 oracle by
the mixed parity tests), at a ragged step count and a partly empty last CTA:
* samples c >= 1 equal bit for bit, c = 0 within FP32 rounding, flags equal;
* the tensor-core spectrum is identical (its digit split reads FP32 either way); the
  FP64 direct sum and the chirp-z step agree to 1e-6 of the spectrum's maximum (one
  sample per row rounded to FP32);
and against the oracle: the F = 3 workload's spectrum from float rows has every peak
within 1 cm^-1 of the FP64 oracle's.  FP32 storage with FP64 precision or with
Herman-Kluk summands is refused before any launch.
"""
import numpy as np
import pytest

import oracle
from paper_1312_4698_gb300 import workloads as wl
from tests import closed_forms as cf
from tests.test_gpu_parity import MIXED_STAB_TOL, _t

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    from paper_1312_4698_gb300 import scivr
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return scivr


def _run(G, w8, p0, q0, f32):
    import torch
    n, K = p0.shape[1], w8.n_steps + 1
    pes = G.scivr_create_pes(w8.pes)
    amp = torch.empty((w8.n_chi, n, K, 2), dtype=torch.float32 if f32 else torch.float64, device="cuda")
    good = torch.empty(n, dtype=torch.uint8, device="cuda")
    G.scivr_propagate(pes, w8.dt, w8.n_steps, w8.gamma, w8.p_eq, w8.q_eq, n, _t(p0), _t(q0), amp, K, good,
                      precision=G.SCIVR_MIXED, stab_tol=MIXED_STAB_TOL)
    torch.cuda.synchronize()
    return amp, good


@pytest.mark.parametrize("F", [3, 6, 9, 12])
def test_float_rows_hold_the_mixed_samples(G, F):
    import torch
    w8 = (wl.config_f3 if F == 3 else lambda **k: wl.config_generic(F, seed=F, **k))(n_traj=67, n_steps=405)
    p0, q0, w = oracle.sample_initial(w8.gamma, w8.p_eq, w8.q_eq, 67, 5)
    a64, g64 = _run(G, w8, p0, q0, False)
    a32, g32 = _run(G, w8, p0, q0, True)
    assert G.scivr_check_status() == G.SCIVR_OK
    assert torch.equal(g64, g32)
    d, f = a64.cpu().numpy(), a32.cpu().numpy()
    sel = g64.cpu().numpy().astype(bool)
    assert sel.sum() >= 60
    # c >= 1: the same FP32 values
    assert np.array_equal(d[:, sel, 1:], f[:, sel, 1:].astype(np.float64))
    # c = 0: FP64 rounded to FP32
    assert np.allclose(d[:, sel, 0], f[:, sel, 0], rtol=2.0 ** -24, atol=0.0)
    n, K = 67, w8.n_steps + 1
    gw, ng = _t(w), torch.zeros(1, dtype=torch.int64, device="cuda")
    for mode, tol in ((G.SCIVR_FT_TC_BF16X3, 0.0), (G.SCIVR_FT_FP64, 1e-6), (G.SCIVR_FT_CZT64, 1e-6)):
        I64 = torch.empty(w8.n_E, dtype=torch.float64, device="cuda")
        I32 = torch.empty_like(I64)
        G.scivr_spectrum(a64[0], K, gw, g64, n, w8.n_steps, w8.dt, w8.E_min, w8.E_max, w8.n_E, I64, ng,
                         ft_mode=mode)
        G.scivr_spectrum(a32[0], K, gw, g32, n, w8.n_steps, w8.dt, w8.E_min, w8.E_max, w8.n_E, I32, ng,
                         ft_mode=mode)
        torch.cuda.synchronize()
        x, y = I64.cpu().numpy(), I32.cpu().numpy()
        err = float(np.max(np.abs(x - y)) / np.max(np.abs(x)))
        print(f"F={F} mode {mode}: float vs double rows {err:.2e}")
        if tol == 0.0:
            assert np.array_equal(x, y), mode
        else:
            assert err <= tol, (mode, err)


def test_float_rows_f3_spectrum_peaks_match_oracle(G):
    import torch
    w8 = wl.config_f3()
    n, K = w8.n_traj, w8.n_steps + 1
    p0, q0, w = oracle.sample_initial(w8.gamma, w8.p_eq, w8.q_eq, n, w8.seed)
    ra, rg = oracle.propagate(w8.pes, w8.gamma, w8.p_eq, w8.q_eq, w8.dt, w8.n_steps, p0, q0)
    ri, _ = oracle.spectrum(ra[0], w, rg, w8.n_steps, w8.dt, w8.E_min, w8.E_max, w8.n_E)
    a32, g32 = _run(G, w8, p0, q0, True)
    I = torch.empty(w8.n_E, dtype=torch.float64, device="cuda")
    G.scivr_spectrum(a32[0], K, _t(w), _t(rg), n, w8.n_steps, w8.dt, w8.E_min, w8.E_max, w8.n_E, I)
    torch.cuda.synchronize()
    gi = I.cpu().numpy()
    E = w8.energies()
    pr = wl.to_cm1(cf.find_peaks(E, ri))
    pg = wl.to_cm1(cf.find_peaks(E, gi))
    assert len(pr) > 0 and len(pr) == len(pg)
    assert np.max(np.abs(pr - pg)) <= 1.0
    assert np.max(np.abs(gi - ri)) <= 2e-2 * np.max(ri)


def test_float_rows_refused_for_fp64_precision_and_hk(G):
    import torch
    w8 = wl.config_f3(n_traj=4, n_steps=5)
    pes = G.scivr_create_pes(w8.pes)
    p0 = torch.zeros((3, 4), dtype=torch.float64, device="cuda")
    amp = torch.empty((1, 4, 6, 2), dtype=torch.float32, device="cuda")
    good = torch.empty(4, dtype=torch.uint8, device="cuda")
    for kw in (dict(precision=G.SCIVR_FP64), dict(precision=G.SCIVR_MIXED, amplitude=G.SCIVR_AMP_HK)):
        with pytest.raises(G.ScivrError) as ei:
            G.scivr_propagate(pes, w8.dt, 5, w8.gamma, w8.p_eq, w8.q_eq, 4, p0, p0, amp, 6, good,
                              stab_tol=MIXED_STAB_TOL, **kw)
        assert ei.value.code == G.SCIVR_EINVAL
        assert "FP32 amplitude storage" in G.last_error()
