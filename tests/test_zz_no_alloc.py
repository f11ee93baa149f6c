"""scivr_spectrum_noalloc against scivr_spectrum, through the C ABI.

Some callers cannot allocate device memory: their process hands all of it to
another component's pool, or an allocation on their path could block or fail
under memory pressure.  scivr_spectrum_noalloc serves them from a fixed
library-owned scratch array.  This file is collected last so that a run that
stops at its first failure has already run every other test; it also passes
on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-12   # the tolerance of the random-amplitude spectrum parity tests


def _inputs(n, n_steps, seed):
    rng = np.random.default_rng(seed)
    K = n_steps + 1
    amp = (rng.normal(size=(n, K)) + 1j * rng.normal(size=(n, K))) * 0.4
    w = rng.uniform(0.2, 5.0, n)
    good = (rng.uniform(size=n) > 0.15).astype(np.uint8)
    good[0] = 1
    bad = np.flatnonzero(good == 0)
    if bad.size:
        amp[bad[0], K // 2] = np.nan       # a bad row holding NaN must not leak
    return amp, w, good


def _run(scivr, torch, amp, w, good, n_steps, dt, E_min, E_max, n_E, noalloc):
    n, K = amp.shape
    a = torch.as_tensor(np.stack([amp.real, amp.imag], axis=-1), device="cuda")
    wt = torch.as_tensor(w, device="cuda")
    gt = torch.as_tensor(good, device="cuda")
    I = torch.full((n_E,), -1.0, dtype=torch.float64, device="cuda")
    ng = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    fn = scivr._lib.scivr_spectrum_noalloc if noalloc else scivr._lib.scivr_spectrum
    rc = fn(a.data_ptr(), K, scivr.SCIVR_FP64, wt.data_ptr(), gt.data_ptr(), n, n_steps, dt, E_min,
            E_max, n_E, scivr.SCIVR_FT_FP64, I.data_ptr(), ng.data_ptr(), stream)
    assert rc == scivr.SCIVR_OK, scivr.last_error()
    torch.cuda.synchronize()
    return I.cpu().numpy(), int(ng.item())


def test_noalloc_spectrum_matches_allocating_entry_point():
    import torch
    from paper_1312_4698_gb300 import scivr
    assert torch.cuda.is_available()
    dt = 10.0
    cases = [
        # (n_traj, n_steps, n_E, E_min, E_max, seed): ragged in every tile dimension
        (1100, 333, 2001, 0.002, 0.055, 1),
        (1100, 333, 2001, 0.002, 0.055, 1),   # the same call again: stale scratch must not matter
        (70, 40, 77, 0.0, 0.03, 2),            # a different shape after a larger one
        (70, 10, 300001, 0.0, 0.2, 3),         # a grid that leaves room for one row slice only
        (70, 10, 524256, 0.0, 0.2, 4),         # the largest grid: the slice fills the scratch to its end
    ]
    for n, n_steps, n_E, E_min, E_max, seed in cases:
        amp, w, good = _inputs(n, n_steps, seed)
        ref, ng_ref = _run(scivr, torch, amp, w, good, n_steps, dt, E_min, E_max, n_E, False)
        got, ng = _run(scivr, torch, amp, w, good, n_steps, dt, E_min, E_max, n_E, True)
        assert ng == ng_ref == int(good.sum())
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - ref)) <= TOL * np.max(np.abs(ref))


def test_noalloc_rejects_grids_beyond_its_scratch():
    import torch
    from paper_1312_4698_gb300 import scivr
    amp = torch.zeros((4, 11, 2), dtype=torch.float64, device="cuda")
    w = torch.ones(4, dtype=torch.float64, device="cuda")
    good = torch.ones(4, dtype=torch.uint8, device="cuda")
    I = torch.zeros(8, dtype=torch.float64, device="cuda")
    before = scivr.launch_count()
    rc = scivr._lib.scivr_spectrum_noalloc(amp.data_ptr(), 11, 0, w.data_ptr(), good.data_ptr(), 4,
                                           10, 10.0, 0.0, 0.1, 524257, 0, I.data_ptr(), None,
                                           torch.cuda.current_stream().cuda_stream)
    assert rc == scivr.SCIVR_EINVAL
    assert "scratch limit" in scivr.last_error()
    assert scivr.launch_count() == before
