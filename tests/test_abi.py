"""The C-ABI library: it builds, loads, exports every declared symbol, and
rejects invalid arguments before touching the GPU (no compute calls here)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1312_4698_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    import glob
    text = "".join(open(f).read() for f in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))))
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(scivr_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    path = B.build()
    return C.CDLL(path)


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("scivr_create_pes", "scivr_destroy_pes", "scivr_sample_initial", "scivr_propagate",
              "scivr_spectrum", "scivr_last_error"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    for s in declared_symbols():
        assert hasattr(lib, s), s


def test_binding_names_match_the_abi():
    from paper_1312_4698_gb300 import scivr
    for s in declared_symbols():
        assert s in scivr.EXPORTED, s
        assert hasattr(scivr._lib, s)
    for s in ("scivr_create_pes", "scivr_sample_initial", "scivr_propagate", "scivr_spectrum"):
        assert callable(getattr(scivr, s))


def test_invalid_potentials_are_rejected(lib):
    from paper_1312_4698_gb300 import scivr
    from paper_1312_4698_gb300 import workloads as wl
    good = wl.config_f3().pes
    bad_cases = []
    d = wl.config_f3().pes
    d.F = 0
    bad_cases.append(d)
    d = wl.config_f3().pes
    d.idx3 = d.idx3[:, ::-1].copy()          # unsorted triples
    bad_cases.append(d)
    d = wl.config_f3().pes
    d.idx3 = d.idx3.copy(); d.idx3[0, 2] = 7  # out of range
    bad_cases.append(d)
    d = wl.config_f3().pes
    d.D = -d.D
    bad_cases.append(d)
    d = wl.config_f3().pes
    d.F = 25
    bad_cases.append(d)
    for d in bad_cases:
        with pytest.raises(scivr.ScivrError) as ei:
            scivr.scivr_create_pes(d)
        assert ei.value.code == scivr.SCIVR_EINVAL
        assert scivr.last_error()
    assert good.F == 3


def test_invalid_propagate_and_spectrum_arguments(lib):
    from paper_1312_4698_gb300 import scivr
    # NULL potential
    prm = scivr.scivr_prop_params(10.0, 10, 0, 1e-6, None, None, None, 1, 0)
    rc = scivr._lib.scivr_propagate(None, C.byref(prm), 4, None, None, None, 11, None, None, None)
    assert rc == scivr.SCIVR_EINVAL
    assert "NULL" in scivr.last_error()
    # spectrum: n_E < 2, E_max <= E_min, amp_ld too small, unsupported modes
    fake = 0x1000
    cases = [
        dict(n_E=1), dict(E_min=1.0, E_max=0.5), dict(amp_ld=5), dict(n_steps=0),
        dict(n_traj=0), dict(dt=0.0),
    ]
    for over in cases:
        a = dict(amp_ld=11, n_traj=4, n_steps=10, dt=10.0, E_min=0.0, E_max=0.1, n_E=16)
        a.update(over)
        rc = scivr._lib.scivr_spectrum(fake, a["amp_ld"], 0, fake, fake, a["n_traj"], a["n_steps"],
                                       a["dt"], a["E_min"], a["E_max"], a["n_E"], 0, fake, None, None)
        assert rc == scivr.SCIVR_EINVAL, over
    rc = scivr._lib.scivr_spectrum(fake, 11, 0, fake, fake, 4, 10, 10.0, 0.0, 0.1, 16, 99, fake, None, None)
    assert rc == scivr.SCIVR_EUNSUPPORTED
    rc = scivr._lib.scivr_spectrum(fake + 8, 11, 0, fake, fake, 4, 10, 10.0, 0.0, 0.1, 16, 0, fake, None, None)
    assert rc == scivr.SCIVR_EINVAL   # misaligned amplitudes


def test_learned_residual_entry_points_validate_before_any_launch(lib):
    from paper_1312_4698_gb300 import scivr
    assert scivr.scivr_mlp_param_count(9) == 9 * 256 + 2 * 256 * 256 + 4 * 256 + 1
    assert scivr.scivr_mlp_param_count(0) == 0
    assert scivr._lib.scivr_pes_set_mlp(None, None) == scivr.SCIVR_EINVAL
    assert scivr._lib.scivr_mlp_eval(None, 4, 1, 1, 1, None, None) == scivr.SCIVR_EINVAL
    assert "NULL potential" in scivr.last_error()
    assert scivr._lib.scivr_mlp_loss_grad(None, 4, 1, 1, 1, 1.0, 1.0, 1, 1, None) == scivr.SCIVR_EINVAL
    assert scivr._lib.scivr_mlp_adamw(None, 1, 1, 1, 1, 1e-3, 0.9, 0.999, 1e-8, 0.0, None) == scivr.SCIVR_EINVAL
    assert scivr._lib.scivr_pes_eval(None, 4, 1, 0, 1, None, None, None) == scivr.SCIVR_EINVAL


def test_plain_scivr_spectrum_arguments_validated(lib):
    from paper_1312_4698_gb300 import scivr
    fake = 0x1000
    cases = [dict(n_E=1), dict(E_min=1.0, E_max=0.5), dict(amp_ld=5), dict(n_steps=0), dict(n_traj=0),
             dict(dt=-1.0), dict(amp=fake + 8), dict(good=None), dict(I_out=None), dict(C_out=fake + 8)]
    for over in cases:
        a = dict(amp=fake, amp_ld=11, good=fake, n_traj=4, n_steps=10, dt=10.0, E_min=0.0, E_max=0.1, n_E=16,
                 I_out=fake, C_out=None)
        a.update(over)
        rc = scivr._lib.scivr_spectrum_hk(a["amp"], a["amp_ld"], a["good"], a["n_traj"], a["n_steps"], a["dt"],
                                          a["E_min"], a["E_max"], a["n_E"], a["I_out"], a["C_out"], None, None)
        assert rc == scivr.SCIVR_EINVAL, over
