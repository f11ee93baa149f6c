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
    # amplitude storage: only FP64 (complex double) and SCIVR_MIXED (complex float, 8-byte aligned)
    rc = scivr._lib.scivr_spectrum(fake, 11, 7, fake, fake, 4, 10, 10.0, 0.0, 0.1, 16, 0, fake, None, None)
    assert rc == scivr.SCIVR_EINVAL and "amp_prec" in scivr.last_error()
    rc = scivr._lib.scivr_spectrum(fake + 4, 11, 1, fake, fake, 4, 10, 10.0, 0.0, 0.1, 16, 0, fake, None, None)
    assert rc == scivr.SCIVR_EINVAL and "aligned" in scivr.last_error()


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


def test_remaining_entry_points_validate_before_any_launch(lib):
    """Sampling, the wait self-test, the allocation-free spectrum and the batch plan
    reject bad arguments on the host, name the failing call, and leave no plan behind."""
    from paper_1312_4698_gb300 import scivr
    L = scivr._lib
    fake = 0x1000
    g = np.ones(3)
    rc = L.scivr_sample_initial(None, g.ctypes.data, g.ctypes.data, g.ctypes.data, 8, 0, fake, fake, fake, None)
    assert rc == scivr.SCIVR_EINVAL and "scivr_sample_initial" in scivr.last_error()
    for s in (0.0, -1.0, 10.5, float("nan")):
        assert L.scivr_selftest_wait_timeout(s, None) == scivr.SCIVR_EINVAL, s
    assert L.scivr_pes_modes(None) == 0

    base = dict(amp=fake, amp_ld=11, prec=0, n_traj=4, n_steps=10, dt=10.0, E_min=0.0, E_max=0.1, n_E=16, ft=0)
    for over, code in ((dict(n_E=1 << 20), scivr.SCIVR_EINVAL), (dict(n_E=1), scivr.SCIVR_EINVAL),
                       (dict(amp=fake + 8), scivr.SCIVR_EINVAL), (dict(E_max=float("inf")), scivr.SCIVR_EINVAL),
                       (dict(prec=7), scivr.SCIVR_EINVAL), (dict(prec=1, amp=fake + 4), scivr.SCIVR_EINVAL),
                       (dict(ft=2), scivr.SCIVR_EUNSUPPORTED)):
        a = dict(base, **over)
        rc = L.scivr_spectrum_noalloc(a["amp"], a["amp_ld"], a["prec"], fake, fake, a["n_traj"], a["n_steps"],
                                      a["dt"], a["E_min"], a["E_max"], a["n_E"], a["ft"], fake, None, None)
        assert rc == code, over
        assert scivr.last_error().startswith("scivr_spectrum_noalloc"), over
    L.scivr_spectrum_noalloc(fake, 11, 0, fake, fake, 4, 10, 10.0, 0.0, 0.1, 1 << 20, 0, fake, None, None)
    assert "scratch limit" in scivr.last_error()

    out = C.c_void_p(7)
    assert L.scivr_batch_create(None, 1, 0, C.byref(out)) == scivr.SCIVR_EINVAL
    items = (scivr.scivr_batch_item * 2)()
    assert L.scivr_batch_create(items, 0, 0, C.byref(out)) == scivr.SCIVR_EINVAL
    assert L.scivr_batch_create(items, 2, 99, C.byref(out)) == scivr.SCIVR_EUNSUPPORTED
    assert not out.value
    assert L.scivr_batch_create(items, 2, 0, C.byref(out)) == scivr.SCIVR_EINVAL
    assert scivr.last_error().startswith("scivr_batch_create: item 0: scivr_propagate: NULL")
    assert not out.value
    n = C.c_int32(-1)
    assert L.scivr_batch_info(None, -1, C.byref(n), None, None, None) == scivr.SCIVR_EINVAL
    assert L.scivr_batch_destroy(None) == scivr.SCIVR_OK


def test_potential_descriptor_checks(lib):
    """Each malformed potential descriptor is refused with SCIVR_EINVAL or
    SCIVR_EUNSUPPORTED before any device allocation."""
    from paper_1312_4698_gb300 import scivr
    from paper_1312_4698_gb300 import workloads as wl
    L = scivr._lib
    d0 = wl.config_f6().pes
    keep = []

    def desc(**over):
        arr = dict(omega=d0.omega, D=d0.D, a=d0.a, idx3=d0.idx3, c3=d0.c3, idx4=d0.idx4, c4=d0.c4)
        arr.update({k: v for k, v in over.items() if k in arr and v is not None})
        arr = {k: np.ascontiguousarray(v, dtype=np.int32 if k.startswith("idx") else np.float64)
               for k, v in arr.items()}
        keep.append(arr)
        n3 = over.get("n3", arr["c3"].size)
        n4 = over.get("n4", arr["c4"].size)
        ptr = lambda k: None if over.get(k, 0) is None else arr[k].ctypes.data
        return scivr.scivr_pes_desc(over.get("F", d0.F), over.get("kind", scivr.SCIVR_PES_POLY),
                                    over.get("diag_kind", d0.diag_kind), ptr("omega"), ptr("D"), ptr("a"),
                                    n3, ptr("idx3"), ptr("c3"), n4, ptr("idx4"), ptr("c4"))

    bad_c3 = d0.c3.copy(); bad_c3[5] = np.nan
    bad_c4 = d0.c4.copy(); bad_c4[-1] = np.inf
    bad_i4 = d0.idx4.copy(); bad_i4[3] = bad_i4[3][::-1]
    bad_om = d0.omega.copy(); bad_om[2] = 0.0
    bad_a = d0.a.copy(); bad_a[0] = -1.0
    cases = [
        (dict(kind=1), scivr.SCIVR_EUNSUPPORTED),
        (dict(diag_kind=7), scivr.SCIVR_EINVAL),
        (dict(omega=bad_om), scivr.SCIVR_EINVAL),
        (dict(a=bad_a), scivr.SCIVR_EINVAL),
        (dict(n3=-1), scivr.SCIVR_EINVAL),
        (dict(idx3=None), scivr.SCIVR_EINVAL),
        (dict(c4=None), scivr.SCIVR_EINVAL),
        (dict(c3=bad_c3), scivr.SCIVR_EINVAL),
        (dict(c4=bad_c4), scivr.SCIVR_EINVAL),
        (dict(idx4=bad_i4), scivr.SCIVR_EINVAL),
        (dict(F=-3), scivr.SCIVR_EINVAL),
    ]
    for over, code in cases:
        h = C.c_void_p(7)
        rc = L.scivr_create_pes(C.byref(desc(**over)), C.byref(h))
        assert rc == code, over
        assert not h.value, over
        assert scivr.last_error().startswith("scivr_create_pes"), over
    assert L.scivr_create_pes(None, None) == scivr.SCIVR_EINVAL


def test_last_error_is_per_thread(lib):
    """scivr_last_error belongs to the calling thread: an error raised in one thread
    does not show in another thread's message."""
    import threading
    from paper_1312_4698_gb300 import scivr
    L = scivr._lib
    seen = {}

    def worker():
        seen["before"] = scivr.last_error()
        L.scivr_selftest_wait_timeout(-1.0, None)
        seen["after"] = scivr.last_error()

    L.scivr_batch_info(None, -1, None, None, None, None)
    mine = scivr.last_error()
    t = threading.Thread(target=worker)
    t.start()
    t.join()
    assert mine.startswith("scivr_batch_info")
    assert seen["before"] == ""
    assert seen["after"].startswith("scivr_selftest_wait_timeout")
    assert scivr.last_error() == mine


def test_binding_constants_equal_the_header_values():
    """Every enumerator and #define of include/*.h that the binding mirrors has the same value."""
    import glob
    from paper_1312_4698_gb300 import scivr
    text = "".join(open(f).read() for f in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))))
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    values = {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(SCIVR_[A-Z0-9_]+)\s*=\s*(-?\d+)", text)}
    values.update({m.group(1): int(m.group(2)) for m in re.finditer(r"#define\s+(SCIVR_[A-Z0-9_]+)\s+(-?\d+)", text)})
    assert len(values) >= 20
    mirrored = [k for k in values if hasattr(scivr, k)]
    assert {"SCIVR_MIXED", "SCIVR_FT_TC_BF16X3", "SCIVR_AMP_HK", "SCIVR_KERNEL_GROUP", "SCIVR_MAX_F",
            "SCIVR_ETIMEOUT"} <= set(mirrored)
    for k in mirrored:
        assert getattr(scivr, k) == values[k], k


def test_binding_struct_layouts_match_the_headers(tmp_path):
    """Each ctypes mirror of a header struct has the C compiler's size and field offsets
    (a probe compiled with gcc against include/*.h)."""
    import shutil
    import subprocess
    from paper_1312_4698_gb300 import scivr
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    structs = [getattr(scivr, n) for n in ("scivr_pes_desc", "scivr_prop_params", "scivr_final_state",
                                           "scivr_batch_item", "scivr_mlp_desc", "scivr_cart_triatomic")]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "scivr.h"', '#include "scivr_mlp.h"',
             'int main(void) {']
    for S in structs:
        lines.append(f'  printf("{S.__name__} size %zu\\n", sizeof({S.__name__}));')
        for f in S._fields_:
            lines.append(f'  printf("{S.__name__} {f[0]} %zu\\n", offsetof({S.__name__}, {f[0]}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        name, field, val = ln.split()
        got[(name, field)] = int(val)
    for S in structs:
        assert got[(S.__name__, "size")] == C.sizeof(S), S.__name__
        for f in S._fields_:
            assert got[(S.__name__, f[0])] == getattr(S, f[0]).offset, (S.__name__, f[0])


def _c_kind(decl):
    """(kind, bytes) of a C parameter or return type as written in include/*.h."""
    t = " ".join(decl.replace("const", " ").split())
    t = re.sub(r"\s+\w+$", "", t) if not t.endswith("*") and len(t.split()) > 1 else t
    if "*" in t or t in ("scivr_pes", "scivr_batch"):
        return ("ptr", C.sizeof(C.c_void_p))
    table = {"int": ("int", 4), "int32_t": ("int", 4), "int64_t": ("int", 8), "uint64_t": ("uint", 8),
             "uint8_t": ("uint", 1), "double": ("float", 8), "float": ("float", 4)}
    return table[t]


def _ctypes_kind(t):
    if t is None:
        return None
    if t in (C.c_void_p, C.c_char_p) or issubclass(t, C._Pointer):
        return ("ptr", C.sizeof(C.c_void_p))
    if t in (C.c_double, C.c_float):
        return ("float", C.sizeof(t))
    signed = t(-1).value < 0
    return ("int" if signed else "uint", C.sizeof(t))


def test_binding_signatures_match_the_headers():
    """argtypes and restype of every declared entry point agree with the C declaration
    (pointer, signed/unsigned integer or floating point, and width)."""
    import glob
    from paper_1312_4698_gb300 import scivr
    text = "".join(open(f).read() for f in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))))
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    decls = re.findall(r"([A-Za-z_][\w\s\*]*?)\b(scivr_\w+)\s*\(([^;{]*?)\)\s*;", text)
    assert len(decls) >= 20
    for ret, name, args in decls:
        fn = getattr(scivr._lib, name)
        params = [a.strip() for a in args.split(",") if a.strip() and a.strip() != "void"]
        assert fn.argtypes is not None and len(fn.argtypes) == len(params), name
        for decl, t in zip(params, fn.argtypes):
            assert _ctypes_kind(t) == _c_kind(decl), (name, decl, t)
        assert _ctypes_kind(fn.restype) == _c_kind(ret.strip()), (name, ret, fn.restype)


def test_missing_library_fails_loudly():
    """Without libscivr.so the binding refuses to import: there is no CPU fallback."""
    import subprocess
    import sys
    code = ("import paper_1312_4698_gb300.build as b; b.LIB = '/nonexistent/libscivr.so'\n"
            "try:\n"
            "    import paper_1312_4698_gb300.scivr\n"
            "except ImportError as e:\n"
            "    print('ImportError:', e)\n"
            "else:\n"
            "    raise SystemExit('imported without the library')\n")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-1500:]
    assert "ImportError: libscivr.so is not built" in out.stdout


def test_no_gpu_means_an_error_not_a_fallback(lib):
    """On a machine without a GPU the first call that needs the device returns a CUDA
    error code; nothing is computed on the host instead."""
    import torch
    from paper_1312_4698_gb300 import scivr
    from paper_1312_4698_gb300 import workloads as wl
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(scivr.ScivrError) as ei:
        scivr.scivr_create_pes(wl.config_f3().pes)
    assert ei.value.code in (scivr.SCIVR_ECUDA, scivr.SCIVR_ENOMEM)
    assert scivr.last_error().startswith("scivr_create_pes")
    import __graft_entry__ as ge
    with pytest.raises(AssertionError, match="needs cuda:0"):
        ge.smoke()
