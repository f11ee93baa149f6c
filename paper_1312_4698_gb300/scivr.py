"""ctypes binding of libscivr (include/scivr.h), same names as the C ABI.

Argument marshalling only: every step of the computation runs in the CUDA
kernels of libscivr.so.  PyTorch supplies device memory and the current
stream.  Importing this module loads the library and raises ImportError if
it has not been built (``paper_1312_4698_gb300.build.build()``); there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

from . import build as _build

SCIVR_OK = 0
SCIVR_EINVAL = -1
SCIVR_ENOMEM = -2
SCIVR_ECUDA = -3
SCIVR_ETIMEOUT = -4
SCIVR_EUNSUPPORTED = -5

SCIVR_DIAG_HARMONIC = 0
SCIVR_DIAG_MORSE = 1
SCIVR_PES_POLY = 0
SCIVR_PES_CART3 = 1
SCIVR_FP64 = 0
SCIVR_MIXED = 1
SCIVR_FT_FP64 = 0
SCIVR_FT_TC_BF16 = 1
SCIVR_FT_TC_BF16X3 = 2
SCIVR_FT_TC_BF16X6 = 3
SCIVR_FT_CZT64 = 4
SCIVR_KERNEL_AUTO = 0
SCIVR_KERNEL_THREAD = 1
SCIVR_KERNEL_GROUP = 2
SCIVR_AMP_TA = 0
SCIVR_AMP_HK = 1
SCIVR_MAX_F = 24
SCIVR_MAX_CHI = 8

if not os.path.exists(_build.LIB):
    raise ImportError(f"libscivr.so is not built ({_build.LIB}); run "
                      "paper_1312_4698_gb300.build.build() on a machine with nvcc")

_lib = C.CDLL(_build.LIB)
LIBRARY_PATH = _build.LIB


class ScivrError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where} failed with status {code}: {last_error()}")


class scivr_pes_desc(C.Structure):
    _fields_ = [("F", C.c_int32), ("kind", C.c_int32), ("diag_kind", C.c_int32),
                ("omega", C.c_void_p), ("D", C.c_void_p), ("a", C.c_void_p),
                ("n3", C.c_int32), ("idx3", C.c_void_p), ("c3", C.c_void_p),
                ("n4", C.c_int32), ("idx4", C.c_void_p), ("c4", C.c_void_p)]


class scivr_prop_params(C.Structure):
    _fields_ = [("dt", C.c_double), ("n_steps", C.c_int32), ("precision", C.c_int32),
                ("stab_tol", C.c_double), ("gamma", C.c_void_p), ("p_eq", C.c_void_p),
                ("q_eq", C.c_void_p), ("n_chi", C.c_int32), ("kernel", C.c_int32),
                ("amplitude", C.c_int32), ("amp_prec", C.c_int32)]


class scivr_final_state(C.Structure):
    _fields_ = [("p", C.c_void_p), ("q", C.c_void_p), ("S", C.c_void_p), ("theta", C.c_void_p),
                ("detM", C.c_void_p), ("detA", C.c_void_p), ("M", C.c_void_p),
                ("stab", C.c_void_p)]


class scivr_batch_item(C.Structure):
    _fields_ = [("pes", C.c_void_p), ("prm", scivr_prop_params), ("n_traj", C.c_int64),
                ("p0", C.c_void_p), ("q0", C.c_void_p), ("w", C.c_void_p), ("amp", C.c_void_p),
                ("amp_ld", C.c_int64), ("good", C.c_void_p), ("E_min", C.c_double),
                ("E_max", C.c_double), ("n_E", C.c_int32), ("I_out", C.c_void_p),
                ("n_good_out", C.c_void_p)]


_vp, _i32, _i64, _d = C.c_void_p, C.c_int32, C.c_int64, C.c_double
_lib.scivr_create_pes.argtypes = [C.POINTER(scivr_pes_desc), C.POINTER(_vp)]
_lib.scivr_create_pes.restype = C.c_int
_lib.scivr_destroy_pes.argtypes = [_vp]
_lib.scivr_destroy_pes.restype = C.c_int
_lib.scivr_pes_modes.argtypes = [_vp]
_lib.scivr_pes_modes.restype = _i32
_lib.scivr_sample_initial.argtypes = [_vp, _vp, _vp, _vp, _i64, C.c_uint64, _vp, _vp, _vp, _vp]
_lib.scivr_sample_initial.restype = C.c_int
_lib.scivr_propagate.argtypes = [_vp, C.POINTER(scivr_prop_params), _i64, _vp, _vp, _vp, _i64,
                                 _vp, C.POINTER(scivr_final_state), _vp]
_lib.scivr_propagate.restype = C.c_int
_lib.scivr_spectrum.argtypes = [_vp, _i64, _i32, _vp, _vp, _i64, _i32, _d, _d, _d, _i32, _i32,
                                _vp, _vp, _vp]
_lib.scivr_spectrum.restype = C.c_int
_lib.scivr_spectrum_noalloc.argtypes = list(_lib.scivr_spectrum.argtypes)
_lib.scivr_spectrum_noalloc.restype = C.c_int
_lib.scivr_spectrum_hk.argtypes = [_vp, _i64, _vp, _i64, _i32, _d, _d, _d, _i32, _vp, _vp, _vp, _vp]
_lib.scivr_spectrum_hk.restype = C.c_int
_lib.scivr_batch_create.argtypes = [C.POINTER(scivr_batch_item), _i32, _i32, C.POINTER(_vp)]
_lib.scivr_batch_create.restype = C.c_int
_lib.scivr_batch_launch.argtypes = [_vp, _vp]
_lib.scivr_batch_launch.restype = C.c_int
_lib.scivr_batch_info.argtypes = [_vp, _i32, C.POINTER(_i32), C.POINTER(_i32), C.POINTER(_i32), C.POINTER(_i32)]
_lib.scivr_batch_info.restype = C.c_int
_lib.scivr_batch_schedule.argtypes = [_vp, C.POINTER(_i32)]
_lib.scivr_batch_schedule.restype = C.c_int
_lib.scivr_batch_destroy.argtypes = [_vp]
_lib.scivr_batch_destroy.restype = C.c_int
_lib.scivr_check_status.argtypes = [_vp]
_lib.scivr_check_status.restype = C.c_int
_lib.scivr_selftest_wait_timeout.argtypes = [_d, _vp]
_lib.scivr_selftest_wait_timeout.restype = C.c_int
_lib.scivr_last_error.argtypes = []
_lib.scivr_last_error.restype = C.c_char_p
_lib.scivr_launch_count.argtypes = [C.c_int]
_lib.scivr_launch_count.restype = _i64

EXPORTED = ["scivr_create_pes", "scivr_destroy_pes", "scivr_pes_modes", "scivr_sample_initial",
            "scivr_propagate", "scivr_spectrum", "scivr_spectrum_noalloc", "scivr_spectrum_hk", "scivr_check_status",
            "scivr_selftest_wait_timeout", "scivr_last_error", "scivr_launch_count",
            "scivr_batch_create", "scivr_batch_launch", "scivr_batch_info", "scivr_batch_destroy",
            "scivr_mlp_param_count", "scivr_pes_set_mlp", "scivr_mlp_eval", "scivr_mlp_get_params",
            "scivr_mlp_set_params", "scivr_mlp_loss_grad", "scivr_mlp_adamw", "scivr_pes_eval",
            "scivr_normal_modes", "scivr_normal_to_cartesian", "scivr_cartesian_to_normal",
            "scivr_create_pes_cartesian", "scivr_fma_probe", "scivr_batch_schedule"]


_lib.scivr_fma_probe.restype = C.c_int
_lib.scivr_fma_probe.argtypes = [_i32, _i64, C.POINTER(_d), _vp]


def scivr_fma_probe(precision, iters, stream=None) -> float:
    """Launch the FMA-rate probe on `stream`; returns the launch's flops."""
    f = _d()
    _check(_lib.scivr_fma_probe(int(precision), int(iters), C.byref(f), _stream(stream)), "scivr_fma_probe")
    return f.value


def scivr_check_status(stream=None) -> int:
    """Synchronise the stream and return (and clear) the device status (SCIVR_OK / SCIVR_ETIMEOUT)."""
    return int(_lib.scivr_check_status(_stream(stream)))


def scivr_selftest_wait_timeout(seconds: float, stream=None):
    _check(_lib.scivr_selftest_wait_timeout(float(seconds), _stream(stream)), "scivr_selftest_wait_timeout")


def last_error() -> str:
    return _lib.scivr_last_error().decode()


def launch_count(reset: bool = False) -> int:
    return int(_lib.scivr_launch_count(1 if reset else 0))


def _check(code, where):
    if code != SCIVR_OK:
        raise ScivrError(code, where)


def _ptr(x):
    """Device/host address of a torch tensor, numpy array, int or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Pes:
    """Owning handle of a scivr_pes (destroyed with the object)."""

    def __init__(self, handle: int, F: int):
        self.handle = handle
        self.F = F

    def close(self):
        if self.handle:
            _lib.scivr_destroy_pes(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class scivr_cart_triatomic(C.Structure):
    _fields_ = [("mass", C.c_double * 3), ("D", C.c_double * 2), ("a", C.c_double * 2),
                ("re", C.c_double * 2), ("k_bend", C.c_double), ("theta_e", C.c_double)]


_lib.scivr_normal_modes.restype = C.c_int
_lib.scivr_normal_modes.argtypes = [C.POINTER(scivr_cart_triatomic), _vp, _vp, _vp]
_lib.scivr_normal_to_cartesian.restype = C.c_int
_lib.scivr_normal_to_cartesian.argtypes = [C.POINTER(scivr_cart_triatomic), _i64, _vp, _vp]
_lib.scivr_cartesian_to_normal.restype = C.c_int
_lib.scivr_cartesian_to_normal.argtypes = [C.POINTER(scivr_cart_triatomic), _i64, _vp, _vp]
_lib.scivr_create_pes_cartesian.restype = C.c_int
_lib.scivr_create_pes_cartesian.argtypes = [C.POINTER(scivr_cart_triatomic), C.POINTER(_vp)]


def _cart_struct(c) -> scivr_cart_triatomic:
    s = scivr_cart_triatomic()
    s.mass[:] = [float(v) for v in c.mass]
    s.D[:] = [float(v) for v in c.D]
    s.a[:] = [float(v) for v in c.a]
    s.re[:] = [float(v) for v in c.re]
    s.k_bend = float(c.k_bend)
    s.theta_e = float(c.theta_e)
    return s


def scivr_normal_modes(c):
    """c: workloads.CartTriatomic.  Returns omega [3], x_eq [9], Lm [9, 3] (host arrays)."""
    om, xe, Lm = np.zeros(3), np.zeros(9), np.zeros((9, 3))
    _check(_lib.scivr_normal_modes(C.byref(_cart_struct(c)), om.ctypes.data, xe.ctypes.data, Lm.ctypes.data),
           "scivr_normal_modes")
    return om, xe, Lm


def scivr_normal_to_cartesian(c, q):
    q = _f64(np.atleast_2d(q))
    x = np.zeros((q.shape[0], 9))
    _check(_lib.scivr_normal_to_cartesian(C.byref(_cart_struct(c)), q.shape[0], q.ctypes.data, x.ctypes.data),
           "scivr_normal_to_cartesian")
    return x


def scivr_cartesian_to_normal(c, x):
    x = _f64(np.atleast_2d(x))
    q = np.zeros((x.shape[0], 3))
    _check(_lib.scivr_cartesian_to_normal(C.byref(_cart_struct(c)), x.shape[0], x.ctypes.data, q.ctypes.data),
           "scivr_cartesian_to_normal")
    return q


def scivr_create_pes_cartesian(c) -> Pes:
    h = _vp()
    _check(_lib.scivr_create_pes_cartesian(C.byref(_cart_struct(c)), C.byref(h)), "scivr_create_pes_cartesian")
    return Pes(h.value, 3)


def scivr_create_pes(desc) -> Pes:
    """desc: workloads.PesDesc-like object (F, diag_kind, omega, D, a, idx3, c3, idx4, c4), or a
    workloads.CartPes (a Cartesian surface in its normal modes)."""
    if getattr(desc, "cart", None) is not None:
        return scivr_create_pes_cartesian(desc.cart)
    keep = [_f64(desc.omega), _f64(desc.D), _f64(desc.a),
            np.ascontiguousarray(desc.idx3, dtype=np.int32), _f64(desc.c3),
            np.ascontiguousarray(desc.idx4, dtype=np.int32), _f64(desc.c4)]
    om, D, a, i3, c3, i4, c4 = keep
    d = scivr_pes_desc(int(desc.F), SCIVR_PES_POLY, int(desc.diag_kind), om.ctypes.data,
                       D.ctypes.data, a.ctypes.data, c3.size, i3.ctypes.data if c3.size else None,
                       c3.ctypes.data if c3.size else None, c4.size,
                       i4.ctypes.data if c4.size else None, c4.ctypes.data if c4.size else None)
    h = _vp()
    _check(_lib.scivr_create_pes(C.byref(d), C.byref(h)), "scivr_create_pes")
    pes = Pes(h.value, int(desc.F))
    if getattr(desc, "mlp", None) is not None:
        scivr_pes_set_mlp(pes, desc.mlp)
    return pes


create_pes = scivr_create_pes


def scivr_sample_initial(pes: Pes, gamma, p_eq, q_eq, n_traj, seed, p0, q0, w, stream=None):
    g, pe, qe = _f64(gamma), _f64(p_eq), _f64(q_eq)
    _check(_lib.scivr_sample_initial(pes.handle, g.ctypes.data, pe.ctypes.data, qe.ctypes.data,
                                     int(n_traj), C.c_uint64(int(seed)), _ptr(p0), _ptr(q0),
                                     _ptr(w), _stream(stream)), "scivr_sample_initial")


sample_initial = scivr_sample_initial


def scivr_propagate(pes: Pes, dt, n_steps, gamma, p_eq, q_eq, n_traj, p0, q0, amp, amp_ld, good,
                    precision=SCIVR_FP64, stab_tol=1e-6, fin: Optional[dict] = None, stream=None,
                    kernel=SCIVR_KERNEL_AUTO, amplitude=SCIVR_AMP_TA, amp_prec=None):
    """p_eq, q_eq: [n_chi, F] host arrays.  fin: optional dict of device tensors.
    amplitude: SCIVR_AMP_TA (time-averaging integrand) or SCIVR_AMP_HK (plain
    Herman-Kluk summand).  amp_prec: SCIVR_FP64 (complex double) or SCIVR_MIXED
    (complex float); None takes it from amp's dtype (float32 -> SCIVR_MIXED)."""
    amp_prec = _amp_prec_of(amp, amp_prec)
    g = _f64(gamma)
    pe = _f64(np.atleast_2d(p_eq))
    qe = _f64(np.atleast_2d(q_eq))
    prm = scivr_prop_params(float(dt), int(n_steps), int(precision), float(stab_tol),
                            g.ctypes.data, pe.ctypes.data, qe.ctypes.data, pe.shape[0], int(kernel),
                            int(amplitude), int(amp_prec))
    fs = None
    if fin:
        fs = scivr_final_state(*[_ptr(fin.get(k)) for k in ("p", "q", "S", "theta", "detM", "detA", "M",
                                                            "stab")])
    _check(_lib.scivr_propagate(pes.handle, C.byref(prm), int(n_traj), _ptr(p0), _ptr(q0), _ptr(amp),
                                int(amp_ld), _ptr(good), C.byref(fs) if fs is not None else None,
                                _stream(stream)), "scivr_propagate")


propagate = scivr_propagate


def _amp_prec_of(amp, amp_prec):
    if amp_prec is None:
        return SCIVR_MIXED if str(getattr(amp, "dtype", "")).endswith("float32") else SCIVR_FP64
    return amp_prec


def scivr_spectrum(amp, amp_ld, w, good, n_traj, n_steps, dt, E_min, E_max, n_E, I_out,
                   n_good_out=None, amp_prec=None, ft_mode=SCIVR_FT_FP64, stream=None):
    """amp_prec None: from amp's dtype (float32 rows are the FP32 storage)."""
    amp_prec = _amp_prec_of(amp, amp_prec)
    _check(_lib.scivr_spectrum(_ptr(amp), int(amp_ld), int(amp_prec), _ptr(w), _ptr(good),
                               int(n_traj), int(n_steps), float(dt), float(E_min), float(E_max),
                               int(n_E), int(ft_mode), _ptr(I_out), _ptr(n_good_out),
                               _stream(stream)), "scivr_spectrum")


spectrum = scivr_spectrum


def scivr_spectrum_hk(amp, amp_ld, good, n_traj, n_steps, dt, E_min, E_max, n_E, I_out, C_out=None,
                      n_good_out=None, stream=None):
    """Plain HK SC-IVR spectrum from the summands written with amplitude=SCIVR_AMP_HK."""
    _check(_lib.scivr_spectrum_hk(_ptr(amp), int(amp_ld), _ptr(good), int(n_traj), int(n_steps), float(dt),
                                  float(E_min), float(E_max), int(n_E), _ptr(I_out), _ptr(C_out),
                                  _ptr(n_good_out), _stream(stream)), "scivr_spectrum_hk")


def scivr_spectrum_noalloc(amp, amp_ld, w, good, n_traj, n_steps, dt, E_min, E_max, n_E, I_out,
                           n_good_out=None, amp_prec=None, ft_mode=SCIVR_FT_FP64, stream=None):
    """scivr_spectrum without device allocations (library-owned fixed scratch; calls must not overlap)."""
    amp_prec = _amp_prec_of(amp, amp_prec)
    _check(_lib.scivr_spectrum_noalloc(_ptr(amp), int(amp_ld), int(amp_prec), _ptr(w), _ptr(good),
                                       int(n_traj), int(n_steps), float(dt), float(E_min),
                                       float(E_max), int(n_E), int(ft_mode), _ptr(I_out),
                                       _ptr(n_good_out), _stream(stream)), "scivr_spectrum_noalloc")


# --------------------------------------------------------------------------
# Convenience: allocate outputs with torch and run the whole path on a workload
# --------------------------------------------------------------------------

@dataclass
class Buffers:
    p0: "object"
    q0: "object"
    w: "object"
    amp: "object"
    good: "object"
    I: "object"
    n_good: "object"


def alloc_buffers(wl, device="cuda", n_traj=None, amp_f32=False):
    """amp_f32: complex-float amplitude rows (the mixed path's 8-byte storage)."""
    import torch
    n = wl.n_traj if n_traj is None else n_traj
    K = wl.n_steps + 1
    return Buffers(
        p0=torch.empty((wl.F, n), dtype=torch.float64, device=device),
        q0=torch.empty((wl.F, n), dtype=torch.float64, device=device),
        w=torch.empty(n, dtype=torch.float64, device=device),
        amp=torch.empty((wl.n_chi, n, K, 2), dtype=torch.float32 if amp_f32 else torch.float64, device=device),
        good=torch.empty(n, dtype=torch.uint8, device=device),
        I=torch.empty((wl.n_chi, wl.n_E), dtype=torch.float64, device=device),
        n_good=torch.zeros(1, dtype=torch.int64, device=device),
    )


def run_spectrum_path(pes: Pes, wl, bufs: Buffers, sample=True, precision=SCIVR_FP64,
                      ft_mode=SCIVR_FT_FP64, stream=None):
    """sample (optional) -> propagate -> spectrum for every reference state, all on the GPU."""
    n = bufs.w.shape[0]
    K = wl.n_steps + 1
    if sample:
        scivr_sample_initial(pes, wl.gamma, wl.p_eq[0], wl.q_eq[0], n, wl.seed, bufs.p0, bufs.q0,
                             bufs.w, stream)
    scivr_propagate(pes, wl.dt, wl.n_steps, wl.gamma, wl.p_eq, wl.q_eq, n, bufs.p0, bufs.q0,
                    bufs.amp, K, bufs.good, precision=precision, stab_tol=wl.stab_tol, stream=stream)
    for x in range(wl.n_chi):
        scivr_spectrum(bufs.amp[x], K, bufs.w, bufs.good, n, wl.n_steps, wl.dt, wl.E_min, wl.E_max,
                       wl.n_E, bufs.I[x], bufs.n_good, ft_mode=ft_mode, stream=stream)


# --------------------------------------------------------------------------
# Batched runs
# --------------------------------------------------------------------------

class Batch:
    """Owning handle of a scivr_batch plan; keeps the host arrays its items point at alive."""

    def __init__(self, handle, keep):
        self.handle = handle
        self._keep = keep

    def one_launch(self) -> bool:
        """True when every mixed-precision molecule runs in one persistent launch."""
        v = _i32()
        _check(_lib.scivr_batch_schedule(self.handle, C.byref(v)), "scivr_batch_schedule")
        return bool(v.value)

    def groups(self):
        n = _i32()
        _check(_lib.scivr_batch_info(self.handle, -1, C.byref(n), None, None, None), "scivr_batch_info")
        out = []
        for g in range(n.value):
            F, pr, w = _i32(), _i32(), _i32()
            _check(_lib.scivr_batch_info(self.handle, g, None, C.byref(F), C.byref(pr), C.byref(w)),
                   "scivr_batch_info")
            out.append((F.value, pr.value, w.value))
        return out

    def close(self):
        if self.handle:
            _lib.scivr_batch_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def scivr_batch_create(entries, ft_mode=SCIVR_FT_FP64) -> Batch:
    """entries: list of dicts with keys pes (Pes), wl (workloads.Workload), bufs (Buffers),
    precision, stab_tol.  Each molecule uses its own buffers (p0, q0, w, amp, good, I, n_good)."""
    n = len(entries)
    arr = (scivr_batch_item * n)()
    keep = []
    for i, e in enumerate(entries):
        wl, bufs = e["wl"], e["bufs"]
        g = _f64(wl.gamma)
        pe = _f64(np.atleast_2d(wl.p_eq))
        qe = _f64(np.atleast_2d(wl.q_eq))
        keep += [g, pe, qe, e["pes"]]
        prm = scivr_prop_params(float(wl.dt), int(wl.n_steps), int(e.get("precision", SCIVR_MIXED)),
                                float(e.get("stab_tol", wl.stab_tol)), g.ctypes.data, pe.ctypes.data,
                                qe.ctypes.data, pe.shape[0], int(e.get("kernel", SCIVR_KERNEL_AUTO)),
                                SCIVR_AMP_TA, int(_amp_prec_of(bufs.amp, None)))
        arr[i] = scivr_batch_item(e["pes"].handle, prm, int(bufs.w.shape[0]), _ptr(bufs.p0), _ptr(bufs.q0),
                                  _ptr(bufs.w), _ptr(bufs.amp), int(wl.n_steps) + 1, _ptr(bufs.good),
                                  float(wl.E_min), float(wl.E_max), int(wl.n_E), _ptr(bufs.I),
                                  _ptr(bufs.n_good))
    h = _vp()
    _check(_lib.scivr_batch_create(arr, n, int(ft_mode), C.byref(h)), "scivr_batch_create")
    return Batch(h.value, keep)


def scivr_batch_launch(batch: Batch, stream=None):
    _check(_lib.scivr_batch_launch(batch.handle, _stream(stream)), "scivr_batch_launch")


# ---------------------------------------------------------------- learned residual (include/scivr_mlp.h)
SCIVR_MLP_HIDDEN = 256
SCIVR_TERMS_ALL = 0
SCIVR_TERMS_DIAG = 1
SCIVR_TERMS_COUPLING = 2


class scivr_mlp_desc(C.Structure):
    _fields_ = [("H", _i32), ("s_in", _vp), ("s_out", _d), ("W1", _vp), ("b1", _vp), ("W2", _vp),
                ("b2", _vp), ("W3", _vp), ("b3", _vp), ("w4", _vp), ("b4", _d)]


_lib.scivr_mlp_param_count.argtypes = [_i32, _i32]
_lib.scivr_mlp_param_count.restype = _i64
_lib.scivr_pes_set_mlp.argtypes = [_vp, C.POINTER(scivr_mlp_desc)]
_lib.scivr_pes_set_mlp.restype = C.c_int
_lib.scivr_mlp_eval.argtypes = [_vp, _i64, _vp, _vp, _vp, _vp, _vp]
_lib.scivr_mlp_eval.restype = C.c_int
_lib.scivr_mlp_get_params.argtypes = [_vp, _vp, _vp]
_lib.scivr_mlp_get_params.restype = C.c_int
_lib.scivr_mlp_set_params.argtypes = [_vp, _vp, _vp]
_lib.scivr_mlp_set_params.restype = C.c_int
_lib.scivr_mlp_loss_grad.argtypes = [_vp, _i64, _vp, _vp, _vp, _d, _d, _vp, _vp, _vp]
_lib.scivr_mlp_loss_grad.restype = C.c_int
_lib.scivr_mlp_adamw.argtypes = [_vp, _vp, _vp, _vp, _i32, _d, _d, _d, _d, _d, _vp]
_lib.scivr_mlp_adamw.restype = C.c_int
_lib.scivr_pes_eval.argtypes = [_vp, _i64, _vp, _i32, _vp, _vp, _vp, _vp]
_lib.scivr_pes_eval.restype = C.c_int


def scivr_mlp_param_count(F: int, H: int = SCIVR_MLP_HIDDEN) -> int:
    return int(_lib.scivr_mlp_param_count(int(F), int(H)))


def scivr_pes_set_mlp(pes: Pes, m):
    """Attach (or with m=None detach) a learned residual; m: workloads.MlpParams-like."""
    if m is None:
        _check(_lib.scivr_pes_set_mlp(pes.handle, None), "scivr_pes_set_mlp")
        return
    keep = [_f64(m.s_in), _f64(m.W1), _f64(m.b1), _f64(m.W2), _f64(m.b2), _f64(m.W3), _f64(m.b3), _f64(m.w4)]
    si, W1, b1, W2, b2, W3, b3, w4 = keep
    d = scivr_mlp_desc(int(m.H), si.ctypes.data, float(m.s_out), W1.ctypes.data, b1.ctypes.data,
                       W2.ctypes.data, b2.ctypes.data, W3.ctypes.data, b3.ctypes.data, w4.ctypes.data,
                       float(m.b4))
    _check(_lib.scivr_pes_set_mlp(pes.handle, C.byref(d)), "scivr_pes_set_mlp")


def scivr_mlp_eval(pes: Pes, n, q, V, g, H=None, stream=None):
    _check(_lib.scivr_mlp_eval(pes.handle, int(n), _ptr(q), _ptr(V), _ptr(g), _ptr(H), _stream(stream)),
           "scivr_mlp_eval")


def scivr_mlp_get_params(pes: Pes, theta, stream=None):
    _check(_lib.scivr_mlp_get_params(pes.handle, _ptr(theta), _stream(stream)), "scivr_mlp_get_params")


def scivr_mlp_set_params(pes: Pes, theta, stream=None):
    _check(_lib.scivr_mlp_set_params(pes.handle, _ptr(theta), _stream(stream)), "scivr_mlp_set_params")


def scivr_mlp_loss_grad(pes: Pes, n, q, Vref, gref, alpha, beta, grad, loss, stream=None):
    _check(_lib.scivr_mlp_loss_grad(pes.handle, int(n), _ptr(q), _ptr(Vref), _ptr(gref), float(alpha),
                                    float(beta), _ptr(grad), _ptr(loss), _stream(stream)), "scivr_mlp_loss_grad")


def scivr_mlp_adamw(pes: Pes, grad, m1, m2, t, lr, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0,
                    stream=None):
    _check(_lib.scivr_mlp_adamw(pes.handle, _ptr(grad), _ptr(m1), _ptr(m2), int(t), float(lr), float(beta1),
                                float(beta2), float(eps), float(weight_decay), _stream(stream)), "scivr_mlp_adamw")


def scivr_pes_eval(pes: Pes, n, q, terms, V, g=None, H=None, stream=None):
    _check(_lib.scivr_pes_eval(pes.handle, int(n), _ptr(q), int(terms), _ptr(V), _ptr(g), _ptr(H),
                               _stream(stream)), "scivr_pes_eval")
