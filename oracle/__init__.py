"""FP64 CPU oracle for TA-SC-IVR power spectra (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The library in ``paper_1312_4698_gb300`` never
imports it, and the two share no code: this wrapper loads ``scivr_oracle.c``
(plain C, libm, compiled with gcc) through ctypes.

Parity status of each function (what pins it, in ``tests/test_oracle_*.py``):
  pes_eval          finite differences, Euler homogeneity, Morse closed forms
  log_overlap       numerical quadrature of the coherent-state wavefunctions
  det_real/complex  numpy.linalg.det (LAPACK) on random matrices
  propagate         harmonic closed form (Glauber coherent-state algebra),
                    also where arg det A turns by more than pi per step
                    (24 modes); symplecticity M^T J M = J (F up to 24),
                    energy O(dt^4), time reversal, finite-difference
                    monodromy, order-4 convergence, generating-function
                    identity of the action; non-finite starts flagged bad;
                    the prefactor matrix is the analytic block of the
                    symplectic map in complex coordinates (A A^+ - B B^+ = I)
    (HK summands)   harmonic ground state (every summand the exact phase),
                    exact survival amplitude for widths gamma != omega
                    (the prefactor modulus |det A|^{1/2}),
                    displaced coherent-state autocorrelation, also for a
                    second state on trajectories drawn around the first
  spectrum          Dirichlet-kernel closed form, harmonic eigen-expansion,
                    Parseval, the sum rule (integral = <chi|chi>), 1D Morse
                    closed-form levels, exact levels and
                    coupling shifts of two coupled Morse modes (sinc DVR)
  spectrum_hk       Dirichlet kernel of the folded rectangle rule, 1D Morse
                    levels, exact levels and line weights of the coupled
                    Morse pair for one and two reference states
  sample_initial    Philox4x32-10 known-answer vectors, moments, the
                    resolution-of-identity expectation of the weights
  mlp_eval          fourth-order finite differences of the value (gradient,
                    Hessian), closed form of a network with zero weights
  mlp_loss_grad     central differences of the training objective
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "scivr_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_scivr.so")
_CFLAGS = ["-O2", "-std=gnu11", "-ffp-contract=off", "-fno-tree-vectorize", "-fopenmp",
           "-shared", "-fPIC"]
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (in-tree shared object)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *_CFLAGS, _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Mlp(C.Structure):
    _fields_ = [("H", C.c_int32), ("s_in", C.c_void_p), ("s_out", C.c_double),
                ("W1", C.c_void_p), ("b1", C.c_void_p), ("W2", C.c_void_p), ("b2", C.c_void_p),
                ("W3", C.c_void_p), ("b3", C.c_void_p), ("w4", C.c_void_p), ("b4", C.c_double)]


class _Pes(C.Structure):
    _fields_ = [("F", C.c_int32), ("diag_kind", C.c_int32),
                ("omega", C.c_void_p), ("D", C.c_void_p), ("a", C.c_void_p),
                ("n3", C.c_int32), ("idx3", C.c_void_p), ("c3", C.c_void_p),
                ("n4", C.c_int32), ("idx4", C.c_void_p), ("c4", C.c_void_p),
                ("mlp", C.c_void_p), ("cart", C.c_void_p)]


class _Cart(C.Structure):
    _fields_ = [("mass", C.c_double * 3), ("D", C.c_double * 2), ("a", C.c_double * 2),
                ("re", C.c_double * 2), ("k_bend", C.c_double), ("theta_e", C.c_double),
                ("x_eq", C.c_double * 9), ("Lm", C.c_double * 27)]


class _Prop(C.Structure):
    _fields_ = [("F", C.c_int32), ("n_steps", C.c_int32), ("dt", C.c_double),
                ("stab_tol", C.c_double), ("gamma", C.c_void_p), ("p_eq", C.c_void_p),
                ("q_eq", C.c_void_p), ("n_chi", C.c_int32), ("amplitude", C.c_int32)]


class _Cplx(C.Structure):
    _fields_ = [("re", C.c_double), ("im", C.c_double)]


class _Final(C.Structure):
    _fields_ = [("p", C.c_void_p), ("q", C.c_void_p), ("S", C.c_void_p), ("theta", C.c_void_p),
                ("detM", C.c_void_p), ("detA", C.c_void_p), ("M", C.c_void_p),
                ("stab", C.c_void_p)]


def _load():
    """Load the oracle library: the in-tree build, or the shared object named by
    SCIVR_ORACLE_LIB (the oracle's mutation tests load deliberately broken builds
    through it, in child processes)."""
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(os.environ.get("SCIVR_ORACLE_LIB") or build())
            vp, i32, i64, d = C.c_void_p, C.c_int32, C.c_int64, C.c_double
            lib.or_pes_eval.restype = d
            lib.or_pes_eval.argtypes = [vp, vp, vp, vp]
            lib.or_cart_eval.restype = d
            lib.or_cart_eval.argtypes = [vp, vp, vp, vp]
            lib.or_normal_modes.restype = d
            lib.or_normal_modes.argtypes = [vp, vp]
            lib.or_det_real.restype = d
            lib.or_det_real.argtypes = [C.c_int, vp]
            lib.or_det_complex.restype = _Cplx
            lib.or_det_complex.argtypes = [C.c_int, vp]
            lib.or_log_overlap.restype = _Cplx
            lib.or_log_overlap.argtypes = [C.c_int, vp, vp, vp, vp, vp]
            lib.or_propagate_one.restype = C.c_int
            lib.or_propagate_one.argtypes = [vp, vp, vp, vp, vp, i64, vp, vp, vp, vp, vp]
            lib.or_propagate.restype = C.c_int
            lib.or_propagate.argtypes = [vp, vp, i64, vp, vp, vp, i64, vp,
                                         vp, vp, vp, vp, vp, vp, vp, vp, C.c_int]
            lib.or_spectrum.restype = C.c_int
            lib.or_spectrum.argtypes = [vp, i64, vp, vp, i64, i32, d, d, d, i32, vp, vp, C.c_int]
            lib.or_spectrum_hk.restype = C.c_int
            lib.or_spectrum_hk.argtypes = [vp, i64, vp, i64, i32, d, d, d, i32, vp, vp, vp]
            lib.or_philox4x32_10.restype = None
            lib.or_philox4x32_10.argtypes = [vp, vp, vp]
            lib.or_sample_initial.restype = C.c_int
            lib.or_sample_initial.argtypes = [i32, vp, vp, vp, i64, C.c_uint64, vp, vp, vp]
            lib.or_max_threads.restype = C.c_int
            lib.or_mlp_eval.restype = None
            lib.or_mlp_eval.argtypes = [vp, C.c_int, vp, vp, vp, vp]
            lib.or_mlp_loss_grad.restype = d
            lib.or_mlp_loss_grad.argtypes = [vp, C.c_int, i64, vp, vp, vp, d, d, vp, vp, vp, vp, vp, vp,
                                             vp, vp]
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Mlp:
    """Owns FP64 copies of an MlpParams and the C struct pointing at them."""

    def __init__(self, m):
        self._keep = [_f64(m.s_in), _f64(m.W1), _f64(m.b1), _f64(m.W2), _f64(m.b2), _f64(m.W3),
                      _f64(m.b3), _f64(m.w4)]
        s_in, W1, b1, W2, b2, W3, b3, w4 = self._keep
        self.s = _Mlp(int(m.H), _p(s_in), float(m.s_out), _p(W1), _p(b1), _p(W2), _p(b2), _p(W3),
                      _p(b3), _p(w4), float(m.b4))


class Cart:
    """The oracle's Cartesian triatomic surface with its own normal-mode analysis
    (equilibrium geometry, Jacobi diagonalisation of the mass-weighted Hessian)."""

    def __init__(self, c):
        self.s = _Cart()
        self.s.mass[:] = [float(v) for v in c.mass]
        self.s.D[:] = [float(v) for v in c.D]
        self.s.a[:] = [float(v) for v in c.a]
        self.s.re[:] = [float(v) for v in c.re]
        self.s.k_bend = float(c.k_bend)
        self.s.theta_e = float(c.theta_e)
        om = np.zeros(3)
        self.rigid = float(_load().or_normal_modes(C.byref(self.s), _p(om)))
        self.omega = om
        self.x_eq = np.array(self.s.x_eq[:])
        self.Lm = np.array(self.s.Lm[:]).reshape(9, 3)


def normal_modes(c):
    """omega [3] (increasing), x_eq [9], Lm [9, 3] with x = x_eq + Lm q, and the largest
    rigid-body eigenvalue magnitude of the mass-weighted Hessian."""
    k = Cart(c)
    return k.omega, k.x_eq, k.Lm, k.rigid


def cart_eval(c, x):
    """V, gradient [9] and Hessian [9, 9] of the Cartesian surface at x [9]."""
    k = Cart(c)
    g = np.zeros(9)
    H = np.zeros((9, 9))
    V = _load().or_cart_eval(C.byref(k.s), _p(_f64(x)), _p(g), _p(H))
    return float(V), g, H


class Pes:
    """Owns contiguous copies of a descriptor's arrays and the C struct pointing at them."""

    def __init__(self, desc):
        cart = getattr(desc, "cart", None)
        if cart is not None:
            self.F = 3
            self._cart = Cart(cart)
            z = np.zeros(3)
            self._keep = [z]
            self.s = _Pes(3, 0, _p(z), _p(z), _p(z), 0, None, None, 0, None, None, None,
                          C.addressof(self._cart.s))
            return
        self.F = int(desc.F)
        self._keep = [_f64(desc.omega), _f64(desc.D), _f64(desc.a),
                      np.ascontiguousarray(desc.idx3, dtype=np.int32), _f64(desc.c3),
                      np.ascontiguousarray(desc.idx4, dtype=np.int32), _f64(desc.c4)]
        om, D, a, i3, c3, i4, c4 = self._keep
        mlp = getattr(desc, "mlp", None)
        self._mlp = Mlp(mlp) if mlp is not None else None
        self.s = _Pes(self.F, int(desc.diag_kind), _p(om), _p(D), _p(a),
                      c3.size, _p(i3), _p(c3), c4.size, _p(i4), _p(c4),
                      C.addressof(self._mlp.s) if self._mlp is not None else None)


def max_threads() -> int:
    return int(_load().or_max_threads())


def pes_eval(desc, q):
    """V, grad V [F], Hessian [F, F] at one point q [F]."""
    lib = _load()
    P = Pes(desc)
    q = _f64(q)
    g = np.zeros(P.F)
    H = np.zeros((P.F, P.F))
    V = lib.or_pes_eval(C.byref(P.s), _p(q), _p(g), _p(H))
    return float(V), g, H


def det_real(A):
    A = _f64(A).copy()
    return float(_load().or_det_real(A.shape[0], _p(A)))


def det_complex(A):
    A = np.ascontiguousarray(A, dtype=np.complex128).copy()
    r = _load().or_det_complex(A.shape[0], _p(A))
    return complex(r.re, r.im)


def log_overlap(gamma, p1, q1, p2, q2):
    """log <p1 q1 | p2 q2> for product coherent states of widths gamma."""
    gamma, p1, q1, p2, q2 = map(_f64, (gamma, p1, q1, p2, q2))
    r = _load().or_log_overlap(gamma.size, _p(gamma), _p(p1), _p(q1), _p(p2), _p(q2))
    return complex(r.re, r.im)


AMP_TA = 0   # time-averaged amplitude: <chi|p q> e^{i (S + theta/2)}
AMP_HK = 1   # Herman-Kluk summand of Eq. I(E)_SCIVR, weight included


def _prop_struct(F, gamma, p_eq, q_eq, dt, n_steps, stab_tol, amplitude=AMP_TA):
    gamma = _f64(gamma)
    p_eq = _f64(np.atleast_2d(p_eq))
    q_eq = _f64(np.atleast_2d(q_eq))
    s = _Prop(F, int(n_steps), float(dt), float(stab_tol), _p(gamma), _p(p_eq), _p(q_eq),
              p_eq.shape[0], int(amplitude))
    return s, (gamma, p_eq, q_eq)


def propagate_one(desc, gamma, p_eq, q_eq, dt, n_steps, p0, q0, stab_tol=1e-6, amplitude=AMP_TA):
    """One trajectory with full diagnostics.

    Returns a dict with amp [n_chi, K], good, the series S, theta, detA, detM
    [K] and the final p, q, M."""
    lib = _load()
    P = Pes(desc)
    F = P.F
    s, keep = _prop_struct(F, gamma, p_eq, q_eq, dt, n_steps, stab_tol, amplitude)
    K = n_steps + 1
    n_chi = keep[1].shape[0]
    amp = np.zeros((n_chi, K), dtype=np.complex128)
    S = np.zeros(K); th = np.zeros(K); dA = np.zeros(K, dtype=np.complex128); dM = np.zeros(K)
    fp = np.zeros(F); fq = np.zeros(F); fS = np.zeros(1); fth = np.zeros(1); fdM = np.zeros(1)
    fdA = np.zeros(1, dtype=np.complex128); fM = np.zeros((2 * F, 2 * F)); fst = np.zeros(1)
    fin = _Final(_p(fp), _p(fq), _p(fS), _p(fth), _p(fdM), _p(fdA), _p(fM), _p(fst))
    p0 = _f64(p0); q0 = _f64(q0)
    ok = lib.or_propagate_one(C.byref(P.s), C.byref(s), _p(p0), _p(q0), _p(amp), K,
                              C.byref(fin), _p(S), _p(th), _p(dA), _p(dM))
    return dict(amp=amp, good=bool(ok), S=S, theta=th, detA=dA, detM=dM, p=fp, q=fq, M=fM,
                stab=float(fst[0]))


def propagate(desc, gamma, p_eq, q_eq, dt, n_steps, p0, q0, stab_tol=1e-6, n_threads=0,
              final=False, amplitude=AMP_TA):
    """Batch propagation; p0, q0 are [F, n_traj] (variable-major).

    Returns amp [n_chi, n_traj, n_steps+1] complex128 and good [n_traj] uint8,
    plus a dict of final-state arrays when final=True."""
    lib = _load()
    P = Pes(desc)
    F = P.F
    p0 = _f64(p0); q0 = _f64(q0)
    n = p0.shape[1]
    s, keep = _prop_struct(F, gamma, p_eq, q_eq, dt, n_steps, stab_tol, amplitude)
    n_chi = keep[1].shape[0]
    K = n_steps + 1
    amp = np.zeros((n_chi, n, K), dtype=np.complex128)
    good = np.zeros(n, dtype=np.uint8)
    fin = None
    if final:
        fin = dict(p=np.zeros((n, F)), q=np.zeros((n, F)), S=np.zeros(n), theta=np.zeros(n),
                   detM=np.zeros(n), detA=np.zeros(n, dtype=np.complex128),
                   M=np.zeros((n, 2 * F, 2 * F)), stab=np.zeros(n))
    g = (lambda k: _p(fin[k])) if final else (lambda k: None)
    lib.or_propagate(C.byref(P.s), C.byref(s), n, _p(p0), _p(q0), _p(amp), K, _p(good),
                     g("p"), g("q"), g("S"), g("theta"), g("detM"), g("detA"), g("M"), g("stab"),
                     int(n_threads))
    return (amp, good, fin) if final else (amp, good)


def spectrum(amp, w, good, n_steps, dt, E_min, E_max, n_E, n_threads=0):
    """Eq. I(E)_discreto on amp [n_traj, K]; returns (I [n_E], n_good)."""
    lib = _load()
    amp = np.ascontiguousarray(amp, dtype=np.complex128)
    w = _f64(w)
    good = np.ascontiguousarray(good, dtype=np.uint8)
    I = np.zeros(int(n_E))
    ng = np.zeros(1, dtype=np.int64)
    lib.or_spectrum(_p(amp), amp.shape[1], _p(w), _p(good), amp.shape[0], int(n_steps),
                    float(dt), float(E_min), float(E_max), int(n_E), _p(I), _p(ng),
                    int(n_threads))
    return I, int(ng[0])


def spectrum_hk(amp, good, n_steps, dt, E_min, E_max, n_E):
    """Eq. I(E)_SCIVR on Herman-Kluk amplitudes amp [n_traj, K] (propagated with
    amplitude=AMP_HK); returns (I [n_E], n_good, survival amplitude C [K])."""
    lib = _load()
    amp = np.ascontiguousarray(amp, dtype=np.complex128)
    good = np.ascontiguousarray(good, dtype=np.uint8)
    I = np.zeros(int(n_E))
    ng = np.zeros(1, dtype=np.int64)
    Cs = np.zeros(amp.shape[1], dtype=np.complex128)
    lib.or_spectrum_hk(_p(amp), amp.shape[1], _p(good), amp.shape[0], int(n_steps), float(dt), float(E_min),
                       float(E_max), int(n_E), _p(I), _p(ng), _p(Cs))
    return I, int(ng[0]), Cs


def philox4x32_10(ctr, key):
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32)
    key = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().or_philox4x32_10(_p(ctr), _p(key), _p(out))
    return out


def sample_initial(gamma, p_eq, q_eq, n_traj, seed):
    """Husimi samples: returns p0, q0 [F, n_traj] and w [n_traj]."""
    gamma = _f64(gamma)
    p_eq = _f64(np.atleast_2d(p_eq)[0])
    q_eq = _f64(np.atleast_2d(q_eq)[0])
    F = gamma.size
    p0 = np.zeros((F, n_traj)); q0 = np.zeros((F, n_traj)); w = np.zeros(n_traj)
    _load().or_sample_initial(F, _p(gamma), _p(p_eq), _p(q_eq), int(n_traj),
                              C.c_uint64(int(seed)), _p(p0), _p(q0), _p(w))
    return p0, q0, w


def run_workload(wl, p0=None, q0=None, w=None, n_threads=0):
    """Sample (unless given), propagate and take the spectrum for every chi."""
    if p0 is None:
        p0, q0, w = sample_initial(wl.gamma, wl.p_eq, wl.q_eq, wl.n_traj, wl.seed)
    amp, good = propagate(wl.pes, wl.gamma, wl.p_eq, wl.q_eq, wl.dt, wl.n_steps, p0, q0,
                          wl.stab_tol, n_threads)
    spectra = []
    ng = 0
    for x in range(amp.shape[0]):
        I, ng = spectrum(amp[x], w, good, wl.n_steps, wl.dt, wl.E_min, wl.E_max, wl.n_E,
                         n_threads)
        spectra.append(I)
    return dict(p0=p0, q0=q0, w=w, amp=amp, good=good, I=np.stack(spectra), n_good=ng)


def mlp_eval(m, q):
    """V_mlp, its gradient [F] and Hessian [F, F] at one point q."""
    F = m.W1.shape[1]
    M = Mlp(m)
    q = _f64(q)
    V = np.zeros(1); g = np.zeros(F); H = np.zeros((F, F))
    _load().or_mlp_eval(C.byref(M.s), F, _p(q), _p(V), _p(g), _p(H))
    return float(V[0]), g, H


def mlp_loss_grad(m, q, Vref, gref, alpha, beta):
    """Training objective over samples q [n, F] and its parameter gradient (an MlpParams-shaped
    flat vector, same order as MlpParams.flat())."""
    F = m.W1.shape[1]
    H = m.H
    M = Mlp(m)
    q = _f64(q); Vref = _f64(Vref); gref = _f64(gref)
    d = [np.zeros(s) for s in m.sizes(F, H)]
    L = _load().or_mlp_loss_grad(C.byref(M.s), F, q.shape[0], _p(q), _p(Vref), _p(gref), float(alpha),
                                 float(beta), *[_p(x) for x in d])
    return float(L), np.concatenate(d)
