"""Seeded synthetic workloads for TA-SC-IVR power spectra.

This module only draws and packs inputs: potential descriptors (Morse
diagonal plus random cubic/quartic couplings), the reference coherent state
chi, the widths gamma, time step, step count and energy grid. It holds none
of the method's arithmetic (no propagation, overlaps, prefactors or Fourier
sums), so both the CPU oracle and the CUDA path can consume its output.

Units: atomic units, hbar = 1, mass-weighted normal coordinates (m = 1).

The molecules of the paper (H2, H2O, H2CO, CH2D2 with F = 1/3/6/9, Sec. IV)
use fitted ab-initio surfaces that are not reproduced here; the synthetic
recipes below have the same numbers of modes and frequency ranges.
"""
from __future__ import annotations

import dataclasses
import itertools
from typing import List, Optional

import numpy as np

CM1_PER_EH = 219474.6313632  # 1 hartree in cm^-1

DIAG_HARMONIC = 0
DIAG_MORSE = 1


def cm1(x):
    """Convert wavenumbers (cm^-1) to hartree."""
    return np.asarray(x, dtype=np.float64) / CM1_PER_EH


def to_cm1(x):
    """Convert hartree to wavenumbers (cm^-1)."""
    return np.asarray(x, dtype=np.float64) * CM1_PER_EH


def offdiag_monomials(F: int, degree: int) -> np.ndarray:
    """Index tuples i <= j <= ... of the given degree, excluding all-equal ones.

    The all-equal (diagonal) anharmonicity is carried by the Morse term, so
    the coupling polynomial only holds mixed monomials.  Lexicographic order.
    """
    out = [t for t in itertools.combinations_with_replacement(range(F), degree)
           if len(set(t)) > 1]
    return np.asarray(out, dtype=np.int32).reshape(-1, degree)


@dataclasses.dataclass
class PesDesc:
    """Potential V(q) = sum_i diag_i(q_i) + sum c3 q_i q_j q_k + sum c4 q_i q_j q_k q_l.

    diag_kind == DIAG_HARMONIC: diag_i = omega_i^2 q_i^2 / 2.
    diag_kind == DIAG_MORSE:    diag_i = D_i (1 - exp(-a_i q_i))^2.
    idx3: [n3, 3] int32 with i <= j <= k; idx4: [n4, 4] int32 with i <= j <= k <= l.
    """
    F: int
    diag_kind: int
    omega: np.ndarray
    D: np.ndarray
    a: np.ndarray
    idx3: np.ndarray
    c3: np.ndarray
    idx4: np.ndarray
    c4: np.ndarray
    mlp: Optional["MlpParams"] = None   # learned residual added to V (None: analytic only)

    def __post_init__(self):
        self.omega = np.ascontiguousarray(self.omega, dtype=np.float64)
        self.D = np.ascontiguousarray(self.D, dtype=np.float64)
        self.a = np.ascontiguousarray(self.a, dtype=np.float64)
        self.idx3 = np.ascontiguousarray(np.asarray(self.idx3, dtype=np.int32).reshape(-1, 3))
        self.c3 = np.ascontiguousarray(self.c3, dtype=np.float64).reshape(-1)
        self.idx4 = np.ascontiguousarray(np.asarray(self.idx4, dtype=np.int32).reshape(-1, 4))
        self.c4 = np.ascontiguousarray(self.c4, dtype=np.float64).reshape(-1)


AMU = 1822.888486209  # unified atomic mass unit in electron masses


@dataclasses.dataclass
class CartTriatomic:
    """Cartesian surface of a bent triatomic: atoms 0 and 2 bonded to the central atom 1,
    V(x) = sum_b D_b (1 - exp(-a_b (r_b - re_b)))^2 + (k_bend / 2) (cos theta - cos theta_e)^2
    with r_0 = |x0 - x1|, r_1 = |x2 - x1| and theta the angle 0-1-2.  x: [9] Cartesian
    coordinates (bohr), atom-major; masses in electron masses.  Its normal modes (the
    coordinates the propagation runs in) come from the mass-weighted Hessian at the
    equilibrium geometry (Sec. III.A)."""
    mass: np.ndarray          # [3]
    D: np.ndarray             # [2] Morse depths (hartree)
    a: np.ndarray             # [2] Morse range parameters (1/bohr)
    re: np.ndarray            # [2] equilibrium bond lengths (bohr)
    k_bend: float             # hartree
    theta_e: float            # equilibrium angle (rad)

    @property
    def F(self) -> int:
        return 3


@dataclasses.dataclass
class CartPes:
    """A potential given as a Cartesian surface (F = 3 vibrational normal modes)."""
    cart: CartTriatomic

    @property
    def F(self) -> int:
        return 3


def water_like_triatomic() -> CartTriatomic:
    """Synthetic water-sized surface: H-O-H masses, bonds of 1.81 bohr at 104.5 degrees,
    Morse depth 0.2 hartree; a = 1.1 / bohr and k_bend = 0.16 hartree put the stretches
    near 3650-3700 cm^-1 and the bend near 1600 cm^-1 (the F = 3 workload's range)."""
    m_h, m_o = 1.00782503223 * AMU, 15.99491461957 * AMU
    return CartTriatomic(mass=np.array([m_h, m_o, m_h]), D=np.array([0.2, 0.2]), a=np.array([1.1, 1.1]),
                         re=np.array([1.81, 1.81]), k_bend=0.16, theta_e=float(np.deg2rad(104.5)))


@dataclasses.dataclass
class MlpParams:
    """Learned residual V_mlp(q) = s_out * (w4 . a3 + b4) on x = s_in * q (a_l = silu(z_l)).
    W1: [H, F], W2, W3: [H, H] (row-major, output index first)."""
    H: int
    s_in: np.ndarray
    s_out: float
    W1: np.ndarray
    b1: np.ndarray
    W2: np.ndarray
    b2: np.ndarray
    W3: np.ndarray
    b3: np.ndarray
    w4: np.ndarray
    b4: float

    def copy(self):
        return MlpParams(self.H, self.s_in.copy(), float(self.s_out), self.W1.copy(), self.b1.copy(),
                         self.W2.copy(), self.b2.copy(), self.W3.copy(), self.b3.copy(), self.w4.copy(),
                         float(self.b4))

    def flat(self) -> np.ndarray:
        return np.concatenate([self.W1.ravel(), self.b1, self.W2.ravel(), self.b2, self.W3.ravel(),
                               self.b3, self.w4, [self.b4]])

    @staticmethod
    def sizes(F, H):
        return [H * F, H, H * H, H, H * H, H, H, 1]

    def with_flat(self, v: np.ndarray) -> "MlpParams":
        F = self.W1.shape[1]
        H = self.H
        o = np.cumsum([0] + self.sizes(F, H))
        return MlpParams(H, self.s_in.copy(), float(self.s_out), v[o[0]:o[1]].reshape(H, F).copy(),
                         v[o[1]:o[2]].copy(), v[o[2]:o[3]].reshape(H, H).copy(), v[o[3]:o[4]].copy(),
                         v[o[4]:o[5]].reshape(H, H).copy(), v[o[5]:o[6]].copy(), v[o[6]:o[7]].copy(),
                         float(v[o[7]]))


def init_mlp(F: int, H: int = 256, seed: int = 0, s_in=None, s_out: float = 1e-6) -> MlpParams:
    """Seeded random initialisation (scaled normal, zero biases)."""
    rng = np.random.default_rng(seed)
    s_in = np.ones(F) if s_in is None else np.asarray(s_in, dtype=np.float64)
    return MlpParams(H, s_in, float(s_out),
                     rng.normal(0, 1 / np.sqrt(F), (H, F)), np.zeros(H),
                     rng.normal(0, 1 / np.sqrt(H), (H, H)), np.zeros(H),
                     rng.normal(0, 1 / np.sqrt(H), (H, H)), np.zeros(H),
                     rng.normal(0, 1 / np.sqrt(H), H), 0.0)


@dataclasses.dataclass
class Workload:
    """Everything one spectrum run needs, apart from the random phase-space samples."""
    name: str
    pes: PesDesc
    gamma: np.ndarray        # [F] coherent-state widths
    p_eq: np.ndarray         # [n_chi, F] reference state momenta
    q_eq: np.ndarray         # [n_chi, F] reference state positions
    n_traj: int
    n_steps: int
    dt: float
    E_min: float
    E_max: float
    n_E: int
    seed: int
    stab_tol: float = 1e-6

    @property
    def F(self) -> int:
        return self.pes.F

    @property
    def n_chi(self) -> int:
        return self.p_eq.shape[0]

    def energies(self) -> np.ndarray:
        """The equally spaced grid E_1 = E_min ... E_k = E_max (Sec. III.A)."""
        return np.linspace(self.E_min, self.E_max, self.n_E)

    def with_(self, **kw) -> "Workload":
        return dataclasses.replace(self, **kw)


def harmonic_pes(omega) -> PesDesc:
    omega = np.asarray(omega, dtype=np.float64)
    F = omega.size
    z = np.zeros(F)
    return PesDesc(F, DIAG_HARMONIC, omega, z, z, np.zeros((0, 3)), np.zeros(0),
                   np.zeros((0, 4)), np.zeros(0))


def morse_pes(omega, D, idx3=None, c3=None, idx4=None, c4=None) -> PesDesc:
    """Morse diagonal with a_i = omega_i / sqrt(2 D_i) (so V ~ omega^2 q^2 / 2 near 0)."""
    omega = np.asarray(omega, dtype=np.float64)
    D = np.broadcast_to(np.asarray(D, dtype=np.float64), omega.shape).copy()
    a = omega / np.sqrt(2.0 * D)
    F = omega.size
    return PesDesc(F, DIAG_MORSE, omega, D, a,
                   np.zeros((0, 3)) if idx3 is None else idx3,
                   np.zeros(0) if c3 is None else c3,
                   np.zeros((0, 4)) if idx4 is None else idx4,
                   np.zeros(0) if c4 is None else c4)


def ground_chi(omega, n_quanta=None):
    """Reference state centred at q = 0 with p_i = sqrt((2 n_i + 1) omega_i)."""
    omega = np.asarray(omega, dtype=np.float64)
    n = np.zeros_like(omega) if n_quanta is None else np.asarray(n_quanta, dtype=np.float64)
    return np.sqrt((2.0 * n + 1.0) * omega), np.zeros_like(omega)


def grid_window(omega, width_cm1=12000.0, below_cm1=1500.0):
    """Energy window for F >= 6 grids: it starts 1500 cm^-1 below the harmonic ZPE."""
    zpe = 0.5 * float(np.sum(omega))
    lo = max(0.0, zpe - float(cm1(below_cm1)))
    return lo, lo + float(cm1(width_cm1))


COUPLING_MASS_WEIGHTED = "mass_weighted"
COUPLING_DIMENSIONLESS = "dimensionless"


def recipe_pes(F: int, rng: np.random.Generator, sigma3=1e-7, sigma4=1e-8,
               w_lo=1100.0, w_hi=3000.0, D_lo=0.15, D_hi=0.25, quartic=True,
               units: str = COUPLING_MASS_WEIGHTED) -> PesDesc:
    """Random Morse + cubic + quartic surface.  Draw order: omega, D, cubic, quartic.

    units == "mass_weighted": the drawn coefficients (hartree) multiply the
    mass-weighted coordinates q directly.
    units == "dimensionless": they multiply dimensionless normal coordinates
    Q_i = sqrt(omega_i) q_i (the usual force-field convention), so the stored
    coefficient of q_i q_j q_k is c_ijk sqrt(omega_i omega_j omega_k), and
    likewise for the quartic terms.
    """
    omega = cm1(rng.uniform(w_lo, w_hi, F))
    D = rng.uniform(D_lo, D_hi, F)
    idx3 = offdiag_monomials(F, 3)
    c3 = rng.normal(0.0, sigma3, idx3.shape[0])
    if quartic:
        idx4 = offdiag_monomials(F, 4)
        c4 = rng.normal(0.0, sigma4, idx4.shape[0])
    else:
        idx4, c4 = np.zeros((0, 4), np.int32), np.zeros(0)
    if units == COUPLING_DIMENSIONLESS:
        c3 = c3 * np.sqrt(np.prod(omega[idx3], axis=1)) if c3.size else c3
        c4 = c4 * np.sqrt(np.prod(omega[idx4], axis=1)) if c4.size else c4
    elif units != COUPLING_MASS_WEIGHTED:
        raise ValueError(f"unknown coupling units {units!r}")
    return morse_pes(omega, D, idx3, c3, idx4, c4)


def _single_chi(omega):
    p, q = ground_chi(omega)
    return p[None, :], q[None, :]


def config_f3(seed: int = 0, n_traj: int = 1024, n_steps: int = 3000, n_E: int = 2000) -> Workload:
    """F = 3 (water-sized): Morse 1600/3650/3750 cm^-1, D = 0.2, 7 cubic couplings."""
    rng = np.random.default_rng(seed)
    omega = cm1([1600.0, 3650.0, 3750.0])
    idx3 = offdiag_monomials(3, 3)
    c3 = rng.normal(0.0, 1e-7, idx3.shape[0])
    pes = morse_pes(omega, 0.2, idx3, c3)
    p_eq, q_eq = _single_chi(omega)
    return Workload("f3_morse_cubic", pes, omega.copy(), p_eq, q_eq, n_traj, n_steps, 10.0,
                    0.0, float(cm1(12000.0)), n_E, seed)


def config_f6(seed: int = 0, n_traj: int = 16384, n_steps: int = 4000, n_E: int = 4000) -> Workload:
    """F = 6 (formaldehyde-sized): Morse + 50 cubic + 120 quartic couplings."""
    rng = np.random.default_rng(seed)
    pes = recipe_pes(6, rng, units=COUPLING_DIMENSIONLESS)
    p_eq, q_eq = _single_chi(pes.omega)
    lo, hi = grid_window(pes.omega)
    return Workload("f6_morse_cubic_quartic", pes, pes.omega.copy(), p_eq, q_eq, n_traj,
                    n_steps, 10.0, lo, hi, n_E, seed)


def config_f9(seed: int = 0, n_traj: int = 65536, n_steps: int = 5000, n_E: int = 4000) -> Workload:
    """F = 9 (methane-sized): Morse + 156 cubic + 486 quartic couplings."""
    rng = np.random.default_rng(seed)
    pes = recipe_pes(9, rng, units=COUPLING_DIMENSIONLESS)
    p_eq, q_eq = _single_chi(pes.omega)
    lo, hi = grid_window(pes.omega)
    return Workload("f9_morse_cubic_quartic", pes, pes.omega.copy(), p_eq, q_eq, n_traj,
                    n_steps, 10.0, lo, hi, n_E, seed)


def config_generic(F: int, seed: int, n_traj: int, n_steps: int, n_E: int = 4000,
                   quartic: bool = True) -> Workload:
    rng = np.random.default_rng(seed)
    pes = recipe_pes(F, rng, quartic=quartic, units=COUPLING_DIMENSIONLESS)
    p_eq, q_eq = _single_chi(pes.omega)
    lo, hi = grid_window(pes.omega)
    return Workload(f"f{F}_s{seed}", pes, pes.omega.copy(), p_eq, q_eq, n_traj, n_steps,
                    10.0, lo, hi, n_E, seed)


def uncoupled_morse(F: int, seed: int = 0, n_traj: int = 1024, n_steps: int = 3000,
                    n_E: int = 2000) -> Workload:
    """F uncoupled Morse oscillators (the paper's speed-up-versus-F comparison, Sec. IV)."""
    rng = np.random.default_rng(seed)
    omega = cm1(rng.uniform(1100.0, 3000.0, F))
    D = rng.uniform(0.15, 0.25, F)
    pes = morse_pes(omega, D)
    p_eq, q_eq = _single_chi(omega)
    lo, hi = grid_window(omega)
    return Workload(f"uncoupled_morse_f{F}", pes, omega.copy(), p_eq, q_eq, n_traj, n_steps,
                    10.0, lo, hi, n_E, seed)


def batch_molecules(n_mol: int = 48, seed: int = 0, Fs=(3, 6, 9, 12, 15, 24),
                    n_traj_lo: int = 512, n_traj_hi: int = 32768,
                    steps_lo: int = 2000, steps_hi: int = 8000, n_E: int = 4000) -> List[Workload]:
    """Mixed batch: F cycles over Fs, n_traj log-uniform, steps uniform; molecule m uses seed m."""
    rng = np.random.default_rng(seed)
    out = []
    for m in range(n_mol):
        F = Fs[m % len(Fs)]
        n_traj = int(np.exp(rng.uniform(np.log(n_traj_lo), np.log(n_traj_hi))))
        n_steps = int(rng.integers(steps_lo, steps_hi + 1))
        out.append(config_generic(F, seed + m, n_traj, n_steps, n_E).with_(name=f"mol{m}_f{F}"))
    return out


def standard_normals(seed: int, n_traj: int, F: int) -> np.ndarray:
    """Plain numpy standard normals [2F, n_traj] for tests that feed explicit samples."""
    return np.random.default_rng(seed).standard_normal((2 * F, n_traj))


def spectrum_peaks(E, I, rel=0.01):
    """Peak positions of a spectrum on a grid: local maxima of at least rel * max(I),
    each refined by the parabola through it and its two neighbours."""
    E = np.asarray(E, dtype=np.float64)
    I = np.asarray(I, dtype=np.float64)
    if I.size < 3 or not np.isfinite(I).all():
        return np.zeros(0)
    thr = rel * I.max()
    k = np.flatnonzero((I[1:-1] >= thr) & (I[1:-1] > I[:-2]) & (I[1:-1] >= I[2:])) + 1
    y0, y1, y2 = I[k - 1], I[k], I[k + 1]
    den = y0 - 2.0 * y1 + y2
    off = np.where(den != 0.0, 0.5 * (y0 - y2) / np.where(den != 0.0, den, 1.0), 0.0)
    return E[k] + off * (E[1] - E[0])


def peak_shift(ref, got):
    """Largest distance from a reference peak to the nearest peak of the other spectrum."""
    ref = np.asarray(ref)
    got = np.asarray(got)
    if ref.size == 0:
        return 0.0
    if got.size == 0:
        return float("inf")
    return float(np.max(np.min(np.abs(got[None, :] - ref[:, None]), axis=1)))
