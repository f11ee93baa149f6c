"""Pins of the oracle's potential, determinants and coherent-state overlap.

Nothing here retypes the oracle's formulas: derivatives are checked by
finite differences and Euler's theorem, the Morse diagonal by its closed-form
limits, determinants by LAPACK, and the overlap by numerical quadrature of
the coherent-state wavefunctions of Eq. coherent_state.
"""
import numpy as np
import pytest

import oracle
from paper_1312_4698_gb300 import workloads as wl


def _rand_pes(F, seed=3):
    return wl.recipe_pes(F, np.random.default_rng(seed))


@pytest.mark.parametrize("F", [1, 2, 3, 6, 9])
def test_gradient_and_hessian_match_finite_differences(F):
    pes = _rand_pes(F)
    rng = np.random.default_rng(F)
    for _ in range(3):
        q = rng.normal(0.0, 8.0, F)
        V, g, H = oracle.pes_eval(pes, q)
        h = 1e-3
        g_fd = np.zeros(F)
        H_fd = np.zeros((F, F))
        for i in range(F):
            e = np.zeros(F); e[i] = h
            # 4th-order central differences
            Vp2, gp2, _ = oracle.pes_eval(pes, q + 2 * e)
            Vp1, gp1, _ = oracle.pes_eval(pes, q + e)
            Vm1, gm1, _ = oracle.pes_eval(pes, q - e)
            Vm2, gm2, _ = oracle.pes_eval(pes, q - 2 * e)
            g_fd[i] = (-Vp2 + 8 * Vp1 - 8 * Vm1 + Vm2) / (12 * h)
            H_fd[:, i] = (-gp2 + 8 * gp1 - 8 * gm1 + gm2) / (12 * h)
        assert np.allclose(g, g_fd, rtol=1e-8, atol=1e-12 * max(1.0, abs(V)))
        assert np.allclose(H, H_fd, rtol=1e-7, atol=1e-12)
        assert np.allclose(H, H.T, rtol=0, atol=1e-18)


def test_euler_homogeneity_of_couplings():
    """q . grad V_n = n V_n for the homogeneous cubic (n=3) and quartic (n=4) parts."""
    F = 5
    rng = np.random.default_rng(11)
    zero = np.zeros(F)
    for deg in (3, 4):
        idx = wl.offdiag_monomials(F, deg)
        c = rng.normal(0.0, 1e-3, idx.shape[0])
        kw = dict(idx3=idx, c3=c) if deg == 3 else dict(idx4=idx, c4=c)
        pes = wl.PesDesc(F, wl.DIAG_HARMONIC, zero, zero, zero,
                         kw.get("idx3", np.zeros((0, 3))), kw.get("c3", np.zeros(0)),
                         kw.get("idx4", np.zeros((0, 4))), kw.get("c4", np.zeros(0)))
        q = rng.normal(0.0, 2.0, F)
        V, g, H = oracle.pes_eval(pes, q)
        assert abs(q @ g - deg * V) <= 1e-12 * max(1.0, abs(V))
        # the Hessian of a degree-n form satisfies H q = (n - 1) grad V
        assert np.allclose(H @ q, (deg - 1) * g, rtol=1e-12, atol=1e-15)


def test_single_monomials():
    F = 4
    zero = np.zeros(F)
    q = np.array([0.3, -1.7, 2.2, 0.9])
    pes = wl.PesDesc(F, wl.DIAG_HARMONIC, zero, zero, zero, np.array([[0, 1, 3]]),
                     np.array([2.5]), np.array([[1, 1, 2, 2]]), np.array([-0.5]))
    V, g, H = oracle.pes_eval(pes, q)
    assert V == pytest.approx(2.5 * q[0] * q[1] * q[3] - 0.5 * q[1] ** 2 * q[2] ** 2, rel=1e-15)
    # d/dq1 of (-0.5 q1^2 q2^2) = -q1 q2^2
    assert g[1] == pytest.approx(2.5 * q[0] * q[3] - q[1] * q[2] ** 2, rel=1e-14)
    # d2/dq1 dq2 of (-0.5 q1^2 q2^2) = -2 q1 q2
    assert H[1, 2] == pytest.approx(-2.0 * q[1] * q[2], rel=1e-14)


def test_morse_diagonal_limits():
    omega = wl.cm1([1600.0, 3650.0])
    pes = wl.morse_pes(omega, [0.2, 0.15])
    V0, g0, H0 = oracle.pes_eval(pes, np.zeros(2))
    assert V0 == 0.0 and np.all(g0 == 0.0)
    assert np.allclose(np.diag(H0), omega ** 2, rtol=1e-14)      # V'' (0) = 2 D a^2 = omega^2
    Vinf, _, _ = oracle.pes_eval(pes, np.array([1e5, 1e5]))
    assert Vinf == pytest.approx(0.35, rel=1e-14)                  # dissociation limit sum D
    # minimum at q = 0 along each axis
    for x in (-0.5, 0.5):
        assert oracle.pes_eval(pes, np.array([x, 0.0]))[0] > 0.0


def test_harmonic_diagonal():
    omega = np.array([0.01, 0.02, 0.03])
    pes = wl.harmonic_pes(omega)
    q = np.array([1.0, -2.0, 0.5])
    V, g, H = oracle.pes_eval(pes, q)
    assert V == pytest.approx(0.5 * np.sum(omega ** 2 * q ** 2), rel=1e-15)
    assert np.allclose(H, np.diag(omega ** 2), rtol=1e-15)


@pytest.mark.parametrize("n", [1, 2, 5, 12, 18])
def test_real_determinant_vs_lapack(n):
    rng = np.random.default_rng(n)
    A = rng.normal(size=(n, n))
    assert oracle.det_real(A) == pytest.approx(np.linalg.det(A), rel=1e-11)


@pytest.mark.parametrize("n", [1, 3, 6, 9, 24])
def test_complex_determinant_vs_lapack(n):
    rng = np.random.default_rng(100 + n)
    A = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    d = oracle.det_complex(A)
    ref = np.linalg.det(A)
    assert abs(d - ref) <= 1e-11 * abs(ref)


def test_singular_determinants_are_zero():
    A = np.ones((3, 3))
    assert oracle.det_real(A) == 0.0
    assert oracle.det_complex(A.astype(complex)) == 0.0


@pytest.mark.parametrize("gamma,p1,q1,p2,q2", [
    (0.0073, 0.085, 0.0, 0.12, 3.0),
    (0.017, -0.2, 1.5, 0.05, -4.0),
    (1.0, 0.3, 0.2, 0.1, 0.5),
])
def test_overlap_vs_quadrature(gamma, p1, q1, p2, q2):
    """<p1 q1|p2 q2> from the wavefunctions of Eq. coherent_state by quadrature."""
    s = 1.0 / np.sqrt(gamma)
    x = np.linspace(min(q1, q2) - 14 * s, max(q1, q2) + 14 * s, 200001)

    def psi(p, q):
        return (gamma / np.pi) ** 0.25 * np.exp(-0.5 * gamma * (x - q) ** 2 + 1j * p * (x - q))

    ref = np.trapezoid(np.conj(psi(p1, q1)) * psi(p2, q2), x)
    got = np.exp(oracle.log_overlap([gamma], [p1], [q1], [p2], [q2]))
    assert abs(got - ref) <= 1e-12
    # normalisation |<pq|pq>| = 1
    assert abs(np.exp(oracle.log_overlap([gamma], [p1], [q1], [p1], [q1])) - 1.0) == 0.0


def test_overlap_is_product_over_modes():
    g = np.array([0.01, 0.02])
    p1, q1, p2, q2 = np.array([0.1, 0.2]), np.array([1.0, -1.0]), np.array([0.0, 0.3]), np.array([2.0, 0.5])
    lo = oracle.log_overlap(g, p1, q1, p2, q2)
    lo0 = oracle.log_overlap(g[:1], p1[:1], q1[:1], p2[:1], q2[:1])
    lo1 = oracle.log_overlap(g[1:], p1[1:], q1[1:], p2[1:], q2[1:])
    assert abs(lo - (lo0 + lo1)) < 1e-15
