"""The Cartesian-surface interface (Sec. III.A: the molecular surfaces are functions of
Cartesian coordinates; the host driver builds the mass-weighted normal modes from the
Hessian at the equilibrium geometry and converts between the two sets of coordinates).

Pins of the oracle's Cartesian surface and normal-mode analysis against what the
mathematics fixes: finite differences of the energy, invariance under rigid motions,
the normal-mode frequencies of a bent symmetric triatomic by Wilson's GF method (a
closed form that involves no diagonalisation of the 9 x 9 Hessian), mass-orthonormality
of the mode matrix and its orthogonality to translations and rotations.  The library's
own (host) normal-mode routine is then held to the pinned oracle."""
import numpy as np
import pytest

import oracle
from paper_1312_4698_gb300 import workloads as wl


def _asym():
    """An unsymmetric variant (different bonds, masses): no closed form, the invariances hold."""
    c = wl.water_like_triatomic()
    return wl.CartTriatomic(mass=np.array([1.00782503223, 15.99491461957, 2.01410177812]) * wl.AMU,
                            D=np.array([0.2, 0.18]), a=np.array([1.1, 1.25]), re=np.array([1.81, 1.86]),
                            k_bend=0.16, theta_e=c.theta_e)


def _rot(rng):
    A = rng.normal(size=(3, 3))
    Q, R = np.linalg.qr(A)
    Q = Q * np.sign(np.diag(R))
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    return Q


@pytest.mark.parametrize("which", ["symmetric", "asymmetric"])
def test_cartesian_derivatives_match_finite_differences(which):
    c = wl.water_like_triatomic() if which == "symmetric" else _asym()
    _, x_eq, _, _ = oracle.normal_modes(c)
    rng = np.random.default_rng(1)
    h = 1e-5
    for _ in range(4):
        x = x_eq + rng.normal(scale=0.15, size=9)
        V, g, H = oracle.cart_eval(c, x)
        gfd = np.array([(oracle.cart_eval(c, x + h * e)[0] - oracle.cart_eval(c, x - h * e)[0]) / (2 * h)
                        for e in np.eye(9)])
        Hfd = np.array([(oracle.cart_eval(c, x + h * e)[1] - oracle.cart_eval(c, x - h * e)[1]) / (2 * h)
                        for e in np.eye(9)])
        assert np.max(np.abs(g - gfd)) < 1e-8 * max(1.0, np.max(np.abs(g)))
        assert np.max(np.abs(H - Hfd)) < 1e-7 * max(1.0, np.max(np.abs(H)))
        assert np.allclose(H, H.T, atol=1e-14)


def test_surface_is_invariant_under_rigid_motions():
    c = _asym()
    _, x_eq, _, _ = oracle.normal_modes(c)
    rng = np.random.default_rng(2)
    x = x_eq + rng.normal(scale=0.2, size=9)
    V, g, H = oracle.cart_eval(c, x)
    for _ in range(3):
        R, t = _rot(rng), rng.normal(size=3)
        y = (x.reshape(3, 3) @ R.T + t).ravel()
        V2, g2, H2 = oracle.cart_eval(c, y)
        Rb = np.kron(np.eye(3), R)
        assert abs(V2 - V) < 1e-14 * max(1.0, abs(V)) + 1e-16
        assert np.allclose(g2, Rb @ g, atol=1e-12)
        assert np.allclose(H2, Rb @ H @ Rb.T, atol=1e-11)
    # no net force or torque on the molecule
    f = g.reshape(3, 3)
    assert np.allclose(f.sum(axis=0), 0.0, atol=1e-13)
    assert np.allclose(np.cross(x.reshape(3, 3), f).sum(axis=0), 0.0, atol=1e-12)


def test_normal_mode_frequencies_match_the_wilson_gf_closed_form():
    """Bent symmetric XY2 with a valence force field (no off-diagonal force constants):
    internal coordinates r1, r2, alpha; f_r = 2 D a^2 (Morse curvature), f_alpha =
    k sin^2(theta_e) (the bend's curvature in alpha); G elements from the atomic masses,
    mu = 1/m (Wilson, Decius and Cross): A1 block of (S1 = (r1 + r2)/sqrt 2, alpha) and the
    B2 antisymmetric stretch, omega^2 the eigenvalues of F G."""
    c = wl.water_like_triatomic()
    om, _, _, rigid = oracle.normal_modes(c)
    muY, muX = 1.0 / c.mass[0], 1.0 / c.mass[1]
    al, r = c.theta_e, c.re[0]
    fr, fa = 2.0 * c.D[0] * c.a[0] ** 2, c.k_bend * np.sin(al) ** 2
    G11 = muY + muX * (1.0 + np.cos(al))
    G12 = -np.sqrt(2.0) * muX * np.sin(al) / r
    G22 = 2.0 / r ** 2 * (muY + muX * (1.0 - np.cos(al)))
    G33 = muY + muX * (1.0 - np.cos(al))
    lam = np.sort(np.linalg.eigvals(np.diag([fr, fa]) @ np.array([[G11, G12], [G12, G22]])).real)
    ref = np.sort(np.sqrt(np.r_[lam, fr * G33]))
    print("normal modes (cm^-1):", wl.to_cm1(om), "GF:", wl.to_cm1(ref))
    assert np.max(np.abs(om - ref)) < 1e-12 * ref.max()
    assert rigid < 1e-12 * om.max() ** 2


@pytest.mark.parametrize("which", ["symmetric", "asymmetric"])
def test_mode_matrix_is_mass_orthonormal_and_free_of_rigid_motions(which):
    c = wl.water_like_triatomic() if which == "symmetric" else _asym()
    om, x_eq, Lm, _ = oracle.normal_modes(c)
    m = np.repeat(c.mass, 3)
    assert np.allclose(Lm.T @ (m[:, None] * Lm), np.eye(3), atol=1e-12)
    X = x_eq.reshape(3, 3)
    rigid = []
    for d in range(3):
        t = np.zeros((3, 3)); t[:, d] = 1.0
        rigid.append(t.ravel())
        e = np.zeros(3); e[d] = 1.0
        rigid.append(np.cross(e, X).ravel())
    for v in rigid:
        assert np.allclose(Lm.T @ (m * v), 0.0, atol=1e-10 * np.linalg.norm(v))
    # increasing frequencies; the mode sign convention
    assert np.all(np.diff(om) > 0)
    for k in range(3):
        col = Lm[:, k] * np.sqrt(m)
        assert col[np.flatnonzero(np.abs(col) > 1e-3)[0]] > 0


def test_normal_mode_surface_is_harmonic_at_the_minimum():
    c = _asym()
    om, _, _, _ = oracle.normal_modes(c)
    pes = wl.CartPes(c)
    V, g, H = oracle.pes_eval(pes, np.zeros(3))
    assert abs(V) < 1e-15
    assert np.max(np.abs(g)) < 1e-13
    assert np.allclose(H, np.diag(om ** 2), atol=1e-12 * om.max() ** 2)
    # V(q) is the Cartesian surface at x_eq + Lm q
    _, x_eq, Lm, _ = oracle.normal_modes(c)
    q = np.array([0.3, -0.2, 0.1]) / np.sqrt(om)
    V1, g1, H1 = oracle.pes_eval(pes, q)
    Vx, gx, Hx = oracle.cart_eval(c, x_eq + Lm @ q)
    assert abs(V1 - Vx) < 1e-15 and np.allclose(g1, Lm.T @ gx, atol=1e-15) and np.allclose(H1, Lm.T @ Hx @ Lm, atol=1e-15)


def test_propagation_on_the_cartesian_surface_is_symplectic_and_conserves_energy():
    c = wl.water_like_triatomic()
    om, _, _, _ = oracle.normal_modes(c)
    pes = wl.CartPes(c)
    p_eq, q_eq = wl.ground_chi(om)
    p0, q0, _ = oracle.sample_initial(om, p_eq, q_eq, 3, 7)
    for j in range(3):
        r = oracle.propagate_one(pes, om, p_eq, q_eq, 10.0, 2000, p0[:, j], q0[:, j])
        M = r["M"]
        Jm = np.block([[np.zeros((3, 3)), -np.eye(3)], [np.eye(3), np.zeros((3, 3))]])
        assert np.max(np.abs(M.T @ Jm @ M - Jm)) < 1e-10 * max(1.0, np.max(np.abs(M)) ** 2)
        # energy error bounded and fourth order: largest deviation at four times along the run,
        # with dt and with dt / 2 (measured ratio ~16)
        E0 = 0.5 * p0[:, j] @ p0[:, j] + oracle.pes_eval(pes, q0[:, j])[0]
        err = []
        for dt, f in ((10.0, 1), (5.0, 2)):
            e = 0.0
            for n in (500, 1000, 1500, 2000):
                rr = oracle.propagate_one(pes, om, p_eq, q_eq, dt, n * f, p0[:, j], q0[:, j])
                e = max(e, abs(0.5 * rr["p"] @ rr["p"] + oracle.pes_eval(pes, rr["q"])[0] - E0))
            err.append(e)
        print(f"trajectory {j}: max |dE|/E {err[0] / E0:.2e} (dt 10), {err[1] / E0:.2e} (dt 5)")
        assert err[0] < 1e-4 * E0
        assert err[0] / err[1] > 10.0


def test_library_normal_modes_match_the_oracle():
    """The library's host routine (its own Hessian formulas and Jacobi variant) against
    the pinned oracle, and the coordinate conversions as inverses on the vibrations."""
    from paper_1312_4698_gb300 import scivr
    for c in (wl.water_like_triatomic(), _asym()):
        om, xe, Lm = scivr.scivr_normal_modes(c)
        om2, xe2, Lm2, _ = oracle.normal_modes(c)
        assert np.max(np.abs(om - om2)) < 1e-12 * om2.max()
        assert np.max(np.abs(xe - xe2)) < 1e-14
        assert np.max(np.abs(Lm - Lm2)) < 1e-10 * np.abs(Lm2).max()
        q = np.random.default_rng(3).normal(size=(7, 3)) * 0.2
        x = scivr.scivr_normal_to_cartesian(c, q)
        assert np.allclose(x, xe2 + q @ Lm2.T, atol=1e-13)
        assert np.allclose(scivr.scivr_cartesian_to_normal(c, x), q, atol=1e-12)
