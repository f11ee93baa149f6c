"""Pins of the oracle's learned-residual potential (MLP) and its training gradient.

The network's gradient and Hessian are checked against finite differences
of its value, the training objective's parameter gradient against finite
differences of the objective, a degenerate network against its closed form,
and a propagation under an MLP-augmented potential against the symplectic
and energy invariants."""
import numpy as np
import pytest

import oracle
from paper_1312_4698_gb300 import workloads as wl


def _mlp(F=4, H=24, seed=2):
    om = wl.cm1(np.linspace(1200, 3000, F))
    return wl.init_mlp(F, H, seed, s_in=np.sqrt(om), s_out=3e-4)


def test_mlp_gradient_and_hessian_vs_finite_differences():
    m = _mlp()
    F = 4
    rng = np.random.default_rng(0)
    for _ in range(3):
        q = rng.normal(0, 6, F)
        V, g, H = oracle.mlp_eval(m, q)
        h = 1e-3
        gf = np.zeros(F)
        Hf = np.zeros((F, F))
        for i in range(F):
            e = np.zeros(F); e[i] = h
            vals = [oracle.mlp_eval(m, q + k * e) for k in (2, 1, -1, -2)]
            gf[i] = (-vals[0][0] + 8 * vals[1][0] - 8 * vals[2][0] + vals[3][0]) / (12 * h)
            Hf[:, i] = (-vals[0][1] + 8 * vals[1][1] - 8 * vals[2][1] + vals[3][1]) / (12 * h)
        assert np.allclose(g, gf, rtol=1e-7, atol=1e-12 * np.max(np.abs(g)))
        assert np.allclose(H, Hf, rtol=1e-6, atol=1e-9 * np.max(np.abs(H)))
        assert np.allclose(H, H.T, rtol=0, atol=1e-15 * np.max(np.abs(H)))


def test_degenerate_network_closed_form():
    m = _mlp()
    m.W1[:] = 0.0
    m.W2[:] = 0.0
    m.W3[:] = 0.0
    m.b3[:] = np.linspace(-1, 1, m.H)
    m.b4 = 0.25
    V, g, H = oracle.mlp_eval(m, np.array([1.0, 2.0, 3.0, 4.0]))
    silu = m.b3 / (1 + np.exp(-m.b3))
    assert V == pytest.approx(m.s_out * (m.w4 @ silu + 0.25), rel=1e-14)
    assert np.all(g == 0.0) and np.all(H == 0.0)


def test_training_gradient_vs_finite_differences():
    F, Hd = 3, 8
    m = _mlp(F, Hd, seed=5)
    rng = np.random.default_rng(1)
    q = rng.normal(0, 5, (6, F))
    Vref = rng.normal(0, 1e-3, 6)
    gref = rng.normal(0, 1e-4, (6, F))
    alpha, beta = 1e6, 1e8
    L, grad = oracle.mlp_loss_grad(m, q, Vref, gref, alpha, beta)
    v = m.flat()
    idx = rng.choice(v.size, 40, replace=False)
    for k in idx:
        h = 1e-6 * max(1.0, abs(v[k]))
        vp = v.copy(); vp[k] += h
        vm = v.copy(); vm[k] -= h
        Lp, _ = oracle.mlp_loss_grad(m.with_flat(vp), q, Vref, gref, alpha, beta)
        Lm, _ = oracle.mlp_loss_grad(m.with_flat(vm), q, Vref, gref, alpha, beta)
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - grad[k]) <= 1e-6 * max(abs(grad).max(), 1e-30) + 1e-7 * abs(fd), (k, fd, grad[k])


def test_propagation_invariants_with_learned_residual():
    F = 3
    w8 = wl.config_f3(n_traj=4, n_steps=1500)
    pes = w8.pes
    pes.mlp = wl.init_mlp(F, 32, seed=3, s_in=np.sqrt(w8.gamma), s_out=2e-4)
    p0, q0, _ = oracle.sample_initial(w8.gamma, w8.p_eq, w8.q_eq, 2, 0)
    r = oracle.propagate_one(pes, w8.gamma, w8.p_eq, w8.q_eq, 10.0, 1500, p0[:, 0], q0[:, 0])
    M = r["M"]
    Z, I = np.zeros((F, F)), np.eye(F)
    J = np.block([[Z, -I], [I, Z]])
    assert np.max(np.abs(M.T @ J @ M - J)) / max(1.0, np.max(np.abs(M)) ** 2) < 1e-10
    # energy error of a fourth-order integrator: halving dt divides it by ~16 (a gradient
    # inconsistent with V would leave an O(1) drift instead)
    E0 = 0.5 * np.sum(p0[:, 0] ** 2) + oracle.pes_eval(pes, q0[:, 0])[0]
    errs = []
    for dt in (10.0, 5.0):
        rr = oracle.propagate_one(pes, w8.gamma, w8.p_eq, w8.q_eq, dt, int(3000 / dt), p0[:, 0], q0[:, 0])
        errs.append(abs(0.5 * np.sum(rr["p"] ** 2) + oracle.pes_eval(pes, rr["q"])[0] - E0))
    assert errs[0] / errs[1] > 10.0, errs
    # the residual really is part of the surface
    V_full = oracle.pes_eval(pes, q0[:, 0])[0]
    pes_plain = wl.config_f3().pes
    V_plain = oracle.pes_eval(pes_plain, q0[:, 0])[0]
    V_m = oracle.mlp_eval(pes.mlp, q0[:, 0])[0]
    assert V_full == pytest.approx(V_plain + V_m, rel=1e-13)
