"""Learned residual on the GPU against the FP64 oracle: batched value, gradient
and Hessian, the training objective and its parameter gradient, AdamW, and the
analytic FP64 evaluation used to make training targets.

Error model of the tensor-core path.  Every GEMM operand is rounded to BF16
(unit roundoff u = 2^-8); each of the three 256-wide contractions contributes a
relative error of order u to its outputs, so values, gradients and Hessians
carry ~3u ~ 1e-2 of their max norm at worst.  Bound: 2.5e-2 of the max norm
for V, grad V and the Hessian.  The parameter gradient's longest path rounds
about five times (the tangent rows through two layers, the reverse rows back,
and the weight-gradient GEMM operands), ~5u ~ 2e-2 in norm.  With random
targets the per-point terms of each sum partly cancel while the rounding of
the shared BF16 weights does not, which lifts the relative error of the sum
(measured 1.4e-2 to 4.3e-2 for n = 50..301): bound 6e-2 of each block's 2-norm
and a cosine of at least 0.998 with the oracle's block.
"""
import numpy as np
import pytest

import oracle
from paper_1312_4698_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL_EVAL = 2.5e-2
TOL_GRAD = 6e-2


@pytest.fixture(scope="module")
def G():
    import torch
    from paper_1312_4698_gb300 import scivr
    assert torch.cuda.is_available()
    return scivr


def _t(x, dtype=None):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), device="cuda", dtype=dtype)


def _pes_with_mlp(F, seed=1, s_out=3e-4):
    w8 = {3: wl.config_f3, 6: wl.config_f6, 9: wl.config_f9}.get(F)
    if w8 is not None:
        pes = w8().pes
    else:
        rng = np.random.default_rng(F)
        pes = wl.recipe_pes(F, rng, units=wl.COUPLING_DIMENSIONLESS)
    m = wl.init_mlp(F, 256, seed, s_in=np.sqrt(pes.omega), s_out=s_out)
    rng = np.random.default_rng(seed + 100)
    m.b1 = rng.normal(0, 0.3, 256)
    m.b2 = rng.normal(0, 0.3, 256)
    m.b3 = rng.normal(0, 0.3, 256)
    m.b4 = 0.1
    return pes, m


def _points(pes, n, seed):
    """Points spread like sampled trajectories: q_i ~ N(0, 2 / omega_i)."""
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, 1.0, (n, pes.F)) * np.sqrt(2.0 / pes.omega)


@pytest.mark.parametrize("F", [1, 3, 6, 9])
@pytest.mark.parametrize("n", [1, 37, 1000])
def test_mlp_value_gradient_hessian_vs_oracle(G, F, n):
    import torch
    pes, m = _pes_with_mlp(F)
    P = G.scivr_create_pes(pes)
    G.scivr_pes_set_mlp(P, m)
    q = _points(pes, n, 7 * F + n)
    qd = _t(q, torch.float32)
    V = torch.zeros(n, device="cuda")
    g = torch.zeros(n, F, device="cuda")
    H = torch.zeros(n, F, F, device="cuda")
    G.scivr_mlp_eval(P, n, qd, V, g, H)
    assert G.scivr_check_status() == G.SCIVR_OK
    Vg, gg, Hg = V.cpu().double().numpy(), g.cpu().double().numpy(), H.cpu().double().numpy()
    ref = [oracle.mlp_eval(m, q[j]) for j in range(n)]
    Vr = np.array([r[0] for r in ref])
    gr = np.array([r[1] for r in ref])
    Hr = np.array([r[2] for r in ref])
    eV = np.max(np.abs(Vg - Vr)) / np.max(np.abs(Vr))
    eg = np.max(np.abs(gg - gr)) / np.max(np.abs(gr))
    eH = np.max(np.abs(Hg - Hr)) / np.max(np.abs(Hr))
    print(f"F={F} n={n}: rel err V {eV:.2e} g {eg:.2e} H {eH:.2e}")
    assert eV <= TOL_EVAL and eg <= TOL_EVAL and eH <= TOL_EVAL
    assert np.array_equal(Hg, np.transpose(Hg, (0, 2, 1)))
    # without the Hessian the value and gradient are unchanged (same reverse pass)
    V2 = torch.zeros(n, device="cuda")
    g2 = torch.zeros(n, F, device="cuda")
    G.scivr_mlp_eval(P, n, qd, V2, g2, None)
    assert G.scivr_check_status() == G.SCIVR_OK
    assert np.max(np.abs(V2.cpu().double().numpy() - Vr)) <= TOL_EVAL * np.max(np.abs(Vr))
    assert np.max(np.abs(g2.cpu().double().numpy() - gr)) <= TOL_EVAL * np.max(np.abs(gr))


def _blocks(F):
    sizes = wl.MlpParams.sizes(F, 256)
    names = ["W1", "b1", "W2", "b2", "W3", "b3", "w4", "b4"]
    o = np.cumsum([0] + sizes)
    return [(names[i], o[i], o[i + 1]) for i in range(len(names))]


@pytest.mark.parametrize("F,n", [(3, 50), (3, 301), (9, 130)])
def test_training_gradient_vs_oracle(G, F, n):
    import torch
    pes, m = _pes_with_mlp(F, seed=4)
    P = G.scivr_create_pes(pes)
    G.scivr_pes_set_mlp(P, m)
    q = _points(pes, n, 11)
    rng = np.random.default_rng(12)
    ref = [oracle.mlp_eval(m, q[j]) for j in range(n)]
    Vm = np.array([r[0] for r in ref])
    gm = np.array([r[1] for r in ref])
    Vref = Vm + rng.normal(0, 1, n) * np.std(Vm)
    gref = gm + rng.normal(0, 1, gm.shape) * np.std(gm)
    alpha, beta = 1.0 / np.var(Vm), 1.0 / np.var(gm)
    L, gr = oracle.mlp_loss_grad(m, q, Vref, gref, alpha, beta)
    npar = G.scivr_mlp_param_count(F)
    assert npar == gr.size
    grad = torch.zeros(npar, device="cuda")
    loss = torch.zeros(1, device="cuda")
    G.scivr_mlp_loss_grad(P, n, _t(q, torch.float32), _t(Vref, torch.float32), _t(gref, torch.float32),
                          alpha, beta, grad, loss)
    assert G.scivr_check_status() == G.SCIVR_OK
    gg = grad.cpu().double().numpy()
    Lg = float(loss.item())
    print(f"F={F} n={n}: loss {Lg:.6e} vs {L:.6e}")
    assert abs(Lg - L) <= 2e-2 * L
    for name, a, b in _blocks(F):
        err = np.linalg.norm(gg[a:b] - gr[a:b]) / max(np.linalg.norm(gr[a:b]), 1e-300)
        cos = gg[a:b] @ gr[a:b] / (np.linalg.norm(gg[a:b]) * np.linalg.norm(gr[a:b]) + 1e-300)
        print(f"  {name}: rel err (2-norm) {err:.2e}, cos {cos:.6f}")
        if name == "b4":
            # dL/db4 = s_out (2 alpha / n) sum_j (V_j - Vref_j): a cancelling sum, so bound its
            # absolute error by the value error instead: 2 alpha s_out max_j |dV_j|
            assert abs(gg[a] - gr[a]) <= 2 * alpha * m.s_out * TOL_EVAL * np.max(np.abs(Vm))
            continue
        assert err <= TOL_GRAD, name
        assert cos >= 0.998, name


def test_params_roundtrip_and_adamw_step(G):
    import torch
    F = 3
    pes, m = _pes_with_mlp(F)
    P = G.scivr_create_pes(pes)
    G.scivr_pes_set_mlp(P, m)
    npar = G.scivr_mlp_param_count(F)
    th = torch.zeros(npar, device="cuda")
    G.scivr_mlp_get_params(P, th)
    torch.cuda.synchronize()
    th0 = th.cpu().double().numpy()
    assert np.allclose(th0, m.flat(), rtol=1e-7, atol=0)     # FP32 copies of the FP64 weights
    rng = np.random.default_rng(3)
    grads = [rng.normal(0, 1e-3, npar) for _ in range(3)]
    m1 = torch.zeros(npar, device="cuda")
    m2 = torch.zeros(npar, device="cuda")
    lr, b1, b2, eps, wd = 1e-3, 0.9, 0.999, 1e-8, 1e-2
    x = th0.copy()
    a = np.zeros(npar)
    v = np.zeros(npar)
    for t, gr in enumerate(grads, start=1):
        G.scivr_mlp_adamw(P, _t(gr, torch.float32), m1, m2, t, lr, b1, b2, eps, wd)
        # AdamW with decoupled weight decay, written out
        a = b1 * a + (1 - b1) * gr
        v = b2 * v + (1 - b2) * gr * gr
        x = x - lr * ((a / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps) + wd * x)
    G.scivr_mlp_get_params(P, th)
    assert G.scivr_check_status() == G.SCIVR_OK
    got = th.cpu().double().numpy()
    assert np.max(np.abs(got - x)) <= 1e-5 * np.max(np.abs(x))
    # set_params refreshes the tiles: evaluation with the new weights matches the oracle
    mm = m.with_flat(got)
    q = _points(pes, 20, 5)
    V = torch.zeros(20, device="cuda")
    g = torch.zeros(20, F, device="cuda")
    G.scivr_mlp_eval(P, 20, _t(q, torch.float32), V, g, None)
    torch.cuda.synchronize()
    Vr = np.array([oracle.mlp_eval(mm, q[j])[0] for j in range(20)])
    assert np.max(np.abs(V.cpu().double().numpy() - Vr)) <= TOL_EVAL * np.max(np.abs(Vr))


@pytest.mark.parametrize("F", [3, 6, 9])
def test_analytic_eval_terms_vs_oracle(G, F):
    import torch
    pes = {3: wl.config_f3, 6: wl.config_f6, 9: wl.config_f9}[F]().pes
    P = G.scivr_create_pes(pes)
    n = 200
    q = _points(pes, n, F)
    qd = _t(q)
    diag = wl.PesDesc(F, pes.diag_kind, pes.omega, pes.D, pes.a, np.zeros((0, 3)), np.zeros(0),
                      np.zeros((0, 4)), np.zeros(0))
    for terms in (G.SCIVR_TERMS_ALL, G.SCIVR_TERMS_DIAG, G.SCIVR_TERMS_COUPLING):
        V = torch.zeros(n, dtype=torch.float64, device="cuda")
        g = torch.zeros(n, F, dtype=torch.float64, device="cuda")
        H = torch.zeros(n, F, F, dtype=torch.float64, device="cuda")
        G.scivr_pes_eval(P, n, qd, terms, V, g, H)
        assert G.scivr_check_status() == G.SCIVR_OK
        Vg, gg, Hg = V.cpu().numpy(), g.cpu().numpy(), H.cpu().numpy()
        for j in range(0, n, 17):
            full = oracle.pes_eval(pes, q[j])
            dg = oracle.pes_eval(diag, q[j])
            want = {G.SCIVR_TERMS_ALL: full, G.SCIVR_TERMS_DIAG: dg,
                    G.SCIVR_TERMS_COUPLING: tuple(a - b for a, b in zip(full, dg))}[terms]
            sc = max(abs(full[0]), 1e-30)
            assert abs(Vg[j] - want[0]) <= 1e-12 * sc
            assert np.max(np.abs(gg[j] - want[1])) <= 1e-12 * max(np.max(np.abs(full[1])), 1e-30)
            assert np.max(np.abs(Hg[j] - want[2])) <= 1e-12 * max(np.max(np.abs(full[2])), 1e-30)


def _diag_only(pes):
    return wl.PesDesc(pes.F, pes.diag_kind, pes.omega, pes.D, pes.a, np.zeros((0, 3)), np.zeros(0),
                      np.zeros((0, 4)), np.zeros(0))


def test_surrogate_propagation_vs_oracle(G):
    """Morse diagonal + a random network residual: amplitudes, final state and
    flags of the split-step surrogate path against the FP64 oracle on the same
    surface.  The network's force error (BF16 operands, ~3u of its magnitude)
    perturbs the action by about T 3u max|V_mlp| and the positions by about
    T^2/2 3u max|grad V_mlp|; the bounds below are those estimates with a
    factor 3 of margin, and the printed errors sit well inside them."""
    from tests.test_gpu_parity import gpu_propagate, MIXED_STAB_TOL, amp_err
    F, n = 3, 64
    w8 = wl.config_f3(n_traj=n, n_steps=300)
    pes = _diag_only(w8.pes)
    m = wl.init_mlp(F, 256, 3, s_in=np.sqrt(w8.gamma), s_out=2e-4)
    rng = np.random.default_rng(9)
    m.b1 = rng.normal(0, 0.3, 256)
    m.b2 = rng.normal(0, 0.3, 256)
    pes.mlp = m
    w8.pes = pes
    p0, q0, w = oracle.sample_initial(w8.gamma, w8.p_eq[0], w8.q_eq[0], n, 0)
    ra, rg, rf = oracle.propagate(pes, w8.gamma, w8.p_eq, w8.q_eq, w8.dt, w8.n_steps, p0, q0, final=True)
    go = gpu_propagate(G, w8, p0, q0, precision=G.SCIVR_MIXED, fin=True, stab_tol=MIXED_STAB_TOL)
    assert G.scivr_check_status() == G.SCIVR_OK
    assert rg.all() and go["good"].all()
    T = w8.n_steps * w8.dt
    ev = [oracle.mlp_eval(m, q0[:, j]) for j in range(n)]
    vmax = max(abs(e[0]) for e in ev)
    gmax = max(np.max(np.abs(e[1])) for e in ev)
    e_amp = amp_err(go["amp"], ra, rg)
    e_q = np.max(np.abs(go["q"].T - rf["q"]))
    e_p = np.max(np.abs(go["p"].T - rf["p"]))
    e_S = np.max(np.abs(go["S"] - rf["S"]))
    print(f"amp {e_amp:.2e} q {e_q:.2e} p {e_p:.2e} S {e_S:.2e}; vmax {vmax:.2e} gmax {gmax:.2e}")
    tol_S = 3 * T * 3 * 2 ** -8 * vmax
    assert e_S <= tol_S
    assert e_amp <= 3 * tol_S + 1e-6
    assert e_q <= 3 * 0.5 * T ** 2 * 3 * 2 ** -8 * gmax + 1e-9
    assert e_p <= 3 * T * 3 * 2 ** -8 * gmax + 1e-9
