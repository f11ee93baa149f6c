"""Learned-residual workflow on the GPU (include/scivr_mlp.h).

The network learns the coupling part of an analytic surface (V minus its
separable Morse/harmonic diagonal) from points visited by trajectories of that
surface; afterwards a potential made of the diagonal plus the network is
propagated with one batched tensor-core evaluation per force stage.  Every
numerical step runs in libscivr's kernels; this module only orders the calls
and moves tensors.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import scivr as G
from . import workloads as wl


def diagonal_part(pes: wl.PesDesc) -> wl.PesDesc:
    """The separable diagonal of a surface (its couplings removed)."""
    return wl.PesDesc(pes.F, pes.diag_kind, pes.omega, pes.D, pes.a, np.zeros((0, 3)), np.zeros(0),
                      np.zeros((0, 4)), np.zeros(0))


def trajectory_points(pes: G.Pes, w8: wl.Workload, n_traj: int, n_seg: int, seg_steps: int, seed: int = 1,
                      precision: int = G.SCIVR_FP64, q_max: float = 6.0):
    """Points q [<= n_traj * n_seg, F] (float64, device) visited by n_traj
    Husimi-sampled trajectories of the analytic surface, taken every seg_steps
    steps (each segment restarts from the previous segment's final p, q).

    Kept are the points of trajectories still flagged stable whose dimensionless
    coordinates sqrt(omega_i) |q_i| are all <= q_max: the coherent-state overlap
    of Eq. I(E)_discreto falls like exp(-omega q^2 / 4) per mode, so a
    trajectory outside that box adds nothing to the spectrum, while the random
    quartic couplings grow without bound there and would dominate the fit."""
    import torch
    F = w8.F
    dev = "cuda"
    p0 = torch.empty((F, n_traj), dtype=torch.float64, device=dev)
    q0 = torch.empty_like(p0)
    w = torch.empty(n_traj, dtype=torch.float64, device=dev)
    G.scivr_sample_initial(pes, w8.gamma, w8.p_eq[0], w8.q_eq[0], n_traj, seed, p0, q0, w)
    K = seg_steps + 1
    amp = torch.empty((1, n_traj, K, 2), dtype=torch.float64, device=dev)
    good = torch.empty(n_traj, dtype=torch.uint8, device=dev)
    out = torch.empty((n_seg, n_traj, F), dtype=torch.float64, device=dev)
    keep = torch.ones(n_traj, dtype=torch.bool, device=dev)
    rw = torch.as_tensor(np.sqrt(w8.pes.omega), dtype=torch.float64, device=dev)[:, None]
    keep_all = torch.empty((n_seg, n_traj), dtype=torch.bool, device=dev)
    p1 = torch.empty_like(p0)
    q1 = torch.empty_like(q0)
    tol = w8.stab_tol if precision == G.SCIVR_FP64 else 1e-6 * 2.0 ** 29
    for s in range(n_seg):
        G.scivr_propagate(pes, w8.dt, seg_steps, w8.gamma, w8.p_eq[:1], w8.q_eq[:1], n_traj, p0, q0, amp, K,
                          good, precision=precision, stab_tol=tol, fin=dict(p=p1, q=q1))
        out[s] = q1.T
        keep &= good.bool() & torch.isfinite(q1).all(0) & torch.isfinite(p1).all(0)
        keep_all[s] = keep & ((rw * q1).abs() <= q_max).all(0)
        p0, p1 = p1, p0
        q0, q1 = q1, q0
    return out[keep_all].contiguous()


def coupling_targets(pes: G.Pes, q):
    """V and grad V of the coupling polynomial at q [n, F] (float64, device)."""
    import torch
    n, F = q.shape
    V = torch.empty(n, dtype=torch.float64, device=q.device)
    g = torch.empty((n, F), dtype=torch.float64, device=q.device)
    G.scivr_pes_eval(pes, n, q.contiguous(), G.SCIVR_TERMS_COUPLING, V, g)
    return V, g


@dataclasses.dataclass
class TrainResult:
    losses: list
    steps: int
    seconds: float


def train(pes: G.Pes, q, V, g, epochs: int = 20, batch: int = 65536, lr: float = 2e-3, lr_min: float = 1e-5,
          weight_decay: float = 0.0, alpha: float | None = None, beta: float | None = None, seed: int = 0):
    """Fit the residual attached to `pes` to (q, V, g) (device tensors) with
    the Sobolev loss alpha |V - Vref|^2 + beta |grad V - gref|^2 (defaults:
    inverse variances of the targets), AdamW and a cosine learning-rate decay.
    Returns the loss of every step."""
    import time
    import torch
    n, F = q.shape
    qf = q.float().contiguous()
    Vf = V.float().contiguous()
    gf = g.float().contiguous()
    if alpha is None:
        alpha = 1.0 / max(float(V.var()), 1e-300)
    if beta is None:
        beta = 1.0 / max(float(g.var()) * F, 1e-300)
    npar = G.scivr_mlp_param_count(F)
    grad = torch.zeros(npar, device=q.device)
    m1 = torch.zeros(npar, device=q.device)
    m2 = torch.zeros(npar, device=q.device)
    loss = torch.zeros(1, device=q.device)
    batch = min(batch, n)
    nb = n // batch
    total = epochs * nb
    gen = torch.Generator(device="cpu").manual_seed(seed)
    losses = []
    t0 = time.perf_counter()
    t = 0
    for ep in range(epochs):
        perm = torch.randperm(n, generator=gen).to(q.device)
        qs, Vs, gs = qf[perm].contiguous(), Vf[perm].contiguous(), gf[perm].contiguous()
        for b in range(nb):
            sl = slice(b * batch, (b + 1) * batch)
            G.scivr_mlp_loss_grad(pes, batch, qs[sl], Vs[sl], gs[sl], alpha, beta, grad, loss)
            t += 1
            lr_t = lr_min + 0.5 * (lr - lr_min) * (1 + math.cos(math.pi * (t - 1) / max(total, 1)))
            G.scivr_mlp_adamw(pes, grad, m1, m2, t, lr_t, weight_decay=weight_decay)
            losses.append(loss.clone())
    torch.cuda.synchronize()
    return TrainResult([float(x.item()) for x in losses], t, time.perf_counter() - t0)


def surrogate_pes(w8: wl.Workload, mlp: wl.MlpParams) -> wl.PesDesc:
    """Diagonal of the workload's surface plus a learned residual."""
    d = diagonal_part(w8.pes)
    d.mlp = mlp
    return d


def initial_network(w8: wl.Workload, V, seed: int = 0) -> wl.MlpParams:
    """Network for the coupling residual: inputs scaled to dimensionless normal
    coordinates (s_in = sqrt(omega)), output scaled by the targets' spread."""
    s_out = max(float(V.std()), 1e-12)
    return wl.init_mlp(w8.F, G.SCIVR_MLP_HIDDEN, seed, s_in=np.sqrt(w8.pes.omega), s_out=s_out)
