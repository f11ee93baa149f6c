"""Batched multi-molecule runs (scivr_batch_*), F from 3 to 24.

The batch must reproduce, bit for bit, what per-molecule scivr_propagate /
scivr_spectrum calls produce (same kernel arithmetic per trajectory), match
the oracle for an FP64 molecule, and replay identically from a captured
CUDA graph."""
import numpy as np
import pytest

import oracle
from paper_1312_4698_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-6 * 2.0 ** 29


@pytest.fixture(scope="module")
def G():
    import torch
    from paper_1312_4698_gb300 import scivr
    assert torch.cuda.is_available()
    return scivr


def _molecules():
    specs = [(3, 100, 70, 1), (6, 257, 150, 2), (9, 64, 40, 3), (6, 1000, 96, 4), (3, 33, 33, 5),
             (4, 50, 61, 6), (12, 45, 37, 7), (15, 70, 29, 8), (24, 21, 13, 9), (20, 9, 8, 10)]
    out = []
    for F, n, steps, seed in specs:
        w8 = wl.config_f3(n_traj=n, n_steps=steps, n_E=150) if F == 3 else \
            wl.config_generic(F, seed, n, steps, n_E=150)
        out.append(w8.with_(seed=seed))
    return out


def _setup(G, mols, precisions, amp_f32=False):
    import torch
    entries = []
    for w8, prec in zip(mols, precisions):
        pes = G.scivr_create_pes(w8.pes)
        bufs = G.alloc_buffers(w8, amp_f32=amp_f32 and prec == 1)   # FP32 rows only on the mixed path
        G.scivr_sample_initial(pes, w8.gamma, w8.p_eq[0], w8.q_eq[0], w8.n_traj, w8.seed, bufs.p0,
                               bufs.q0, bufs.w)
        entries.append(dict(pes=pes, wl=w8, bufs=bufs, precision=prec,
                            stab_tol=MIXED_TOL if prec == 1 else w8.stab_tol))
    torch.cuda.synchronize()
    return entries


def _reference(G, e, ft_mode):
    import torch
    w8, b = e["wl"], e["bufs"]
    n, K = w8.n_traj, w8.n_steps + 1
    amp = torch.empty_like(b.amp)
    good = torch.empty_like(b.good)
    I = torch.empty_like(b.I)
    ng = torch.zeros_like(b.n_good)
    G.scivr_propagate(e["pes"], w8.dt, w8.n_steps, w8.gamma, w8.p_eq, w8.q_eq, n, b.p0, b.q0, amp, K, good,
                      precision=e["precision"], stab_tol=e["stab_tol"],
                      kernel=G.SCIVR_KERNEL_GROUP if e["precision"] == 1 else G.SCIVR_KERNEL_AUTO)
    G.scivr_spectrum(amp[0], K, b.w, good, n, w8.n_steps, w8.dt, w8.E_min, w8.E_max, w8.n_E, I[0], ng,
                     ft_mode=ft_mode)
    torch.cuda.synchronize()
    return amp, good, I, ng


@pytest.mark.parametrize("ft_mode", [0, 2])
def test_batch_matches_per_molecule_runs(G, ft_mode):
    import torch
    mols = _molecules()
    entries = _setup(G, mols, [1, 1, 1, 1, 1, 0])
    plan = G.scivr_batch_create(entries, ft_mode=ft_mode)
    groups = plan.groups()
    assert sorted(F for F, _, _ in groups) == [3, 6, 9]
    G.scivr_batch_launch(plan)
    torch.cuda.synchronize()
    for e in entries:
        amp, good, I, ng = _reference(G, e, ft_mode)
        b = e["bufs"]
        assert torch.equal(b.good, good)
        assert torch.equal(b.amp, amp)
        assert torch.equal(b.I, I)
        assert int(b.n_good.item()) == int(ng.item())
    assert G.scivr_check_status() == G.SCIVR_OK


@pytest.mark.parametrize("ft_mode", [0, 2])
def test_batch_with_float_amplitude_rows_matches_per_molecule_runs(G, ft_mode):
    """Mixed molecules with complex-float amplitude rows (amp_prec = SCIVR_MIXED) beside an
    FP64 molecule with complex-double rows: the batch equals the per-molecule calls on the
    same row types bit for bit."""
    import torch
    entries = _setup(G, _molecules(), [1, 1, 1, 1, 1, 0], amp_f32=True)
    assert entries[0]["bufs"].amp.dtype == torch.float32 and entries[5]["bufs"].amp.dtype == torch.float64
    plan = G.scivr_batch_create(entries, ft_mode=ft_mode)
    G.scivr_batch_launch(plan)
    torch.cuda.synchronize()
    for e in entries:
        amp, good, I, ng = _reference(G, e, ft_mode)
        b = e["bufs"]
        assert torch.equal(b.good, good)
        assert torch.equal(b.amp, amp)
        assert torch.equal(b.I, I)
        assert int(b.n_good.item()) == int(ng.item())
    assert G.scivr_check_status() == G.SCIVR_OK


def test_batch_of_every_recipe_f_matches_per_molecule_runs(G):
    """The batch recipe's F set, 3, 6, 9, 12, 15 and 24 (with F = 20 besides), in one plan,
    all mixed precision: bit for bit the per-molecule runs, and the same again from a
    captured graph."""
    import torch
    mols = [_molecules()[i] for i in (0, 1, 2, 6, 7, 8, 9)]
    entries = _setup(G, mols, [1] * len(mols))
    plan = G.scivr_batch_create(entries, ft_mode=2)
    assert sorted(F for F, _, _ in plan.groups()) == [3, 6, 9, 12, 15, 20, 24]
    G.scivr_batch_launch(plan)
    torch.cuda.synchronize()
    assert G.scivr_check_status() == G.SCIVR_OK
    for e in entries:
        amp, good, I, ng = _reference(G, e, 2)
        b = e["bufs"]
        assert torch.equal(b.good, good) and torch.equal(b.amp, amp) and torch.equal(b.I, I)
    eager = [(e["bufs"].amp.clone(), e["bufs"].I.clone()) for e in entries]
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    with torch.cuda.graph(graph, stream=side):
        G.scivr_batch_launch(plan, stream=side)
    for e in entries:
        e["bufs"].amp.zero_()
        e["bufs"].I.zero_()
    graph.replay()
    torch.cuda.synchronize()
    for e, (amp, I) in zip(entries, eager):
        assert torch.equal(e["bufs"].amp, amp) and torch.equal(e["bufs"].I, I)


def test_batch_one_persistent_launch_across_f_classes(G, monkeypatch):
    """The one-launch schedule (SCIVR_BATCH_SCHEDULE=one): every molecule of F = 3..24 in one
    persistent kernel that dispatches on each work item's F.  Up to F = 9 (coupling tensors
    in shared memory in both schedules) and at F = 24 (in L2 in both) the results equal the
    per-molecule runs bit for bit; at F = 12 and 15 the one launch reads the tensors from
    L2, so amplitudes agree to rounding (within 1e-5 of each row's largest) and spectra to
    1e-6.  A captured graph replays the plan bit for bit."""
    import torch
    mols = [_molecules()[i] for i in (0, 1, 2, 6, 7, 8)]
    entries = _setup(G, mols, [1] * len(mols))
    monkeypatch.setenv("SCIVR_BATCH_SCHEDULE", "one")
    plan = G.scivr_batch_create(entries, ft_mode=2)
    assert plan.one_launch()
    G.scivr_batch_launch(plan)
    torch.cuda.synchronize()
    assert G.scivr_check_status() == G.SCIVR_OK
    for e in entries:
        amp, good, I, ng = _reference(G, e, 2)
        b = e["bufs"]
        F = e["wl"].F
        if F <= 9 or F == 24:
            assert torch.equal(b.good, good) and torch.equal(b.amp, amp) and torch.equal(b.I, I), F
        else:
            assert torch.equal(b.good, good), F
            a1 = b.amp[0].cpu().numpy()
            a0 = amp[0].cpu().numpy()
            z1, z0 = a1[..., 0] + 1j * a1[..., 1], a0[..., 0] + 1j * a0[..., 1]
            sel = good.cpu().numpy().astype(bool)
            err = np.max(np.abs(z1[sel] - z0[sel]) / np.max(np.abs(z0[sel]), axis=-1, keepdims=True))
            eI = float(torch.max(torch.abs(b.I - I)) / torch.max(torch.abs(I)))
            print(f"F={F}: one launch vs per-class amplitudes {err:.2e}, spectrum {eI:.2e}")
            assert err < 1e-5 and eI < 1e-6
    eager = [(e["bufs"].amp.clone(), e["bufs"].I.clone()) for e in entries]
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    with torch.cuda.graph(graph, stream=side):
        G.scivr_batch_launch(plan, stream=side)
    for e in entries:
        e["bufs"].amp.zero_()
    graph.replay()
    torch.cuda.synchronize()
    for e, (amp, I) in zip(entries, eager):
        assert torch.equal(e["bufs"].amp, amp) and torch.equal(e["bufs"].I, I)
    monkeypatch.setenv("SCIVR_BATCH_SCHEDULE", "per-class")
    assert not G.scivr_batch_create(entries, ft_mode=2).one_launch()


def test_batch_fp64_item_matches_oracle(G):
    import torch
    mols = _molecules()[:3]
    entries = _setup(G, mols, [1, 0, 1])
    plan = G.scivr_batch_create(entries, ft_mode=0)
    G.scivr_batch_launch(plan)
    torch.cuda.synchronize()
    e = entries[1]
    w8, b = e["wl"], e["bufs"]
    p0, q0, w = b.p0.cpu().numpy(), b.q0.cpu().numpy(), b.w.cpu().numpy()
    # the oracle re-samples its own inputs from the same Philox stream
    rp, rq, rw = oracle.sample_initial(w8.gamma, w8.p_eq, w8.q_eq, w8.n_traj, w8.seed)
    assert np.allclose(p0, rp, rtol=1e-13, atol=1e-15)
    ref = oracle.run_workload(w8, rp, rq, rw)
    good = b.good.cpu().numpy()
    assert np.array_equal(good, ref["good"])
    gi = b.I[0].cpu().numpy()
    assert np.max(np.abs(gi - ref["I"][0])) <= 1e-9 * np.max(ref["I"][0])


def test_batch_replays_from_a_captured_graph(G):
    import torch
    mols = _molecules()
    entries = _setup(G, mols, [1] * 6)
    plan = G.scivr_batch_create(entries, ft_mode=2)
    G.scivr_batch_launch(plan)
    torch.cuda.synchronize()
    eager = [(e["bufs"].amp.clone(), e["bufs"].I.clone()) for e in entries]
    for e in entries:
        e["bufs"].amp.zero_()
        e["bufs"].I.zero_()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    with torch.cuda.graph(graph, stream=side):
        G.scivr_batch_launch(plan, stream=side)
    for _ in range(2):
        for e in entries:
            e["bufs"].amp.zero_()
            e["bufs"].I.zero_()
        graph.replay()
        torch.cuda.synchronize()
        for e, (amp, I) in zip(entries, eager):
            assert torch.equal(e["bufs"].amp, amp)
            assert torch.equal(e["bufs"].I, I)


def test_batch_rejects_invalid_items(G):
    mols = _molecules()[:2]
    entries = _setup(G, mols, [1, 1])
    entries[1]["wl"] = entries[1]["wl"].with_(n_E=1)
    with pytest.raises(G.ScivrError) as ei:
        G.scivr_batch_create(entries)
    assert ei.value.code == G.SCIVR_EINVAL
    assert "item 1" in G.last_error()
