"""Multi-rank spectrum combination, run as world_size-2 gloo process groups on CPU.

Each rank computes the oracle spectrum of its shard of trajectories; the
combined spectrum must equal the spectrum of all trajectories at once."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_1312_4698_gb300 import shards
from paper_1312_4698_gb300 import workloads as wl


def test_shard_ranges_partition():
    for n in (1, 7, 64, 1001):
        for world in (1, 2, 3, 8):
            ranges = [shards.shard_range(n, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            for (a, b), (c, d) in zip(ranges, ranges[1:]):
                assert b == c
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, inputs, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    amp, w, good, n_steps, dt, E_min, E_max, n_E = inputs
    a, b = shards.shard_range(amp.shape[0], rank, world)
    I, ng = oracle.spectrum(amp[a:b], w[a:b], good[a:b], n_steps, dt, E_min, E_max, n_E)
    Ic, ngc = shards.combine_spectra(torch.as_tensor(I), ng)
    out.put((rank, Ic.numpy(), ngc))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_combination_equals_single_run():
    import torch.multiprocessing as mp
    w8 = wl.config_f3(n_traj=37, n_steps=120, n_E=90)
    p0, q0, w = oracle.sample_initial(w8.gamma, w8.p_eq, w8.q_eq, w8.n_traj, 3)
    amp, good = oracle.propagate(w8.pes, w8.gamma, w8.p_eq, w8.q_eq, w8.dt, w8.n_steps, p0, q0)
    good[4] = 0     # a bad trajectory on rank 0 changes n_good there
    inputs = (amp[0], w, good, w8.n_steps, w8.dt, w8.E_min, w8.E_max, w8.n_E)
    ref, ng_ref = oracle.spectrum(*inputs)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, inputs, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, I, ng in results:
        assert ng == ng_ref
        assert np.max(np.abs(I - ref)) <= 1e-12 * np.max(ref)


def _rank_main_hk(rank, world, port, inputs, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    amp, good, n_steps, dt, E_min, E_max, n_E = inputs
    a, b = shards.shard_range(amp.shape[0], rank, world)
    I, ng, _ = oracle.spectrum_hk(amp[a:b], good[a:b], n_steps, dt, E_min, E_max, n_E)
    Ic, ngc = shards.combine_spectra(torch.as_tensor(I), ng)
    out.put((rank, Ic.numpy(), ngc))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_hk_combination_with_an_all_bad_rank():
    """The plain HK spectrum is linear in the mean summand, so the same n_good-weighted
    combination is exact; rank 1's trajectories are all flagged bad (its n_good is 0)."""
    import torch.multiprocessing as mp
    w8 = wl.config_f3(n_traj=30, n_steps=100, n_E=80)
    p0, q0, w = oracle.sample_initial(w8.gamma, w8.p_eq, w8.q_eq, w8.n_traj, 5)
    amp, good = oracle.propagate(w8.pes, w8.gamma, w8.p_eq, w8.q_eq, w8.dt, w8.n_steps, p0, q0,
                                 amplitude=oracle.AMP_HK)
    a, b = shards.shard_range(w8.n_traj, 1, 2)
    good[a:b] = 0
    inputs = (amp[0], good, w8.n_steps, w8.dt, w8.E_min, w8.E_max, w8.n_E)
    ref, ng_ref, _ = oracle.spectrum_hk(*inputs)
    assert ng_ref == int(good.sum()) > 0
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main_hk, args=(r, 2, port, inputs, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, I, ng in results:
        assert ng == ng_ref
        assert np.max(np.abs(I - ref)) <= 1e-12 * np.max(np.abs(ref))
