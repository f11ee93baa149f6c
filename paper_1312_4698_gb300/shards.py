"""Trajectory sharding across ranks and the combination of per-rank spectra.

Trajectories are independent (Sec. III.B of arXiv:1312.4698), so N ranks each
propagate and transform their own trajectories; the only exchange is the sum
of n_good * I(E) and of n_good over ranks (n_E + 1 numbers), after which
I(E) = sum_r n_good_r I_r(E) / sum_r n_good_r.
"""
from __future__ import annotations


def shard_range(n_traj: int, rank: int, world: int):
    """Contiguous [start, stop) of trajectories owned by `rank` (sizes differ by at most one)."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank/world")
    base, extra = divmod(n_traj, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def combine_spectra_async(I_local, n_good_local, group=None):
    """All-reduce (n_good * I, n_good) without a host synchronisation.

    I_local: 1-D float64 tensor; n_good_local: 1-element int64 tensor on the
    same device.  Returns the reduced (n_E + 1)-vector [sum n_good I, sum n_good]."""
    import torch
    import torch.distributed as dist
    ng = n_good_local.to(torch.float64).reshape(1)
    buf = torch.cat([I_local.to(torch.float64) * ng, ng])
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(buf, group=group)
    return buf


def combine_spectra(I_local, n_good_local, group=None):
    """All-reduce (n_good * I, n_good) and return the combined spectrum and n_good.

    I_local: 1-D float64 torch tensor; n_good_local: int or 1-element tensor.
    Works with any torch.distributed backend (NCCL on GPUs, gloo on CPU)."""
    import torch
    if not torch.is_tensor(n_good_local):
        n_good_local = torch.tensor([int(n_good_local)], dtype=torch.int64, device=I_local.device)
    buf = combine_spectra_async(I_local, n_good_local, group)
    ng = int(round(float(buf[-1].item())))
    I = buf[:-1] / ng if ng > 0 else torch.zeros_like(buf[:-1])
    return I, ng
