"""Partition of one lattice over ranks by timeslice slabs.

Smearing acts only in the three directions other than j_decay, and every
contraction is a sum within one timeslice, so a lattice split into slabs of
whole timeslices along j_decay needs no exchange at all while the fields are
smeared and contracted: each rank holds the links and propagators of its
own timeslices [t0, t0 + nt) as a lattice of extent nt in that direction,
runs the whole path on it, and the only collective is a gather of the
[channel][momentum][t] correlators at the end (a few KB to MB).  The paper
names multi-GPU operation as future work (Sec. 6); this is the partition its
path allows.

Host logic only: the per-slab computation is a callable (the CUDA path on a
GPU rank, any implementation in a test), and the gather runs over whatever
torch.distributed process group is current (NCCL on GPUs, gloo on CPUs).
"""
from __future__ import annotations

from typing import Callable


def slab(Nt: int, world: int, rank: int) -> tuple[int, int]:
    """First timeslice and count of rank's slab: contiguous, balanced, the
    first Nt % world ranks one timeslice longer."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside a world of {world}")
    if Nt < world:
        raise ValueError(f"{Nt} timeslices cannot give each of {world} ranks a slab")
    base, extra = divmod(Nt, world)
    t0 = rank * base + min(rank, extra)
    return t0, base + (1 if rank < extra else 0)


def slab_dims(dims, j_decay: int, nt: int) -> tuple[int, int, int, int]:
    """Extents of a slab lattice: dims with the decay extent replaced by nt."""
    d = list(dims)
    d[j_decay] = nt
    return tuple(d)


def gather_timeslices(local, Nt: int, world: int, rank: int, group=None):
    """Assemble the full [..., Nt] array on every rank from each rank's
    [..., nt_r] block (torch tensors, complex or real; the last axis is t).
    Slabs of unequal length are padded to the longest for the collective and
    trimmed after it."""
    import torch
    import torch.distributed as dist

    t0, nt = slab(Nt, world, rank)
    if local.shape[-1] != nt:
        raise ValueError(f"rank {rank} holds {local.shape[-1]} timeslices, its slab has {nt}")
    if world == 1:
        return local
    width = slab(Nt, world, 0)[1]
    as_real = torch.view_as_real(local) if local.is_complex() else local
    if as_real is not local:
        as_real = as_real.movedim(-1, -2)            # [..., 2, nt]: t stays last
    pad = torch.zeros(as_real.shape[:-1] + (width,), dtype=as_real.dtype, device=as_real.device)
    pad[..., :nt] = as_real
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad.contiguous(), group=group)
    full = torch.cat([p[..., :slab(Nt, world, r)[1]] for r, p in enumerate(parts)], dim=-1)
    if local.is_complex():
        full = torch.view_as_complex(full.movedim(-2, -1).contiguous())
    return full


def run_partitioned(dims, j_decay: int, world: int, rank: int,
                    compute: Callable[[int, int], "object"], group=None):
    """Compute this rank's slab with compute(t0, nt) -> tensor [..., nt] and
    return the gathered [..., Nt] result (identical on every rank)."""
    Nt = dims[j_decay]
    t0, nt = slab(Nt, world, rank)
    return gather_timeslices(compute(t0, nt), Nt, world, rank, group)
