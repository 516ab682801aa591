"""Several processes (one GPU each) sharing the slice terms of the same amplitudes.

The 2^k slice terms are independent (Section 3.B.2): rank r of `world` takes the
contiguous range slice_range(2^k, r, world), computes the FP64 sum of its terms per
bitstring through qvx_amplitude_slices, and the ranks exchange those B complex128 partial
sums once (all_gather) and add them in a fixed rank order with compensation, so every
rank ends with the same amplitudes regardless of the backend's reduction order.
"""
from __future__ import annotations


def slice_range(total: int, rank: int, world: int) -> tuple:
    """[begin, end) of rank's contiguous share of `total` slice terms (sizes differ by <= 1)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    base, extra = divmod(total, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def compensated_sum(parts):
    """Neumaier sum over the first axis of a [world, B] complex array (rank order)."""
    import numpy as np
    parts = np.asarray(parts, dtype=np.complex128)
    out = np.zeros(parts.shape[1:], dtype=np.complex128)
    for comp in (np.real, np.imag):
        s = np.zeros(parts.shape[1:], dtype=np.float64)
        c = np.zeros_like(s)
        for v in comp(parts):
            t = s + v
            c += np.where(np.abs(s) >= np.abs(v), (s - t) + v, (v - t) + s)
            s = t
        if comp is np.real:
            out.real = s + c
        else:
            out.imag = s + c
    return out


def sharded_amplitude(partial, total: int, group=None):
    """partial(begin, count) -> this rank's complex128 numpy partial sums [B]; returns the
    full amplitudes [B] on every rank of the torch.distributed group."""
    import numpy as np
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    b, e = slice_range(total, rank, world)
    mine = np.asarray(partial(b, e - b), dtype=np.complex128)
    t = torch.from_numpy(np.stack([mine.real, mine.imag], axis=-1).copy())
    backend = dist.get_backend(group)
    if backend == "nccl":
        t = t.cuda()
    gathered = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(gathered, t, group=group)
    parts = np.stack([g.cpu().numpy() for g in gathered])
    return compensated_sum(parts[..., 0] + 1j * parts[..., 1])


def plan_partial(plan, bitstrings):
    """The partial function for a qvx plan on this rank's GPU."""
    def f(begin, count):
        return plan.amplitude(bitstrings, slice_begin=begin, slice_count=count).cpu().numpy()
    return f
