"""Slabs along t: the partition of a volume among ranks (or among turns on one GPU), the one
exchange between ranks, and the per-rank pipeline of the C ABI's slab calls.

The method's only global quantity is the (min, max) of each S_m before Eq. 6; everything
else depends on a bounded neighbourhood (h = (L-1)/2 planes of V for E, r_t planes of E for
S_m).  So each rank is given its own planes plus H = h + r_t planes of V on each side (read
straight from the input; no intermediate is exchanged), computes its S_m and their local
statistics, all-gathers the 9 doubles, merges them (a library kernel) and combines its own
planes.  Marshalling and the collective only: the arithmetic runs in libsal's kernels.
"""
from __future__ import annotations

from dataclasses import dataclass


@dataclass(frozen=True)
class Slab:
    own_lo: int
    own_hi: int
    ext_lo: int
    ext_hi: int


def slab_partition(T: int, parts: int, halo: int) -> list[Slab]:
    """Splits the T planes into `parts` contiguous slabs of sizes differing by at most one
    (the first T % parts slabs take the extra plane), each with its halo of `halo` planes
    clipped to the volume.  Every plane is owned by exactly one slab; parts > T is refused."""
    if parts < 1 or T < 1:
        raise ValueError("need T >= 1 and parts >= 1")
    if parts > T:
        raise ValueError(f"{parts} slabs of a volume of {T} planes would leave some empty")
    base, extra = divmod(T, parts)
    out, lo = [], 0
    for r in range(parts):
        hi = lo + base + (1 if r < extra else 0)
        out.append(Slab(lo, hi, max(0, lo - halo), min(T, hi + halo)))
        lo = hi
    return out


def gather_stats(stats_local, group=None):
    """All ranks' 9 statistics as one [world, 9] tensor on the device of `stats_local` (an
    all-gather of 9 doubles per rank: NCCL for CUDA tensors, gloo for CPU tensors)."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    parts = [torch.empty_like(stats_local) for _ in range(world)]
    dist.all_gather(parts, stats_local.contiguous(), group=group)
    return torch.stack(parts)


def saliency_slab(V_ext, dims, slab: Slab, p, group=None, stream=None):
    """One rank's part of the sharded method on its GPU: S of its own planes [own, X, Y] and
    the merged statistics [9].  V_ext holds the planes [slab.ext_lo, slab.ext_hi) of V."""
    import torch.distributed as dist

    from . import api

    Sm, st = api.sal_slab_maps(V_ext, dims, slab.ext_lo, slab.ext_hi, slab.own_lo, slab.own_hi, p, stream=stream)
    every = gather_stats(st, group) if dist.is_available() and dist.is_initialized() else st.reshape(1, -1)
    merged = api.sal_stats_merge(every, stream=stream)
    return api.sal_combine(Sm, merged, p, stream=stream), merged
