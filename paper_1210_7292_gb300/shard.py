"""Splitting one level's M2L across ranks (one process per GPU).

Target cells are independent: each local expansion is owned by exactly one
rank, so the level shards by contiguous ranges of target cells with no
reduction across ranks.  A rank reads the multipoles of every source in its
targets' interaction lists, up to three cells beyond its range in each
direction (|t|_inf <= 3, Sec. 3.2); with each rank owning the multipoles of
the same range of cells, those arrive through one exchange per level, an
all-gather of the level's multipole vectors, before the rank's apply.

Everything here is integer bookkeeping on the host plus that one collective.
"""
from __future__ import annotations

import numpy as np


def target_ranges(ntgt: int, world: int):
    """[(t0, t1)] contiguous target ranges, sizes differing by at most one."""
    base, extra = divmod(ntgt, world)
    out, t = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append((t, t + n))
        t += n
    return out


def shard_level(offsets: np.ndarray, sources: np.ndarray, rank: int, world: int):
    """The sub-problem of `rank`: its target range [t0, t1), the sorted global ids
    of the source cells its lists read, and its CSR lists re-indexed into them.
    The order of each target's list is kept."""
    offsets = np.asarray(offsets, dtype=np.int64)
    sources = np.asarray(sources, dtype=np.int64)
    t0, t1 = target_ranges(len(offsets) - 1, world)[rank]
    e0, e1 = int(offsets[t0]), int(offsets[t1])
    src_g = sources[e0:e1]
    needed = np.unique(src_g)
    return {"t0": t0, "t1": t1, "needed": needed.astype(np.int64),
            "offsets": (offsets[t0:t1 + 1] - e0).astype(np.int32),
            "sources": np.searchsorted(needed, src_g).astype(np.int32)}


def exchange_multipoles(local_rows, ranges, needed, group=None):
    """All-gather of one level's multipole vectors (each rank holds the rows of its
    own range, `local_rows` [t1 - t0, n3]); returns the rows `needed` by this rank.
    torch.distributed must be initialised (NCCL on GPUs, gloo on CPU)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    n3 = local_rows.shape[1]
    width = max(r[1] - r[0] for r in ranges)
    buf = torch.zeros(width, n3, dtype=local_rows.dtype, device=local_rows.device)
    buf[: local_rows.shape[0]] = local_rows
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    full = torch.cat([p[: r[1] - r[0]] for p, r in zip(parts, ranges)], dim=0)
    idx = torch.as_tensor(np.asarray(needed), dtype=torch.long, device=full.device)
    return full.index_select(0, idx)
