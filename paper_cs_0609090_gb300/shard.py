"""Frame sharding over ranks (one process per GPU).

Frames are independent (every decode step of Sections III-V acts on one frame),
so a batch is split into contiguous frame ranges with the code replicated on
every rank; nothing is exchanged during decoding.  Afterwards the ranks gather
their decisions and iteration counts (``gather_outputs``) or sum their error
counts (``sum_counts``): one collective each, outside the decode.
"""
from __future__ import annotations

import numpy as np


def frame_range(n_frames: int, world: int, rank: int) -> tuple:
    """[start, stop) of rank's frames: contiguous, sizes differing by at most one."""
    if world < 1 or not 0 <= rank < world or n_frames < 0:
        raise ValueError(f"bad shard request: n_frames={n_frames} world={world} rank={rank}")
    base, extra = divmod(n_frames, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def gather_outputs(parts: dict, n_frames: int, group=None) -> dict:
    """All-gathers per-rank outputs (dict of [f_local, ...] arrays, frames in
    rank order) into full [n_frames, ...] arrays on every rank.  Ranks may hold
    different frame counts (``frame_range``)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    out = {}
    for key in sorted(parts):
        a = np.ascontiguousarray(parts[key])
        rows = max(frame_range(n_frames, world, r)[1] - frame_range(n_frames, world, r)[0] for r in range(world))
        pad = np.zeros((rows,) + a.shape[1:], dtype=a.dtype)
        pad[:a.shape[0]] = a
        t = torch.from_numpy(pad)
        bufs = [torch.empty_like(t) for _ in range(world)]
        dist.all_gather(bufs, t, group=group)
        pieces = []
        for r, b in enumerate(bufs):
            s, e = frame_range(n_frames, world, r)
            pieces.append(b.numpy()[:e - s])
        out[key] = np.concatenate(pieces, axis=0)
    return out


def sum_counts(values, group=None) -> np.ndarray:
    """Sums small integer counters (frame errors, bit errors, frames) over ranks."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(np.asarray(values, dtype=np.int64))
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.numpy()


def max_over_ranks(values, group=None) -> np.ndarray:
    """Maximum of small float vectors over ranks (the bench's timing rule)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor(np.asarray(values, dtype=np.float64))
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return t.numpy()
