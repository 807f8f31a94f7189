"""One row stream split across ranks (one process per GPU).

The paper states the sketching problem for streams that may be distributed
(Sec. 1). FD sketches merge: a sketch's rows, appended to another stream as
ordinary rows, give a sketch of the union, and Lemma 1 (Sec. 3.1) applied to
every reduction of both streams bounds the union's error by the sum of all
deltas. So each rank sketches a contiguous part of the stream on its own
GPU, the parts' sketches (at most ell rows each, plus their FP64 counters)
are gathered with one collective, and one rank folds them together with a
fixed merge tree. The exchange is the only data-path collective.

This module holds the host logic of that plan: the contiguous split, the
packing of a sketch and its counters into one FP64 vector, the gather
(torch.distributed: NCCL between GPUs, gloo on CPU) and the fold order. The
sketch arithmetic itself runs in the library (``fd.FDSketch.merge_sketch``
and ``fd.merge_tree``); any object with the same ``merge_sketch`` /
``merge`` / ``sketch`` / ``stats`` methods can be folded, which is how the
host logic is tested without a GPU.
"""
from __future__ import annotations

import numpy as np

# counters of a sketch that travel with its rows (fd_stats_t fields)
COUNTERS = ("d", "ell", "n_seen", "reductions", "norm_a2", "sketch_sum_delta", "sketch_removed")


def shard_bounds(n: int, world: int, rank: int):
    """Rows [r0, r1) of rank ``rank`` in a contiguous split of n rows: the
    first n % world ranks take one row more."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    base, extra = divmod(int(n), int(world))
    r0 = rank * base + min(rank, extra)
    return r0, r0 + base + (1 if rank < extra else 0)


def retained_rows(B) -> int:
    """Rows of a sketch up to its last nonzero row (the ones a merge appends)."""
    B = np.asarray(B)
    nz = np.flatnonzero(np.any(B != 0.0, axis=1))
    return int(nz[-1]) + 1 if nz.size else 0


def pack(B, stats: dict) -> np.ndarray:
    """One FP64 vector: [rows, counters..., B (ell x d, row-major)]."""
    B = np.asarray(B, dtype=np.float64)
    head = [float(retained_rows(B))] + [float(stats[f]) for f in COUNTERS]
    return np.concatenate([np.array(head), B.ravel()])


def unpack(v, ell: int, d: int):
    """Inverse of ``pack``: (rows of the sketch up to its last nonzero row,
    the counters as a dict)."""
    v = np.asarray(v, dtype=np.float64)
    rows = int(v[0])
    h = 1 + len(COUNTERS)
    stats = {f: v[1 + i] for i, f in enumerate(COUNTERS)}
    for f in ("d", "ell", "n_seen", "reductions"):
        stats[f] = int(round(stats[f]))
    B = v[h:h + ell * d].reshape(ell, d)
    return B[:rows].copy(), stats


def gather_sketches(B, stats: dict, ell: int, d: int, group=None, device="cpu"):
    """All ranks' sketches on every rank, in rank order, as (rows, counters)
    pairs: one all_gather of equal-length FP64 vectors (ell x d values plus
    the counters, about 1.6 MB at ell = 100, d = 2,000)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    mine = torch.from_numpy(pack(B, stats)).to(device)
    parts = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(parts, mine, group=group)
    return [unpack(p.cpu().numpy(), ell, d) for p in parts]


def merge_pairs(count: int):
    """The fold order of ``merge_tree``: per level, (0, 1), (2, 3), ... with
    the right member merged into the left one, until one is left."""
    level = list(range(count))
    out = []
    while len(level) > 1:
        nxt = []
        for i in range(0, len(level) - 1, 2):
            out.append((level[i], level[i + 1]))
            nxt.append(level[i])
        if len(level) % 2:
            nxt.append(level[-1])
        level = nxt
    return out


def fold(make_sketch, gathered):
    """Rank 0's step: one empty sketch per gathered part takes that part's
    rows and counters (``merge_sketch``), then the parts are merged in the
    order of ``merge_pairs``. Returns the root sketch and all handles (the
    caller closes them)."""
    handles = []
    for B, st in gathered:
        h = make_sketch()
        h.merge_sketch(B, st)
        handles.append(h)
    for a, b in merge_pairs(len(handles)):
        handles[a].merge(handles[b])
    return handles[0], handles
