"""One stream split across ranks (Sec. 1, distributed streams; the bound of
Lemma 1, Sec. 3.1, carried through the merges).

Each rank sketches a contiguous part of the stream, the parts' sketches and
counters are gathered with one all_gather, and rank 0 folds them with the
fixed merge tree of ``paper_1501_06561_gb300.distributed``. Here the ranks
are gloo processes on CPU and the per-part sketcher is the FP64 oracle (the
host logic under test does not depend on where the sketch arithmetic runs);
rank 0's result must equal the oracle's plain replay of the same plan, and
keep FD's guarantees for the union. The GPU test at the end runs the same
plan through the library (fd_merge_sketch) on one GPU.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp

from oracle import FDOracle, cov_spectrum
from paper_1501_06561_gb300 import distributed as D
from paper_1501_06561_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N, DIM, ELL = 3001, 60, 8


def _stream():
    return W.random_noisy(N, DIM, m=12, seed=31, dtype=np.float64)


class OracleSketch:
    """The oracle behind the interface ``distributed.fold`` uses; merge_sketch
    has the semantics fd_merge_sketch documents."""

    def __init__(self, d, ell):
        self.o = FDOracle(d, ell, "fd")

    def merge_sketch(self, B, st):
        na2, ns = self.o.normA2, self.o.n_seen
        self.o.append(np.asarray(B, dtype=np.float64))
        self.o.normA2 = na2 + st["norm_a2"]
        self.o.n_seen = ns + st["n_seen"]
        self.o.sum_delta += st["sketch_sum_delta"]
        self.o.removed += st["sketch_removed"]
        self.o.reductions += st["reductions"]

    def merge(self, other):
        self.o.merge(other.o)


def _part(A, world, rank):
    r0, r1 = D.shard_bounds(A.shape[0], world, rank)
    o = FDOracle(A.shape[1], ELL, "fd")
    o.append(A[r0:r1])
    B, info = o.sketch()
    stats = dict(d=A.shape[1], ell=ELL, n_seen=info["n_seen"], reductions=info["reductions"],
                 norm_a2=info["normA2"], sketch_sum_delta=info["sum_delta"],
                 sketch_removed=info["removed"])
    return B, stats


def _replay(A, world):
    """The plan written out with the oracle alone, in one process."""
    roots = []
    for r in range(world):
        B, st = _part(A, world, r)
        h = FDOracle(A.shape[1], ELL, "fd")
        rows = B[: D.retained_rows(B)]
        h.append(rows)
        h.normA2, h.n_seen = st["norm_a2"], st["n_seen"]
        h.sum_delta, h.removed, h.reductions = (st["sketch_sum_delta"], st["sketch_removed"],
                                                st["reductions"])
        roots.append(h)
    level = roots
    while len(level) > 1:
        nxt = []
        for i in range(0, len(level) - 1, 2):
            level[i].merge(level[i + 1])
            nxt.append(level[i])
        if len(level) % 2:
            nxt.append(level[-1])
        level = nxt
    return level[0].sketch()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    A = _stream()
    B, st = _part(A, world, rank)
    gathered = D.gather_sketches(B, st, ELL, A.shape[1])
    if rank == 0:
        root, _ = D.fold(lambda: OracleSketch(A.shape[1], ELL), gathered)
        Bm, info = root.o.sketch()
        out[0] = (Bm, info["sum_delta"], info["normA2"], info["n_seen"])
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_fold_the_parts_like_the_oracle_replay(world):
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        Bm, delta, na2, nseen = out[0]
    A = _stream()
    Bo, io = _replay(A, world)
    np.testing.assert_array_equal(Bm, Bo)        # same FP64 operations, same order
    assert delta == io["sum_delta"] and nseen == N
    assert na2 == pytest.approx(float(np.sum(A * A)), rel=1e-13)
    # Lemma 1 over every reduction of every part and of the merges
    lam = cov_spectrum(A, Bm)
    assert lam[-1] >= -1e-9 * na2 and lam[0] <= delta * (1 + 1e-9) + 1e-9 * na2


def test_split_and_fold_order():
    assert [D.shard_bounds(10, 3, r) for r in range(3)] == [(0, 4), (4, 7), (7, 10)]
    assert D.merge_pairs(5) == [(0, 1), (2, 3), (0, 2), (0, 4)]
    rng = np.random.default_rng(3)
    B = np.zeros((ELL, 5))
    B[:3] = rng.standard_normal((3, 5))
    st = dict(d=5, ell=ELL, n_seen=77, reductions=4, norm_a2=12.5, sketch_sum_delta=0.25,
              sketch_removed=3.0)
    rows, back = D.unpack(D.pack(B, st), ELL, 5)
    np.testing.assert_array_equal(rows, B[:3])
    assert back == st


@pytest.mark.gpu
def test_gpu_fold_of_parts_matches_the_oracle_replay():
    """The plan on one GPU: each part sketched by its own handle, its rows and
    counters folded into fresh handles with fd_merge_sketch, then merged with
    fd_merge in the tree order; the oracle replays the same plan."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_06561_gb300 import fd
    from oracle import cov_err
    from helpers import COV_ABS, assert_sigma_parity
    A = _stream()
    world = 3
    gathered = []
    for r in range(world):
        r0, r1 = D.shard_bounds(N, world, r)
        with fd.FDSketch(DIM, ELL, "fd", 1.0, "fp64") as s:
            s.append(torch.from_numpy(A[r0:r1]).cuda())
            B = s.sketch()
            st = s.stats()
        gathered.append(D.unpack(D.pack(B, st), ELL, DIM))
    root, hs = D.fold(lambda: fd.FDSketch(DIM, ELL, "fd", 1.0, "fp64"), gathered)
    Bg = root.sketch()
    stg = root.stats()
    for h in hs:
        h.close()
    Bo, io = _replay(A, world)
    assert stg["n_seen"] == N
    assert abs(stg["norm_a2"] - io["normA2"]) <= 1e-12 * io["normA2"]
    assert_sigma_parity(Bg, Bo, io["normA2"], "fp64", what="distributed fold")
    assert abs(cov_err(A, Bg) - cov_err(A, Bo)) <= COV_ABS


def test_fold_with_empty_parts_equals_replay():
    """More ranks than rows leaves some parts empty: their packed sketches
    carry no rows and zero counters, and the fold gives the oracle's sketch
    of the rows that exist (the merge of an empty sketch is the identity)."""
    A = W.random_noisy(5, DIM, m=3, seed=33, dtype=np.float64)
    world = 8
    gathered = []
    for r in range(world):
        r0, r1 = D.shard_bounds(A.shape[0], world, r)
        o = FDOracle(DIM, ELL, "fd")
        o.append(A[r0:r1])
        B, info = o.sketch()
        st = dict(d=DIM, ell=ELL, n_seen=info["n_seen"], reductions=info["reductions"],
                  norm_a2=info["normA2"], sketch_sum_delta=info["sum_delta"],
                  sketch_removed=info["removed"])
        gathered.append(D.unpack(D.pack(B, st), ELL, DIM))
    assert sum(rows.shape[0] == 0 for rows, _ in gathered) == world - A.shape[0]
    root, _ = D.fold(lambda: OracleSketch(DIM, ELL), gathered)
    Bm, info = root.o.sketch()
    # fewer than ell rows in all: exact recovery, no reduction, Delta = 0
    np.testing.assert_allclose(Bm.T @ Bm, A.T @ A, rtol=0, atol=1e-10 * float(np.sum(A * A)))
    assert info["sum_delta"] == 0.0 and info["n_seen"] == A.shape[0]
