"""The host logic of a run over several ranks, on CPU with gloo (world size 2).

bench.py times each rank on its own GPU and reports the slowest rank's time
(a barrier and a max-reduction over ranks); batched and serving work is
sharded by sketch, every rank drawing its own streams. Here two gloo ranks
check the reduction, the aggregate throughput and that the ranks' batched
streams differ, with no GPU.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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
    import bench
    from paper_1501_06561_gb300 import workloads
    r, wsize, _ = bench.dist_env()
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, wsize, device="cpu")
    w = dict(bench.WORKLOADS["c3"])
    specs = workloads.batch_specs(8, seed=bench.rank_batch_seed(w, r))
    dist.barrier()
    out[r] = (ms, [(sp["d"], sp["ell"], sp["n"]) for sp in specs])
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_shard_by_sketch():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert set(res) == {0, 1}
    assert res[0][0] == res[1][0] == 15.0  # every rank reports the slowest (rank 1: 15 ms)
    rows = 1000
    assert rows * world / (res[0][0] / 1e3) == pytest.approx(133333.33, rel=1e-6)
    assert res[0][1] != res[1][1]  # the ranks draw different sketches
