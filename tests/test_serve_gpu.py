"""Serving (fd_serve_*): continuous batching of append requests over many live
sketches. Requests that arrive while others are on the GPU are admitted as
budget frees up; every sketch must end as it would alone (single handle, same
rows in the same order), within the parity tolerance."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cov_err, fd_sketch
from paper_1501_06561_gb300 import fd
from paper_1501_06561_gb300 import workloads as W
from helpers import COV_ABS, assert_sigma_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    fd.load()


def test_serving_mix_equals_solo():
    count, d, ell = 40, 96, 8
    rng = np.random.default_rng(3)
    pool = W.sparse_nonneg_rows(20000, d=d, density=0.1, seed=4)
    reqs = []
    pos = 0
    for _ in range(400):
        sid = int(rng.integers(0, count))
        n = int(np.exp(rng.uniform(0, np.log(300))))
        reqs.append((sid, pos, n))
        pos = (pos + n) % (pool.shape[0] - 400)
    per = {i: [] for i in range(count)}
    tickets = []
    # a small budget forces deferrals: requests wait for earlier ones to finish
    with fd.FDServer(count, d, ell, budget_bytes=64 * d * 4 * 20, streams=2) as srv:
        for sid, p0, n in reqs:
            rows = pool[p0:p0 + n]
            while True:
                t = srv.submit(sid, rows)
                if t is not None:
                    break
                time.sleep(1e-4)
            tickets.append(t)
            per[sid].append(rows)
        srv.drain()
        done = srv.poll()
        assert sorted(t for t, _ in done) == sorted(tickets)
        assert all(lat >= 0 for _, lat in done)
        c = srv.counters()
        assert c["admitted"] == len(reqs) and c["launches"] >= 1
        for sid in range(count):
            if not per[sid]:
                continue
            A = np.vstack(per[sid])
            Bm = srv.sketch(sid)
            with fd.FDSketch(d, ell, "fd", 1.0, "fp32") as s:
                s.append(torch.from_numpy(A).cuda())
                Bs = s.sketch()
            na2 = float(np.sum(A.astype(np.float64) ** 2))
            assert_sigma_parity(Bm, Bs, na2, "fp32", what=f"serve sketch {sid}")
            assert abs(cov_err(A, Bm) - cov_err(A, Bs)) <= COV_ABS
            # and against the FP64 oracle on the same rows
            Bo, io = fd_sketch(A, ell, "fd", 1.0)
            assert_sigma_parity(Bm, Bo, io["normA2"], "fp32", what=f"serve sketch {sid} vs oracle")
            assert abs(cov_err(A, Bm) - cov_err(A, Bo)) <= COV_ABS


def test_serving_matches_oracle_at_the_serving_shape():
    """The serving configuration's sketch shape (d = 512, ell = 32, sparse
    non-negative rows at 2% density with lognormal row norms, request sizes
    log-uniform in 1..4,096) on 12 live sketches: every sketch against the
    FP64 oracle on its own rows, in arrival order."""
    count, d, ell = 12, 512, 32
    rng = np.random.default_rng(11)
    pool = W.sparse_nonneg_rows(40000, d=d, density=0.02, seed=12)
    per = {i: [] for i in range(count)}
    pos = 0
    with fd.FDServer(count, d, ell, budget_bytes=8 * 4096 * d * 4, streams=2) as srv:
        for _ in range(60):
            sid = int(rng.integers(0, count))
            n = int(np.exp(rng.uniform(0, np.log(4096))))
            if pos + n > pool.shape[0]:
                pos = 0
            rows = pool[pos:pos + n]
            pos += n
            while srv.submit(sid, rows) is None:
                time.sleep(1e-4)
            per[sid].append(rows)
        srv.drain()
        srv.poll()
        for sid in range(count):
            if not per[sid]:
                continue
            A = np.vstack(per[sid])
            Bm = srv.sketch(sid)
            Bo, io = fd_sketch(A, ell, "fd", 1.0)
            assert_sigma_parity(Bm, Bo, io["normA2"], "fp32", what=f"serve {sid} (n={A.shape[0]})")
            assert abs(cov_err(A, Bm) - cov_err(A, Bo)) <= COV_ABS
