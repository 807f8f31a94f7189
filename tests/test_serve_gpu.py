"""Serving (fd_serve_*): continuous batching of append requests over many live
sketches. Requests that arrive while others are on the GPU are admitted as
budget frees up; every sketch must end as it would alone (single handle, same
rows in the same order), within the parity tolerance."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cov_err
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
