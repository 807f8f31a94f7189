"""Full-size parity on the single-stream benchmark workload: Random Noisy,
200,000 x 2,000 FP32 rows (k = 50 signal dimensions, zeta = 10, seed 1),
ell = 100, FD, through the same calls the benchmark times.

The FP64 oracle takes minutes at this length. Its values are stored in
golden/c1_full_oracle.json, written by golden/make_c1_full_oracle.py, which
calls only the oracle and the input generator. The test compares what is
unique at any size:
- cov-err (Sec. 1.1) within the 1e-5 absolute bar;
- ||A||_F^2 in FP64;
- the GPU evaluator against the oracle's cov-err of the same GPU sketch;
- Lemma 1 (Sec. 3.1) on the GPU's own counters;
- the removed mass of at least ell * delta per reduction.

Both paths meet the cov-err bar. The FP32 path also meets the per-value
sigma bar; the split-precision BF16x3 path resolves the smallest values near
the cut to about 2^-17 sigma_1^2, and that check is an expected failure for it.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cov_err
from paper_1501_06561_gb300 import fd
from paper_1501_06561_gb300 import workloads as W
from helpers import COV_ABS, assert_sigma_parity

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
with open(os.path.join(HERE, "golden", "c1_full_oracle.json")) as _f:
    GOLD = json.load(_f)
WL = GOLD["workload"]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    fd.load()


@pytest.fixture(scope="module")
def rows():
    A = W.random_noisy(WL["n"], WL["d"], m=WL["m"], zeta=WL["zeta"], seed=WL["seed"],
                       dtype=np.float32, row_stop=WL["n"])
    norm2 = 0.0
    for i in range(0, A.shape[0], 8192):
        blk = A[i:i + 8192].astype(np.float64)
        norm2 += float(np.sum(blk * blk))
    return A, torch.from_numpy(A).cuda(), norm2


def _run(A_dev, prec):
    with fd.FDSketch(WL["d"], WL["ell"], WL["variant"], 1.0, prec) as s:
        s.append(A_dev)
        B = s.sketch()
        st = s.stats()
        ce = s.cov_err(A_dev)
    return B, st, ce


def test_full_stream_fp32_matches_oracle(rows):
    A, A_dev, norm2 = rows
    B, st, ce = _run(A_dev, "fp32")
    ell = WL["ell"]
    assert st["n_seen"] == WL["n"]
    # ||A||_F^2: the FP64 sum of this machine's rows, and the stored workload
    assert abs(st["norm_a2"] - norm2) <= 1e-11 * norm2
    assert abs(st["norm_a2"] - GOLD["normA2"]) <= 1e-6 * GOLD["normA2"]
    # cov-err of the GPU sketch against the oracle's sketch of the same stream
    assert abs(ce - GOLD["cov_err"]) <= COV_ABS, (ce, GOLD["cov_err"])
    # the evaluator against the definition (d x d difference in FP64), same sketch
    co = cov_err(A, B, norm2)
    assert abs(ce - co) <= 1e-6, (ce, co)
    # Lemma 1 summed over the reductions: ||A^T A - B^T B||_2 <= Delta
    delta = st["sketch_sum_delta"]
    assert ce <= delta / st["norm_a2"] + COV_ABS, (ce, delta / st["norm_a2"])
    assert abs(delta - GOLD["sum_delta"]) <= 1e-2 * GOLD["sum_delta"]
    # every reduction removes at least ell * delta (a 2*ell-row buffer)
    assert ell * delta <= (st["norm_a2"] - st["sketch_norm_b2"]) * (1.0 + 1e-6)
    # singular values, per value against the oracle's
    assert_sigma_parity(B, _gold_sketch_diag(), GOLD["normA2"], "fp32", what="C1 full fp32")


def _gold_sketch_diag():
    """A matrix whose singular values are the oracle's stored sigma(B)."""
    return np.diag(np.array(GOLD["sigma"], dtype=np.float64))


def test_full_stream_bf16x3_matches_oracle(rows):
    A, A_dev, norm2 = rows
    B, st, ce = _run(A_dev, "bf16x3")
    assert abs(st["norm_a2"] - norm2) <= 1e-11 * norm2
    assert abs(ce - GOLD["cov_err"]) <= COV_ABS, (ce, GOLD["cov_err"])
    # Lemma 1 (Sec. 3.1) on the path's own counters
    assert ce <= st["sketch_sum_delta"] / st["norm_a2"] + COV_ABS


@pytest.mark.xfail(reason="BF16x3: the smallest values near the cut reach about 2.5x the "
                          "per-value bar on this stream", strict=False)
def test_full_stream_bf16x3_sigma(rows):
    A, A_dev, norm2 = rows
    B, st, ce = _run(A_dev, "bf16x3")
    assert_sigma_parity(B, _gold_sketch_diag(), GOLD["normA2"], "bf16x3", what="C1 full bf16x3")
