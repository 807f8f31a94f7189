"""Host-side helpers of bench.py that need no GPU.

mass_account turns a sketch's counters into the bookkeeping the benchmark
reports: ||A||_F^2 - removed - ||B||_F^2 (zero in exact arithmetic, since
every reduction removes exactly the mass it takes off the spectrum) and
Lemma 1's bound Delta / ||A||_F^2 on cov-err (Sec. 3.1). Fed with the FP64
oracle's counters, the gap is zero to rounding and the bound holds.
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from oracle import cov_err, fd_sketch  # noqa: E402
from paper_1501_06561_gb300 import workloads as W  # noqa: E402


def _stats_from_oracle(info):
    return {"norm_a2": info["normA2"], "sketch_removed": info["removed"],
            "sketch_norm_b2": info["normB2"], "sketch_sum_delta": info["sum_delta"]}


def test_mass_account_of_an_oracle_sketch():
    A = W.random_noisy(3000, 200, m=20, seed=41, dtype=np.float64)
    B, info = fd_sketch(A, 20, "fd")
    acc = bench.mass_account(_stats_from_oracle(info))
    assert abs(acc["gap_rel"]) <= 1e-12
    assert acc["norm_b2"] == info["normB2"]
    ce = cov_err(A, B, info["normA2"])
    assert 0.0 <= ce <= acc["lemma1_bound"] * (1 + 1e-12)


def test_mass_account_values():
    acc = bench.mass_account({"norm_a2": 10.0, "sketch_removed": 3.0, "sketch_norm_b2": 6.5,
                              "sketch_sum_delta": 0.25})
    assert acc == {"norm_a2": 10.0, "removed": 3.0, "norm_b2": 6.5, "sum_delta": 0.25,
                   "gap_rel": 0.05, "lemma1_bound": 0.025}
    empty = bench.mass_account({"norm_a2": 0.0, "sketch_removed": 0.0, "sketch_norm_b2": 0.0,
                                "sketch_sum_delta": 0.0})
    assert empty["gap_rel"] == 0.0 and empty["lemma1_bound"] == 0.0
