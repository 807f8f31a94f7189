"""Host-side helpers of bench.py that need no GPU.

mass_account turns a sketch's counters into the bookkeeping the benchmark
reports: ||A||_F^2 - removed - ||B||_F^2 (zero in exact arithmetic, since
every reduction removes exactly the mass it takes off the spectrum) and
Lemma 1's bound Delta / ||A||_F^2 on cov-err (Sec. 3.1). Fed with the FP64
oracle's counters, the gap is zero to rounding and the bound holds.
mass_trajectory reads the same account at evenly spaced prefixes of the
stream; a fake sketch checks that its chunks cover the stream once.
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


class _FakeSketch:
    """Stands in for FDSketch: counts appended rows and reports a mass
    account whose gap grows with them."""

    def __init__(self):
        self.rows, self.chunks, self.sketches = 0, [], 0

    def reset(self):
        self.rows, self.chunks = 0, []

    def append(self, A):
        self.chunks.append(int(A.shape[0]))
        self.rows += int(A.shape[0])

    def sketch(self, out=None):
        self.sketches += 1
        return out

    def stats(self):
        a2 = float(self.rows)
        return {"norm_a2": a2, "sketch_removed": 0.5 * a2, "sketch_norm_b2": 0.5 * a2 - 1e-3 * a2,
                "sketch_sum_delta": 0.25 * a2}


def test_mass_trajectory_points_cover_the_stream():
    A = np.zeros((1003, 4))
    sk = _FakeSketch()
    traj = bench.mass_trajectory(sk, A, None, points=8)
    assert [p["rows"] for p in traj] == sorted({round(1003 * (k + 1) / 8) for k in range(8)})
    assert traj[-1]["rows"] == 1003 and sum(sk.chunks) == 1003 and sk.sketches == 8
    for p in traj:
        assert abs(p["gap_rel"] - 1e-3) < 1e-12 and p["lemma1_bound"] == 0.25
    # fewer rows than points: every point is a distinct, nonempty prefix
    traj = bench.mass_trajectory(_FakeSketch(), np.zeros((3, 2)), None, points=8)
    assert [p["rows"] for p in traj] == [1, 2, 3]
