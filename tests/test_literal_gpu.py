"""The literal, unbuffered Algorithms 1-3 on the GPU (fd_create_buffered with
buffer_rows == ell) against the oracle's literal mode, through the C ABI.

Algorithm 1 as printed keeps an ell-row sketch: each row goes into a zero row,
and when none is left the sketch is reduced (Sec. 2.3), which for generic data
leaves exactly ell-1 nonzero rows, so a reduction follows every row once the
sketch is full. The ReduceRank rules are those of FD (Sec. 2.3), alpha-FD
(Algorithm 2), SpaceSaving Directions (Algorithm 3) and iSVD (Sec. 2.1). The
oracle replays the printed algorithm row by row (``mode="literal"``), with
its own zero-row bookkeeping; the GPU uses the buffered machinery with a
buffer of ell rows. Same bar as the other parity tests.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import FDOracle, cov_err, cov_spectrum
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


# SS takes discrete merge decisions, so its element-wise comparison is kept to
# a short stream (see the SS parity reading); the others run 600 rows.
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("variant,alpha,n", [("fd", 1.0, 600), ("pfd", 0.25, 600),
                                             ("isvd", 1.0, 600), ("ss", 1.0, 24)])
def test_literal_algorithms_match_oracle(variant, alpha, n, prec):
    ell, d = 8, 40
    A = W.random_noisy(n, d, m=5, seed=71, dtype=np.float32)
    with fd.FDSketch(d, ell, variant, alpha, prec, buffer_rows=ell) as s:
        s.append(torch.from_numpy(A).cuda())
        B = s.sketch()
        st = s.stats()
    o = FDOracle(d, ell, variant, alpha, mode="literal")
    o.append(A)
    Bo, io = o.sketch()
    assert st["n_seen"] == n
    # one reduction per row once the sketch is full
    assert st["reductions"] == io["reductions"] == n - ell + 1
    assert abs(st["norm_a2"] - io["normA2"]) <= 1e-12 * io["normA2"]
    assert abs(st["sketch_sum_delta"] - io["sum_delta"]) <= 1e-5 * max(io["sum_delta"], 1e-30)
    assert_sigma_parity(B, Bo, io["normA2"], prec, what=f"literal {variant}/{prec}")
    ce_g, ce_o = cov_err(A, B), cov_err(A, Bo)
    assert abs(ce_g - ce_o) <= COV_ABS, (ce_g, ce_o)
    if variant in ("fd", "pfd"):
        # Lemma 1 (Sec. 3.1) on the GPU's own counters
        lam = cov_spectrum(A, B)
        assert lam[-1] >= -1e-9 * io["normA2"]
        assert lam[0] <= st["sketch_sum_delta"] * (1 + 1e-6) + 1e-9 * io["normA2"]


def test_literal_rejects_other_small_buffers():
    """Buffers between ell and 2*ell rows are refused (FD_EINVAL)."""
    with pytest.raises(fd.FDError):
        fd.FDSketch(40, 8, "fd", 1.0, "fp32", buffer_rows=12)
