"""Compensative FD (fd_sketch_compensated, Sec. 3.1) vs the FP64 oracle.

The GPU rescales each nonzero row of the (orthogonal-row) sketch; the oracle
takes the SVD of its sketch and rebuilds S-hat V^T. The two agree up to a
left rotation, so they are compared through what is unique: singular values
(per-value allowance), cov-err (1e-5 absolute) and the two-sided bound with
the GPU's own Delta.
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


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
@pytest.mark.parametrize("variant,alpha", [("fd", 1.0), ("pfd", 0.4)])
def test_compensated_matches_oracle(variant, alpha, prec):
    """3,001 x 290 Random Noisy stream (ragged tail at the flush), ell = 21."""
    A = W.random_noisy(3001, 290, m=10, seed=91, dtype=np.float32)
    with fd.FDSketch(290, 21, variant, alpha, prec) as s:
        s.append(torch.from_numpy(A).cuda())
        B0 = s.sketch()
        Bh = s.sketch_compensated()
        B1 = s.sketch()
        st = s.stats()
        Bd = torch.zeros((21, 290), dtype=torch.float32, device="cuda")
        s.sketch_compensated(out=Bd)
        torch.cuda.synchronize()
    np.testing.assert_array_equal(B0, B1)  # non-destructive
    np.testing.assert_allclose(Bd.cpu().numpy(), Bh.astype(np.float32), rtol=0, atol=0)
    o = FDOracle(290, 21, variant, alpha)
    o.append(A)
    Bho, io = o.sketch_compensated()
    assert abs(st["sketch_sum_delta"] - io["sum_delta"]) <= 1e-4 * io["sum_delta"]
    assert_sigma_parity(Bh, Bho, io["normA2"], prec, what=f"cfd {variant}/{prec}")
    ce_g, ce_o = cov_err(A, Bh), cov_err(A, Bho)
    assert abs(ce_g - ce_o) <= COV_ABS, (ce_g, ce_o)
    lam = cov_spectrum(A, Bh)
    D = st["sketch_sum_delta"]
    assert lam[0] >= -D * (1 + 1e-3) and lam[-1] <= D * (1 + 1e-3), (lam[0], lam[-1], D)


def test_compensated_short_stream_is_the_sketch():
    """No reduction (Delta = 0): the compensated sketch is the sketch."""
    A = W.random_noisy(15, 64, m=4, seed=92, dtype=np.float32)
    with fd.FDSketch(64, 20) as s:
        s.append(torch.from_numpy(A).cuda())
        np.testing.assert_array_equal(s.sketch_compensated(), s.sketch())


def test_compensated_rejects_other_variants():
    for v in ("ss", "isvd"):
        with fd.FDSketch(32, 4, v) as s:
            with pytest.raises(fd.FDError):
                s.sketch_compensated()
