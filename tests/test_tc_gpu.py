"""Split-precision tensor-core path (FD_PREC_BF16X3: tcgen05 Gram and rotate,
FP32 Jacobi, FP64 shrink) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cov_err, fd_sketch
from paper_1501_06561_gb300 import fd
from paper_1501_06561_gb300 import workloads as W
from helpers import COV_ABS, EPS32, assert_sigma_close, assert_sigma_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    if not fd.load().fd_create:
        pytest.skip("library not loaded")


def _run(A, ell, variant, alpha=1.0, prec="bf16x3"):
    with fd.FDSketch(A.shape[1], ell, variant, alpha, prec) as s:
        s.append(torch.from_numpy(np.ascontiguousarray(A)).cuda())
        B = s.sketch()
        st = s.stats()
    return B, st


def test_tc_one_reduction_tiny():
    """2*ell rows, one reduction: smallest shapes (one k-block, one d tile)."""
    A = W.random_noisy(16, 64, m=4, seed=31, dtype=np.float32)
    B, st = _run(A, 8, "fd")
    Bo, io = fd_sketch(A, 8, "fd")
    assert st["reductions"] == 1
    assert_sigma_parity(B, Bo, io["normA2"], "bf16x3", what="tc tiny")


@pytest.mark.parametrize("variant", ["fd", "pfd", "isvd"])
def test_tc_parity_ragged(variant):
    alpha = 0.2 if variant == "pfd" else 1.0
    A = W.random_noisy(3001, 333, m=12, seed=21, dtype=np.float32)
    B, st = _run(A, 23, variant, alpha)
    Bo, io = fd_sketch(A, 23, variant, alpha)
    assert_sigma_parity(B, Bo, io["normA2"], "bf16x3", what=f"tc {variant}")
    assert abs(cov_err(A, B) - cov_err(A, Bo)) <= COV_ABS
    assert abs(st["norm_a2"] - io["normA2"]) <= 1e-12 * io["normA2"]
    assert st["noconv"] == 0


def test_tc_parity_c0_shape():
    A = W.random_noisy(10000, 500, m=30, seed=0, dtype=np.float32)
    B, st = _run(A, 50, "fd")
    Bo, io = fd_sketch(A, 50, "fd")
    assert_sigma_parity(B, Bo, io["normA2"], "bf16x3", what="tc C0")
    assert abs(cov_err(A, B) - cov_err(A, Bo)) <= COV_ABS


def test_tc_multi_tile_gram_and_flush():
    """2*ell = 200 rows (two 128-row Gram tiles), d = 1100 (9 d tiles), and a
    flush of pending rows at the end."""
    A = W.random_noisy(2 * 100 + 101 * 7 + 55, 1100, m=40, seed=32, dtype=np.float32)
    B, st = _run(A, 100, "fd")
    Bo, io = fd_sketch(A, 100, "fd")
    assert_sigma_parity(B, Bo, io["normA2"], "bf16x3", what="tc 2 tiles")
    assert abs(cov_err(A, B) - cov_err(A, Bo)) <= COV_ABS


def test_tc_ss_short_stream():
    A = W.random_noisy(2 * 30 + 5 * 31 + 7, 257, m=10, seed=22, dtype=np.float32)
    B, st = _run(A, 30, "ss")
    Bo, io = fd_sketch(A, 30, "ss")
    assert_sigma_parity(B, Bo, io["normA2"], "bf16x3", what="tc ss")
    assert abs(st["sketch_norm_b2"] - io["normA2"]) <= 1e-5 * io["normA2"]
