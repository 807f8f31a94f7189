"""fd_cov_err_noalloc: the covariance-error evaluator for callers that cannot
allocate device memory (inside an allocator or pool callback, under strict
memory accounting, or after a server has frozen its allocations). It must give
the value the allocating evaluator (fd_cov_err_pair) gives, on consecutive
calls that share its fixed workspace, and refuse sizes beyond that workspace.
This file is collected last so a failure here comes after every other test."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1501_06561_gb300 import fd
from paper_1501_06561_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-7   # the evaluator tolerance used against the oracle elsewhere


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.init()
    fd.load()


def _pair(n, d, r, seed):
    A = W.random_noisy(n, d, m=min(10, d), seed=seed, dtype=np.float32)
    rng = np.random.default_rng(seed)
    B = (rng.standard_normal((r, d)) * np.sqrt(n / d)).astype(np.float32)
    return torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()


def test_noalloc_matches_allocating_evaluator_twice():
    cases = [_pair(6000, 300, 20, 1), _pair(20000, 1024, 64, 2)]
    ref = [fd.cov_err_pair(A, B)[0] for A, B in cases]
    # two calls in a row on each case, interleaved, through the C ABI
    for _ in range(2):
        for (A, B), r in zip(cases, ref):
            v = fd.cov_err_noalloc(A, B)
            assert abs(v - r) <= TOL, (v, r)


def test_noalloc_fp64_inputs_and_real_sketch():
    A = torch.from_numpy(W.random_noisy(4000, 500, m=30, seed=3, dtype=np.float64)).cuda()
    with fd.FDSketch(500, 40, "fd", 1.0, "fp64") as s:
        s.append(A)
        B = torch.from_numpy(s.sketch()).cuda()
    r = fd.cov_err_pair(A, B)[0]
    for _ in range(2):
        assert abs(fd.cov_err_noalloc(A, B) - r) <= TOL


def test_noalloc_rejects_sizes_beyond_workspace():
    lib = fd.load()
    out = ctypes.c_double()
    A = torch.zeros(8, 1025, device="cuda")
    B = torch.zeros(2, 1025, device="cuda")
    rc = lib.fd_cov_err_noalloc(ctypes.c_void_p(A.data_ptr()), 8, 1025, 1025, 0,
                                ctypes.c_void_p(B.data_ptr()), 2, 0, None, ctypes.byref(out))
    assert rc == -6 and lib.fd_strerror(rc)
    A = torch.zeros(8, 64, device="cuda")
    B = torch.zeros(513, 64, device="cuda")
    rc = lib.fd_cov_err_noalloc(ctypes.c_void_p(A.data_ptr()), 8, 64, 64, 0,
                                ctypes.c_void_p(B.data_ptr()), 513, 0, None, ctypes.byref(out))
    assert rc == -6


def _rel(v, r):
    return abs(v - r) / max(1.0, abs(r))


@pytest.mark.parametrize("d", [1, 3, 5, 1024])
def test_noalloc_against_the_oracle_for_small_and_large_d(d):
    """Widths down to one column: the Lanczos run ends after d steps, and the
    value of that last step is the answer (Sec. 1.1 definition, FP64 oracle)."""
    from oracle import cov_err
    A = W.random_noisy(400, d, m=min(4, d), seed=10 + d, dtype=np.float32)
    rng = np.random.default_rng(d)
    B = (rng.standard_normal((3, d)) * np.sqrt(400 / d)).astype(np.float32)
    ref = cov_err(A, B)
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    for _ in range(2):
        assert _rel(fd.cov_err_noalloc(Ad, Bd), ref) <= TOL
    assert _rel(fd.cov_err_pair(Ad, Bd)[0], ref) <= TOL


def test_noalloc_without_sketch_rows_and_with_strided_views():
    """rows = 0 gives ||A^T A||_2 / ||A||_F^2; an A view with row stride above d
    and a column-sliced B view give the values of their contiguous copies."""
    from oracle import cov_err
    A = W.random_noisy(3000, 200, m=10, seed=21, dtype=np.float32)
    Ad = torch.from_numpy(A).cuda()
    B0 = torch.zeros(0, 200, device="cuda")
    assert _rel(fd.cov_err_noalloc(Ad, B0), cov_err(A, np.zeros((0, 200)))) <= TOL
    big = torch.zeros(3000, 256, device="cuda")
    big[:, :200] = Ad
    Aview = big[:, :200]                      # row stride 256 > d
    rng = np.random.default_rng(22)
    Bbig = torch.from_numpy(rng.standard_normal((12, 300)).astype(np.float32) * 4.0).cuda()
    Bview = Bbig[:, :200]                      # column slice, row stride 300
    ref = fd.cov_err_pair(Ad, Bview.contiguous())[0]
    for _ in range(2):
        assert abs(fd.cov_err_noalloc(Aview, Bview) - ref) <= TOL
