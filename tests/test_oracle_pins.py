"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each check is independent of the oracle's own code path: hand-derived
ReduceRank values (golden file), a replay of the whole stream in covariance
form (eigendecomposition of the d x d matrix instead of the SVD of the rows),
exact recovery of low-rank input, Properties 1-3 and Lemmas 1 and 3 (Sec. 3.1),
the alpha-FD error bound (Theorem, Sec. 3.1), the SS mass identity and bound
(Theorem on SpaceSaving Directions, Sec. 3.1), closed forms / brute force
for the covariance error and the projection error (Sec. 1.1), and the bounds
of compensative FD (Sec. 3.1).
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import (FDOracle, compensate, cov_err, cov_spectrum, fast_pfd_split, fd_sketch,
                    jacobi_svd_rows, proj_err, reduce_rank)
from paper_1501_06561_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
VARS = ["fd", "pfd", "ss", "isvd", "fastpfd"]


def _alpha(v):
    return {"pfd": 0.5, "fastpfd": 0.4}.get(v, 1.0)


# --------------------------------------------------------------------------
# ReduceRank rules: hand-derived values
# --------------------------------------------------------------------------
def test_reduce_rank_golden_cases():
    cases = json.load(open(os.path.join(HERE, "golden", "reduce_rank_cases.json")))["cases"]
    for c in cases:
        sigma = np.sqrt(np.array(c["mass"], dtype=float))
        sp, deltas = reduce_rank(sigma, c["ell"], c["variant"], c["alpha"], c.get("mass_floor", 0.0))
        np.testing.assert_allclose(sp * sp, c["mass_prime"], rtol=1e-12, atol=1e-12,
                                   err_msg=c["name"])
        np.testing.assert_allclose(deltas, c["deltas"], rtol=1e-12, atol=1e-12,
                                   err_msg=c["name"])


# --------------------------------------------------------------------------
# Whole-stream replay in covariance form (independent of the row SVD)
# --------------------------------------------------------------------------
def _cov_replay(A, ell, variant, alpha, mode):
    """Track C = B^T B (d x d) through the stream using eigh of C only.

    An SVD of the sketch rows X gives sigma_j^2 = eigenvalues of X^T X and
    v_j = its eigenvectors, so one reduction maps C to
    sum_j sigma'_j^2 v_j v_j^T. The cadence is the oracle contract: buffered
    mode reduces at 2*ell rows and leaves ell-1; literal mode reduces when the
    ell-row sketch has no zero row (rank-nullity: the number of nonzero rows
    after a reduction is the number of nonzero sigma').
    """
    d = A.shape[1]
    C = np.zeros((d, d))
    cap = 2 * ell if (mode == "buffered" and variant != "fastpfd") else ell
    left = ell - 1 if variant != "fastpfd" else fast_pfd_split(ell, alpha)[1] - 1
    rows = 0
    sum_delta = 0.0

    def reduce(C, nrows):
        lam, V = np.linalg.eigh(C)
        lam, V = lam[::-1], V[:, ::-1]
        k = min(nrows, d)
        lam = np.clip(lam[:k], 0.0, None)
        sig = np.zeros(nrows)
        sig[:k] = np.sqrt(lam)
        sp, deltas = reduce_rank(sig, ell, variant, alpha)
        Cn = (V[:, :k] * (sp[:k] ** 2)[None, :]) @ V[:, :k].T
        return Cn, deltas, int(np.sum(sp > 0))

    for a in A:
        C = C + np.outer(a, a)
        rows += 1
        if rows == cap:
            C, deltas, nz = reduce(C, rows)
            sum_delta += sum(deltas)
            rows = left if mode == "buffered" else nz
    if mode == "buffered" and rows > ell - 1:
        C, deltas, _ = reduce(C, rows)
        sum_delta += sum(deltas)
    return C, sum_delta


@pytest.mark.parametrize("variant", VARS)
@pytest.mark.parametrize("mode", ["buffered", "literal"])
def test_covariance_form_replay(variant, mode):
    rng = np.random.default_rng(11)
    for (n, d, ell) in [(57, 9, 3), (83, 12, 4), (40, 8, 3)]:
        A = rng.standard_normal((n, d)) * np.linspace(2.0, 0.3, d)[None, :]
        B, info = fd_sketch(A, ell, variant, _alpha(variant), mode)
        C, sd = _cov_replay(A, ell, variant, _alpha(variant), mode)
        scale = np.abs(C).max()
        # literal SS reduces at every row and moves mass onto the least
        # well-determined direction, which the d x d eigh resolves only to
        # eps * ||C||: a looser floor there.
        tol = 1e-8 if (variant == "ss" and mode == "literal") else 1e-10
        np.testing.assert_allclose(B.T @ B, C, rtol=0, atol=tol * scale)
        assert abs(info["sum_delta"] - sd) <= 1e-10 * max(1.0, sd)


# --------------------------------------------------------------------------
# Exact recovery when rank(A) <= ell - 1 (delta = sigma_ell^2 = 0)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("variant", VARS)
@pytest.mark.parametrize("mode", ["buffered", "literal"])
def test_exact_recovery_low_rank(variant, mode):
    ell = 6
    # Fast alpha-FD keeps t-1 rows, so exact recovery needs rank <= t-1
    rank = ell - 1 if variant != "fastpfd" else fast_pfd_split(ell, _alpha(variant))[1] - 1
    A = W.low_rank_rows(300, 20, rank=rank)
    B, info = fd_sketch(A, ell, variant, _alpha(variant), mode)
    lam = cov_spectrum(A, B)
    assert max(abs(lam[0]), abs(lam[-1])) <= 1e-10 * info["normA2"]
    assert info["sum_delta"] <= 1e-10 * info["normA2"]


# --------------------------------------------------------------------------
# Properties 1-2 and Lemma 1 (per reduction), Property 3 / Lemma 3
# --------------------------------------------------------------------------
@pytest.mark.parametrize("variant", ["fd", "pfd", "isvd", "fastpfd"])
@pytest.mark.parametrize("mode", ["buffered", "literal"])
def test_properties_1_2(variant, mode):
    A = W.random_noisy(700, 24, m=6, seed=3, dtype=np.float64)
    B, info = fd_sketch(A, 5, variant, _alpha(variant), mode)
    lam = cov_spectrum(A, B)
    tol = 1e-10 * info["normA2"]
    assert lam[0] >= -tol                       # Property 1
    assert lam[-1] <= info["sum_delta"] + tol   # Property 2


@pytest.mark.parametrize("variant", ["fd", "pfd", "isvd", "fastpfd"])
@pytest.mark.parametrize("mode", ["buffered", "literal"])
def test_lemma1_each_reduction(variant, mode):
    A = W.random_noisy(200, 16, m=5, seed=4, dtype=np.float64)
    _, info = fd_sketch(A, 4, variant, _alpha(variant), mode, record=True)
    assert len(info["records"]) > 5
    for r in info["records"]:
        C, Bn, delta = r["C"], r["B"], r["deltas"][0]
        lam = np.linalg.eigvalsh(C.T @ C - Bn.T @ Bn)
        tol = 1e-10 * float(np.sum(C * C))
        assert lam[0] >= -tol
        assert lam[-1] <= delta + tol


def test_lemma3_literal_equality():
    """Literal alpha-FD: ||A||_F^2 - ||B||_F^2 = alpha * ell * Delta exactly."""
    A = W.random_noisy(400, 30, m=8, seed=5, dtype=np.float64)
    for variant, ell, alpha in [("fd", 6, 1.0), ("pfd", 10, 0.4), ("pfd", 5, 0.2)]:
        B, info = fd_sketch(A, ell, variant, alpha, "literal")
        lhs = info["normA2"] - info["normB2"]
        rhs = alpha * ell * info["sum_delta"]
        assert abs(lhs - rhs) <= 1e-10 * info["normA2"], (variant, lhs, rhs)


@pytest.mark.parametrize("variant,alpha", [("fd", 1.0), ("pfd", 0.2), ("pfd", 0.5)])
def test_property3_buffered_accounting(variant, alpha):
    """Buffered: mass removed = ||A||^2 - ||B||^2 >= alpha*ell*Delta; the surplus
    is the mass of the values past ell, which a 2*ell buffer zeroes."""
    ell = 8
    A = W.random_noisy(900, 40, m=10, seed=6, dtype=np.float64)
    B, info = fd_sketch(A, ell, variant, alpha, "buffered", record=True)
    lhs = info["normA2"] - info["normB2"]
    assert abs(lhs - info["removed"]) <= 1e-10 * info["normA2"]
    s = ell - int(math.floor((1 - alpha) * ell + 1e-9))
    assert lhs >= s * info["sum_delta"] * (1 - 1e-12)
    tails = 0.0
    for r in info["records"]:
        tails += float(np.sum(r["sigma"][ell:] ** 2))
    # flush reduction in sketch() is not recorded: rebuild it from the totals
    assert lhs >= s * info["sum_delta"] + tails - 1e-9 * info["normA2"]


# --------------------------------------------------------------------------
# Error bound of the alpha-FD theorem (Sec. 3.1)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("variant,alpha", [("fd", 1.0), ("pfd", 0.5), ("pfd", 0.2)])
@pytest.mark.parametrize("mode", ["buffered", "literal"])
def test_alpha_fd_error_bound(variant, alpha, mode):
    ell = 10
    A = W.random_noisy(1500, 50, m=12, seed=7, dtype=np.float64)
    B, info = fd_sketch(A, ell, variant, alpha, mode)
    lam = cov_spectrum(A, B)
    err = max(abs(lam[0]), abs(lam[-1]))
    s = np.linalg.svd(A, compute_uv=False)
    for k in range(0, int(alpha * ell)):
        if alpha * ell - k <= 0:
            continue
        tail = float(np.sum(s[k:] ** 2))
        assert err <= tail / (alpha * ell - k) * (1 + 1e-10), (k, err, tail)


# --------------------------------------------------------------------------
# SpaceSaving Directions (Theorem, Sec. 3.1)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("mode", ["buffered", "literal"])
def test_ss_mass_preserved(mode):
    A = W.random_noisy(800, 30, m=6, seed=8, dtype=np.float64)
    B, info = fd_sketch(A, 7, "ss", 1.0, mode)
    assert abs(info["normA2"] - info["normB2"]) <= 1e-11 * info["normA2"]


def test_ss_literal_two_sided_bound():
    ell = 12
    A = W.random_noisy(1200, 40, m=5, seed=9, dtype=np.float64)
    B, info = fd_sketch(A, ell, "ss", 1.0, "literal")
    lam = cov_spectrum(A, B)
    err = max(abs(lam[0]), abs(lam[-1]))
    s = np.linalg.svd(A, compute_uv=False)
    for k in range(0, ell // 2):
        den = ell / 2 - 0.5 - k
        if den <= 0:
            continue
        assert err <= float(np.sum(s[k:] ** 2)) / den * (1 + 1e-10)


# --------------------------------------------------------------------------
# Covariance error (Sec. 1.1): closed forms and brute force
# --------------------------------------------------------------------------
def test_cov_err_closed_forms():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((50, 6))
    s = np.linalg.svd(A, compute_uv=False)
    # B = 0: ||A^T A||_2 / ||A||_F^2 = sigma_1^2 / sum sigma^2
    assert abs(cov_err(A, np.zeros((3, 6))) - s[0] ** 2 / np.sum(s ** 2)) < 1e-13
    # B with the same covariance: zero
    q, r = np.linalg.qr(A)
    assert cov_err(A, r) < 1e-13
    # orthogonal rows: the largest missing squared norm wins
    A = np.diag([5.0, 4.0, 3.0, 2.0])
    B = np.diag([5.0, 0.0, 3.0, 0.0])
    assert abs(cov_err(A, B) - 16.0 / 54.0) < 1e-15
    # indefinite difference: B over-estimates one direction
    B = np.diag([5.0, 4.0, 3.0, 2.0]) ; B[0, 0] = 7.0
    assert abs(cov_err(A, B) - (49.0 - 25.0) / 54.0) < 1e-15


def test_cov_err_brute_force_d2():
    """max over unit x of |(||Ax||^2 - ||Bx||^2)| on a fine grid of the circle."""
    rng = np.random.default_rng(2)
    A = rng.standard_normal((30, 2))
    B = rng.standard_normal((3, 2))
    t = np.linspace(0, np.pi, 200001)
    X = np.stack([np.cos(t), np.sin(t)])
    val = np.abs(np.sum((A @ X) ** 2, 0) - np.sum((B @ X) ** 2, 0)).max()
    assert abs(cov_err(A, B) * np.sum(A * A) - val) <= 1e-8 * val


# --------------------------------------------------------------------------
# Stream handling
# --------------------------------------------------------------------------
@pytest.mark.parametrize("variant", VARS)
def test_chunked_append_is_identical(variant):
    A = W.random_noisy(333, 20, m=5, seed=10, dtype=np.float64)
    B0, i0 = fd_sketch(A, 5, variant, _alpha(variant))
    o = FDOracle(20, 5, variant, _alpha(variant))
    for a, b in [(0, 1), (1, 17), (17, 18), (18, 200), (200, 333)]:
        o.append(A[a:b])
    B1, i1 = o.sketch()
    np.testing.assert_array_equal(B0, B1)
    assert i0["sum_delta"] == i1["sum_delta"]


def test_short_stream_returns_rows():
    A = np.arange(12, dtype=float).reshape(3, 4) + 1
    B, info = fd_sketch(A, 5, "fd")
    np.testing.assert_array_equal(B[:3], A)
    assert info["sum_delta"] == 0.0 and info["reductions"] == 0


def test_buffered_cadence():
    ell = 4
    A = W.random_noisy(2 * ell + 3 * (ell + 1), 10, m=3, seed=12, dtype=np.float64)
    o = FDOracle(10, ell, "fd")
    o.append(A)
    assert o.reductions == 4 and o.m == ell - 1


# --------------------------------------------------------------------------
# Sanity (not pins): generators and the paper's qualitative findings
# --------------------------------------------------------------------------
def test_random_noisy_numeric_rank_near_table():
    """Table 5 lists numeric rank 14.93 for Random Noisy (n=10000, d=500, m=30);
    the generator with D from 1 to 0.1 lands close to it."""
    A = W.random_noisy(10000, 500, m=30, seed=0, dtype=np.float64)
    s = np.linalg.svd(A, compute_uv=False)
    nr = float(np.sum(s ** 2) / s[0] ** 2)
    assert 12.0 < nr < 20.0, nr


def test_isvd_fails_on_paper_adversarial():
    """Sec. 5 ("Data adversarial to iSVD"): iSVD keeps discarding the late
    subspace while FD adapts; FD's error falls well below iSVD's."""
    A = W.paper_adversarial(n=3000, d=120, m1=60, m2=4)
    e = {v: cov_err(A, fd_sketch(A, 20, v)[0]) for v in ("fd", "isvd")}
    assert e["fd"] < 0.5 * e["isvd"], e


# ---- merge of two sketches -------------------------------------------------

def _merged(A1, A2, ell, variant="fd", alpha=1.0):
    o1 = FDOracle(A1.shape[1], ell, variant, alpha)
    o2 = FDOracle(A2.shape[1], ell, variant, alpha)
    o1.append(A1)
    o2.append(A2)
    o1.merge(o2)
    return o1


@pytest.mark.parametrize("variant", ["fd", "pfd", "isvd"])
def test_merge_keeps_lemma1_bounds(variant):
    """After a merge, 0 <= x^T (A^T A - B^T B) x <= sum of all deltas for the
    union of both streams (Lemma 1, Sec. 3.1, applied to every reduction of
    both streams), and the counters cover both streams."""
    A1 = W.random_noisy(700, 40, m=6, seed=31)
    A2 = W.random_noisy(450, 40, m=6, seed=32)
    o = _merged(A1, A2, 8, variant, 0.5)
    B, info = o.sketch()
    A = np.vstack([A1, A2]).astype(np.float64)
    lam = cov_spectrum(A, B)
    na2 = float(np.sum(A * A))
    assert abs(info["normA2"] - na2) <= 1e-12 * na2
    assert info["n_seen"] == A.shape[0]
    assert lam[0] >= -1e-10 * na2
    assert lam[-1] <= info["sum_delta"] * (1 + 1e-10) + 1e-10 * na2
    # a merge is not the same as one stream: at least the bound must not be free
    assert info["sum_delta"] > 0.0


def test_merge_exact_when_rank_fits():
    """Rows spanning at most ell-1 dimensions in total: every delta is zero,
    so the merged sketch reproduces A^T A exactly (Sec. 2.3, sigma_ell = 0)."""
    basis = W.low_rank_rows(5, 30, 5, seed=7)
    rng = np.random.default_rng(3)
    A1 = rng.standard_normal((300, 5)) @ basis
    A2 = rng.standard_normal((200, 5)) @ basis
    o = _merged(A1, A2, 8)
    B, info = o.sketch()
    A = np.vstack([A1, A2])
    assert cov_err(A, B) <= 1e-11
    assert info["sum_delta"] <= 1e-9 * info["normA2"]


def test_merge_ss_conserves_mass():
    """SS keeps ||B||_F^2 = ||A||_F^2 (Sec. 3.1) through a merge as well."""
    A1 = W.random_noisy(500, 30, m=5, seed=41)
    A2 = W.random_noisy(333, 30, m=5, seed=42)
    o = _merged(A1, A2, 6, "ss")
    B, info = o.sketch()
    A = np.vstack([A1, A2]).astype(np.float64)
    na2 = float(np.sum(A * A))
    assert abs(float(np.sum(B * B)) - na2) <= 1e-10 * na2


def test_merge_of_empty_sketch_is_identity():
    A1 = W.random_noisy(400, 20, m=4, seed=51)
    o1 = FDOracle(20, 6, "fd")
    o1.append(A1)
    B0, i0 = o1.sketch()
    o1.merge(FDOracle(20, 6, "fd"))
    B1, i1 = o1.sketch()
    np.testing.assert_array_equal(B0, B1)
    assert i1["normA2"] == i0["normA2"] and i1["sum_delta"] == i0["sum_delta"]


# --------------------------------------------------------------------------
# Compensative FD (Sec. 3.1) and proj-err (Sec. 1.1)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("variant", ["fd", "pfd"])
def test_compensative_two_sided_bound(variant):
    """|x^T (A^T A - B-hat^T B-hat) x| <= Delta for every unit x (Sec. 3.1), and
    what is added is Delta times the projector onto B's row space (pinv route,
    independent of the SVD that compensate() takes)."""
    A = W.random_noisy(700, 40, m=8, seed=81, dtype=np.float64)
    o = FDOracle(40, 9, variant, _alpha(variant))
    o.append(A)
    B, _ = o.sketch()
    Bh, info = o.sketch_compensated()
    D = info["sum_delta"]
    assert D > 0
    lam = cov_spectrum(A, Bh)
    assert lam[0] >= -D * (1 + 1e-9) and lam[-1] <= D * (1 + 1e-9), (lam[0], lam[-1], D)
    P = B.T @ np.linalg.pinv(B @ B.T) @ B
    np.testing.assert_allclose(Bh.T @ Bh - B.T @ B, D * P, atol=1e-9 * float(np.sum(B * B)))


def test_compensative_without_reduction_keeps_the_covariance():
    """A stream that never reduced has Delta = 0: B-hat^T B-hat = B^T B."""
    A = W.random_noisy(7, 30, m=4, seed=84, dtype=np.float64)
    o = FDOracle(30, 9, "fd")
    o.append(A)
    B, _ = o.sketch()
    Bh, info = o.sketch_compensated()
    assert info["sum_delta"] == 0.0
    np.testing.assert_allclose(Bh.T @ Bh, B.T @ B, atol=1e-12 * float(np.sum(B * B)))
    with pytest.raises(ValueError):
        FDOracle(30, 9, "isvd").sketch_compensated()


def test_proj_err_closed_forms():
    """proj-err of B = A is 1; brute force against an explicit projector (eigh
    of B^T B) over the tail of A's SVD; never below 1 (Sec. 1.1)."""
    A = W.random_noisy(600, 30, m=12, seed=82, dtype=np.float64)
    assert proj_err(A, A, 5) == pytest.approx(1.0, rel=1e-9)
    rng = np.random.default_rng(85)
    B = rng.standard_normal((7, 30))
    _, Q = np.linalg.eigh(B.T @ B)
    Qk = Q[:, -5:]
    num = float(np.sum((A - A @ Qk @ Qk.T) ** 2))
    sv = np.linalg.svd(A, compute_uv=False)
    den = float(np.sum(sv[5:] ** 2))
    pe = proj_err(A, B, 5)
    assert pe == pytest.approx(num / den, rel=1e-9)
    assert pe >= 1.0 - 1e-12
    # B of rank 2 < k: B_k spans those two directions only
    B2 = B[:2]
    _, Q2 = np.linalg.eigh(B2.T @ B2)
    Q2 = Q2[:, -2:]
    num2 = float(np.sum((A - A @ Q2 @ Q2.T) ** 2))
    assert proj_err(A, B2, 5) == pytest.approx(num2 / den, rel=1e-9)


@pytest.mark.parametrize("variant,alpha", [("fd", 1.0), ("pfd", 0.5)])
def test_proj_err_bounds(variant, alpha):
    """||A - pi_{B_k}(A)||_F^2 <= alpha ell / (alpha ell - k) ||A - A_k||_F^2
    (Sec. 3.1); compensative FD keeps V, so its proj-err is the same and within
    ell / (ell - k)."""
    A = W.random_noisy(900, 50, m=10, seed=83, dtype=np.float64)
    ell, k = 16, 4
    o = FDOracle(50, ell, variant, alpha)
    o.append(A)
    B, _ = o.sketch()
    Bh, _ = o.sketch_compensated()
    pe = proj_err(A, B, k)
    assert 1.0 - 1e-12 <= pe <= alpha * ell / (alpha * ell - k), pe
    peh = proj_err(A, Bh, k)
    assert peh == pytest.approx(pe, rel=1e-9)
    assert peh <= ell / (ell - k)


# --------------------------------------------------------------------------
# Fast alpha-FD (Sec. 3.1) and buffers of c*ell rows
# --------------------------------------------------------------------------
@pytest.mark.parametrize("ell,alpha", [(20, 0.2), (12, 0.5), (10, 1.0)])
@pytest.mark.parametrize("mode", ["buffered", "literal"])
def test_fast_alpha_fd_bounds(ell, alpha, mode):
    """Each reduction removes delta from the values keep .. t (t - keep of
    them, at least alpha*ell/2) and at most delta from any direction, so
    ||A||^2 - ||B||^2 >= (t - keep) Delta, 0 <= x^T (A^T A - B^T B) x <= Delta, and
    Delta <= ||A - A_k||^2 / ((t - keep) - k): the bound the paper states for
    ell = 2(k + 1/eps)/alpha. A reduction leaves t-1 rows."""
    keep, t = fast_pfd_split(ell, alpha)
    assert t - keep >= alpha * ell / 2 - 1e-12
    A = W.random_noisy(1500, 50, m=12, seed=87, dtype=np.float64)
    o = FDOracle(50, ell, "fastpfd", alpha, mode, record=True)
    o.append(A)
    B, info = o.sketch()
    assert info["reductions"] > 10
    for r in o.records:
        assert int(np.sum(r["sigma_prime"] > 0)) <= t - 1
    lhs = info["normA2"] - info["normB2"]
    D = info["sum_delta"]
    assert lhs >= (t - keep) * D * (1 - 1e-12)
    lam = cov_spectrum(A, B)
    tol = 1e-10 * info["normA2"]
    assert lam[0] >= -tol and lam[-1] <= D + tol
    s = np.linalg.svd(A, compute_uv=False)
    for k in range(0, t - keep):
        tail = float(np.sum(s[k:] ** 2))
        assert D <= tail / ((t - keep) - k) * (1 + 1e-10), (k, D, tail)


@pytest.mark.parametrize("variant", ["fd", "pfd", "ss", "isvd"])
def test_larger_buffer(variant):
    """A buffer of 3*ell rows: the same index rules, a reduction every 2*ell+1
    rows; FD's guarantees hold as for 2*ell, and a stream of rank below ell is
    recovered exactly."""
    ell = 6
    A = W.random_noisy(700, 24, m=6, seed=88, dtype=np.float64)
    o = FDOracle(24, ell, variant, _alpha(variant), buffer_rows=3 * ell)
    o.append(A)
    B, info = o.sketch()
    assert info["reductions"] == 1 + (700 - 3 * ell) // (2 * ell + 1) + 1  # + the flush
    lam = cov_spectrum(A, B)
    tol = 1e-10 * info["normA2"]
    if variant != "isvd":
        assert lam[-1] <= info["sum_delta"] + tol
    if variant != "ss":
        assert lam[0] >= -tol
    L = W.low_rank_rows(300, 20, rank=ell - 1)
    o = FDOracle(20, ell, variant, _alpha(variant), buffer_rows=3 * ell)
    o.append(L)
    B, info = o.sketch()
    lam = cov_spectrum(L, B)
    assert max(abs(lam[0]), abs(lam[-1])) <= 1e-10 * info["normA2"]



@pytest.mark.parametrize("ell,alpha", [(20, 0.2), (12, 0.5), (10, 1.0)])
def test_fast_alpha_fd_fixed_cadence_equals_literal(ell, alpha):
    """For generic data a Fast alpha-FD reduction leaves exactly t-1 nonzero
    rows, so keeping t-1 rows per reduction (the buffered form) reduces at the
    same rows as the literal algorithm, where zero rows are free, and gives
    the same sketch."""
    A = W.random_noisy(800, 40, m=10, seed=89, dtype=np.float64)
    Bb, ib = fd_sketch(A, ell, "fastpfd", alpha, "buffered")
    Bl, il = fd_sketch(A, ell, "fastpfd", alpha, "literal")
    assert ib["reductions"] == il["reductions"]
    assert ib["sum_delta"] == pytest.approx(il["sum_delta"], rel=1e-10)
    np.testing.assert_allclose(Bb.T @ Bb, Bl.T @ Bl, rtol=0, atol=1e-9 * ib["normA2"])


@pytest.mark.parametrize("variant,alpha", [("fd", 1.0), ("pfd", 0.25), ("isvd", 1.0), ("ss", 1.0)])
def test_literal_reduces_at_every_row_once_full(variant, alpha):
    """Algorithm 1 as printed (the literal mode): for generic data a reduction
    of the full ell-row sketch frees exactly one row (FD and alpha-FD zero
    sigma_ell only, iSVD drops it, SS merges one pair), so once the sketch is
    full every row triggers a reduction: n - ell + 1 of them, with ell - 1
    nonzero rows after each. A GPU sketch with an ell-row buffer keeping
    ell - 1 rows follows the same cadence."""
    ell, n = 8, 120
    A = W.random_noisy(n, 30, m=5, seed=91, dtype=np.float64)
    o = FDOracle(30, ell, variant, alpha, mode="literal")
    for i in range(n):
        o.append(A[i:i + 1])
        nz = int(np.count_nonzero(np.any(o.buf != 0.0, axis=1)))
        if i + 1 >= ell:
            assert nz == ell - 1, (i, nz)
    assert o.reductions == n - ell + 1


# --------------------------------------------------------------------------
# The oracle's own SVD (one-sided Jacobi) against the textbook SVD and a
# closed form; whole streams through either SVD route agree
# --------------------------------------------------------------------------
@pytest.mark.parametrize("m,d", [(5, 8), (20, 64), (64, 64), (40, 30), (1, 7)])
def test_jacobi_svd_matches_textbook_svd(m, d):
    rng = np.random.default_rng(100 + m + d)
    X = rng.standard_normal((m, d)) * np.logspace(3, 0, m)[:, None]  # graded rows
    sigma, V, sweeps = jacobi_svd_rows(X)
    ref = np.linalg.svd(X, compute_uv=False)
    k = min(m, d)
    np.testing.assert_allclose(sigma[:k], ref, rtol=1e-12, atol=1e-12 * ref[0])
    assert np.all(np.abs(sigma[k:]) <= 1e-12 * ref[0])
    live = sigma > 1e-12 * ref[0]
    Vl = V[live]
    np.testing.assert_allclose(Vl @ Vl.T, np.eye(Vl.shape[0]), atol=1e-13)
    # X^T X = V^T diag(sigma^2) V (the right vectors span the row space)
    np.testing.assert_allclose(Vl.T @ np.diag(sigma[live] ** 2) @ Vl, X.T @ X,
                               atol=1e-12 * ref[0] ** 2)
    assert sweeps < 60


def test_jacobi_svd_closed_form():
    """Rows 3 q_1, 2 q_2, 1 q_3 of orthonormal q, mixed by a rotation: sigma = 3, 2, 1."""
    q, _ = np.linalg.qr(np.random.default_rng(7).standard_normal((6, 3)))
    c, s = math.cos(0.3), math.sin(0.3)
    mix = np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])
    X = mix @ (np.diag([3.0, 2.0, 1.0]) @ q.T)
    sigma, V, _ = jacobi_svd_rows(X)
    np.testing.assert_allclose(sigma, [3.0, 2.0, 1.0], rtol=1e-14)
    np.testing.assert_allclose(np.abs(V @ q), np.eye(3), atol=1e-13)


@pytest.mark.parametrize("variant", ["fd", "pfd", "isvd", "ss"])
def test_stream_through_jacobi_svd_equals_lapack_route(variant):
    A = W.random_noisy(400, 48, m=8, seed=55, dtype=np.float64)
    Bl, il = fd_sketch(A, 6, variant, _alpha(variant))
    Bj, ij = fd_sketch(A, 6, variant, _alpha(variant), svd="jacobi")
    np.testing.assert_allclose(np.linalg.svd(Bj, compute_uv=False),
                               np.linalg.svd(Bl, compute_uv=False), rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(Bj.T @ Bj, Bl.T @ Bl, atol=1e-9 * il["normA2"])
    assert abs(ij["sum_delta"] - il["sum_delta"]) <= 1e-10 * il["normA2"]
