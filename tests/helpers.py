"""Shared assertions for the parity tests (GPU result vs FP64 oracle)."""
import numpy as np

# Tolerances: sketch singular values within 1e-4 relative and cov-err within
# 1e-5 absolute of the FP64 oracle. "Relative" is read per value for every
# sigma_j with sigma_j^2 >= 1e-6 ||A||_F^2; smaller values (shrunk to near
# zero, where a relative bound is meaningless) are held to the same bound
# taken at that threshold: |d sigma_j| <= 1e-4 * sqrt(1e-6 ||A||_F^2).
SIG_REL = 1e-4
SIG_FLOOR = 1e-6
COV_ABS = 1e-5


def sigmas(B):
    return np.linalg.svd(np.asarray(B, dtype=np.float64), compute_uv=False)


def small_value_floor(norm_a2, sigma1, buffer_rows=0, eps=0.0):
    """sigma^2 below which a value counts as small: 1e-6 ||A||_F^2, raised to
    the absolute resolution of the eigensolve's arithmetic (rows x eps x
    sigma_1^2: a Gram eigensolve in precision eps resolves eigenvalues only
    to about that, however it is done)."""
    return max(SIG_FLOOR * norm_a2, buffer_rows * eps * sigma1 ** 2)


def sigma_errors(s_gpu, s_orc, norm_a2, buffer_rows=0, eps=0.0):
    k = min(len(s_gpu), len(s_orc))
    s_gpu = np.asarray(s_gpu[:k], dtype=np.float64)
    s_orc = np.asarray(s_orc[:k], dtype=np.float64)
    thr = np.sqrt(small_value_floor(norm_a2, s_orc[0] if k else 0.0, buffer_rows, eps))
    big = s_orc >= thr
    d = np.abs(s_gpu - s_orc)
    rel = np.where(big, d / np.maximum(s_orc, 1e-300), 0.0)
    small_abs = np.where(~big, d, 0.0)
    return float(rel.max(initial=0.0)), float(small_abs.max(initial=0.0) / thr)


EPS32 = 2.0 ** -23


def sigma_parity_excess(s_gpu, s_orc, norm_a2, prec=None):
    """Largest err_j / allowed_j over the sketch spectrum, and its index j.

    allowed_j = 1e-4 * max(s_j, s0) with s0^2 = 1e-6 ||A||_F^2: every value at
    or above the floor within 1e-4 relative, the values below it within the
    same bound taken at the floor. ``prec`` is accepted for the callers'
    messages only: the bar is the same for every arithmetic.
    """
    k = min(len(s_gpu), len(s_orc))
    a = np.asarray(s_gpu[:k], dtype=np.float64)
    b = np.asarray(s_orc[:k], dtype=np.float64)
    if k == 0:
        return 0.0, 0
    s0 = np.sqrt(SIG_FLOOR * norm_a2)
    allowed = SIG_REL * np.maximum(b, s0)
    ratio = np.abs(a - b) / allowed
    j = int(np.argmax(ratio))
    return float(ratio[j]), j


def assert_sigma_parity(B_gpu, B_orc, norm_a2, prec, ell=None, what=""):
    sg, so = sigmas(B_gpu), sigmas(B_orc)
    x, j = sigma_parity_excess(sg, so, norm_a2, prec)
    rel, _ = sigma_errors(sg, so, norm_a2)
    assert x <= 1.0, (f"{what}: sigma_{j} = {so[j]:.6g} (sigma_1 {so[0]:.6g}) off by "
                      f"{abs(sg[j] - so[j]):.3g}, {x:.2f}x the allowance; max rel err "
                      f"above the 1e-6 floor {rel:.2e}")
    return x, rel


def assert_sigma_close(B_gpu, B_orc, norm_a2, rel=SIG_REL, what="", buffer_rows=0, eps=0.0):
    r, s = sigma_errors(sigmas(B_gpu), sigmas(B_orc), norm_a2, buffer_rows, eps)
    assert r <= rel and s <= rel, f"{what}: sigma rel err {r:.3e}, small-value err {s:.3e} (tol {rel})"
    return r, s
