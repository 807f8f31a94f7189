"""FP64 oracle: Frequent Directions with the four ReduceRank rules, step by step.

Test infrastructure only (see ``oracle/__init__.py``): a plain, slow and
deliberately unoptimised replay of the paper's method in float64 with numpy.

What it follows
---------------
* Algorithm 1 (generic FD loop, Sec. 2.3): keep a sketch whose rows are the
  scaled right singular vectors ``S' V^T`` of the rows seen so far; when no
  free (zero) row is left, take ``[U, S, V] = svd(B)``, apply ReduceRank to
  ``S`` and set ``B = S' V^T``. The ``svd`` step is numpy's LAPACK SVD, used as
  a library primitive, or (``svd="jacobi"``) the oracle's own one-sided
  Jacobi SVD of the buffer rows; the two are pinned against each other.
* ReduceRank rules:
    - iSVD (Sec. 2.3): keep ``sigma_j`` for ``j < ell``, zero ``sigma_ell``.
    - FD   (Sec. 2.3): ``sigma'_j = sqrt(sigma_j^2 - delta)``,
      ``delta = sigma_ell^2``; with a buffer larger than ``ell`` (the Fast FD
      form of Sec. 2.3) values below ``delta`` are clipped at zero.
    - alpha-FD / PFD (Algorithm 2, Sec. 3.1): the first ``ell(1-alpha)``
      values are kept, values ``ell(1-alpha)+1 .. ell`` are shrunk by
      ``delta = sigma_ell^2``.
    - SpaceSaving Directions / SS (Algorithm 3, Sec. 3.1): the squared value
      of the second smallest direction is added to the smallest direction and
      the second smallest is freed (``delta = sigma_{ell-1}^2``).
* Two modes:
    - ``"buffered"`` (what the GPU path computes): the working buffer holds
      ``2*ell`` rows; a reduction fires whenever it is full and always leaves
      ``ell-1`` rows (retained directions first, zero rows after them), so a
      reduction happens after the first ``2*ell`` rows and then every
      ``ell+1`` rows. The index rules above are applied with ``ell`` itself
      (``delta`` is the ``ell``-th squared singular value of the ``2*ell``
      rows). PFD zeroes every value past ``ell``; SS repeats Algorithm 3 on
      the spectrum until ``ell-1`` directions remain, freeing zero-mass
      directions first.
    - ``"literal"``: Algorithm 1 as printed, with an ``ell``-row sketch;
      a row is free exactly when it is all zeros.
* ``cov_err`` (Sec. 1.1): ``||A^T A - B^T B||_2 / ||A||_F^2`` with the
  spectral norm taken as the largest absolute eigenvalue of the explicit
  ``d x d`` difference (numpy ``eigvalsh``, a library primitive).
* ``compensate`` (Compensative FD, Sec. 3.1): the final sketch ``S' V^T``
  becomes ``S-hat V^T`` with ``sigma-hat_j = sqrt(sigma'_j^2 + Delta)``.
* ``proj_err`` (Sec. 1.1): ``||A - pi_{B_k}(A)||_F^2 / ||A - A_k||_F^2`` with
  ``B_k`` the top ``k`` right singular vectors of ``B``.

Readings taken where the paper is silent or ambiguous (each is listed in
the design notes): the buffer size and cadence, PFD and SS in a buffer of
``2*ell`` rows, ``ell(1-alpha)`` rounded down, ties broken by slot index,
the final flush in ``sketch()``, and ``max |lambda|`` for an indefinite
difference (SS).
"""
from __future__ import annotations

import math

import numpy as np

VARIANTS = ("fd", "pfd", "ss", "isvd", "fastpfd")


def shrink_index_split(ell: int, alpha: float) -> int:
    """Number of values PFD shrinks: ``s = ell - floor((1 - alpha) * ell)``.

    Algorithm 2 keeps ``sigma_1 .. sigma_{ell(1-alpha)}`` unchanged and shrinks
    the remaining ones up to index ``ell``; ``ell(1-alpha)`` is rounded down
    (so that ``s = ceil(alpha*ell)`` for integral ``alpha*ell``).
    A tiny epsilon guards ``(1-alpha)*ell`` computed as e.g. 39.99999.
    """
    keep = int(math.floor((1.0 - alpha) * ell + 1e-9))
    keep = max(0, min(ell - 1, keep))   # alpha > 0: at least one value shrinks
    return ell - keep


def fast_pfd_split(ell: int, alpha: float):
    """``(keep, t)`` of Fast alpha-FD (Sec. 3.1, "Fast Parameterized FD").

    ``delta = sigma_t^2`` with ``t = ell - ell*alpha/2``; the first
    ``ell(1-alpha)`` values are kept, the others become
    ``sqrt(max(sigma^2 - delta, 0))``, so values ``t .. ell`` become zero.
    ``ell*alpha/2`` is rounded down but taken as at least 1, and
    ``ell(1-alpha)`` is rounded down and capped at ``t-1`` so that at least
    one value before ``t`` is shrunk; a reduction then leaves ``t-1`` rows.
    """
    half = max(1, int(math.floor(alpha * ell / 2.0 + 1e-9)))
    t = ell - half
    keep = int(math.floor((1.0 - alpha) * ell + 1e-9))
    keep = max(0, min(t - 1, keep))
    return keep, t


def reduce_rank(sigma, ell: int, variant: str, alpha: float = 1.0,
                mass_floor: float = 0.0):
    """Apply one ReduceRank step to a descending spectrum.

    ``sigma`` holds the singular values of the rows being reduced, sorted
    descending and padded with zeros to the number of rows. Index ``j`` in the
    paper is ``j - 1`` here. Returns ``(sigma_prime, deltas)`` where
    ``sigma_prime`` is aligned with ``sigma`` (slot ``j`` keeps direction
    ``v_j``) and ``deltas`` lists every delta the step subtracted (one entry,
    or several for SS which repeats Algorithm 3).

    ``mass_floor`` (SS only): squared values at or below it count as empty
    slots and are freed before any merge, so that SS never moves mass onto a
    direction the SVD left undetermined (a numerically zero singular value);
    their total is added to the smallest retained direction at the end (one
    more delta), so that SS keeps ``||B||_F^2 = ||A||_F^2``.
    """
    s = np.asarray(sigma, dtype=np.float64)
    L = s.shape[0]
    sq = s * s
    # sigma_ell (1-based) is sq[ell-1]; it is zero when fewer values exist.
    sig_ell_sq = sq[ell - 1] if L >= ell else 0.0
    if variant == "fd":
        delta = sig_ell_sq
        sp = np.sqrt(np.maximum(sq - delta, 0.0))
        return sp, [delta]
    if variant == "isvd":
        delta = sig_ell_sq
        sp = s.copy()
        sp[ell - 1:] = 0.0
        return sp, [delta]
    if variant == "pfd":
        delta = sig_ell_sq
        nshrink = shrink_index_split(ell, alpha)
        keep = ell - nshrink
        sp = np.zeros_like(s)
        top = min(keep, L)
        sp[:top] = s[:top]
        hi = min(ell, L)
        if hi > keep:
            sp[keep:hi] = np.sqrt(np.maximum(sq[keep:hi] - delta, 0.0))
        return sp, [delta]
    if variant == "fastpfd":
        keep, t = fast_pfd_split(ell, alpha)
        delta = sq[t - 1] if L >= t else 0.0
        sp = np.zeros_like(s)
        top = min(keep, L)
        sp[:top] = s[:top]
        hi = min(ell, L)
        if hi > keep:
            sp[keep:hi] = np.sqrt(np.maximum(sq[keep:hi] - delta, 0.0))
        return sp, [delta]
    if variant == "ss":
        mu = sq.copy()
        alive = [j for j in range(L) if mu[j] > mass_floor]
        freed = float(sum(mu[j] for j in range(L) if not mu[j] > mass_floor))
        deltas = []
        while len(alive) > ell - 1:
            # smallest mass first; among equal masses the larger slot index
            # counts as the smaller one
            alive.sort(key=lambda j: (mu[j], -j))
            q, p = alive[0], alive[1]
            delta = mu[p]
            mu[q] = mu[q] + mu[p]
            mu[p] = 0.0
            alive.remove(p)
            deltas.append(delta)
        if freed > 0.0 and alive:
            # the freed masses go to the smallest retained direction, so that
            # SS keeps the mass of the stream
            q = min(alive, key=lambda j: (mu[j], -j))
            mu[q] = mu[q] + freed
            deltas.append(freed)
        sp = np.zeros_like(s)
        for j in range(L):
            if j not in alive:
                mu[j] = 0.0
        for j in alive:
            sp[j] = math.sqrt(mu[j])
        return sp, deltas
    raise ValueError(f"unknown variant {variant!r}")


def jacobi_svd_rows(X: np.ndarray, tol: float = 1e-15, max_sweeps: int = 60):
    """The oracle's own SVD of the rows of ``X``: one-sided (Hestenes) Jacobi.

    Pairs of rows ``(r_p, r_q)`` are rotated in their plane until every pair
    is orthogonal, ``|<r_p, r_q>| <= tol * ||r_p|| ||r_q||`` (Hestenes 1958).
    A rotation by the angle that zeroes ``<r_p, r_q>``: with
    ``a = ||r_p||^2, b = ||r_q||^2, g = <r_p, r_q>``, ``zeta = (b - a) / (2 g)``,
    ``t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2))``, ``c = 1 / sqrt(1 + t^2)``,
    ``s = c t``: ``r_p <- c r_p - s r_q``, ``r_q <- s r_p + c r_q``. The pairs
    of one sweep are visited in round-robin rounds of disjoint pairs (the
    rows of a round are independent, so a round is one vector operation).
    Then ``sigma_j = ||r_j||`` and ``v_j = r_j / sigma_j``, sorted by sigma
    descending (ties by row index).

    Returns ``(sigma, V, sweeps)``; V has zero rows where sigma is zero.
    """
    R = np.array(X, dtype=np.float64, copy=True)
    m, d = R.shape
    if m == 0:
        return np.zeros(0), np.zeros((0, d)), 0
    mp = m + (m & 1)
    if mp != m:
        R = np.vstack([R, np.zeros((1, d))])
    # rows whose squared norm is at the FP64 resolution of the matrix are
    # numerically zero: rotating them only moves rounding noise around
    zfloor = (max(m, d) * np.finfo(np.float64).eps * np.sqrt(np.sum(R * R))) ** 2
    sweeps = 0
    for sweeps in range(1, max_sweeps + 1):
        rotated = False
        for r in range(mp - 1):
            # round r: position 0 fixed, the others rotate by one place
            idx = [0] + [1 + (k - 1 + r) % (mp - 1) for k in range(1, mp)]
            P = np.array(idx[: mp // 2])
            Q = np.array(idx[mp // 2:][::-1])
            rp, rq = R[P], R[Q]
            a = np.einsum("ij,ij->i", rp, rp)
            b = np.einsum("ij,ij->i", rq, rq)
            g = np.einsum("ij,ij->i", rp, rq)
            act = (np.abs(g) > tol * np.sqrt(a * b)) & (a > zfloor) & (b > zfloor)
            if not np.any(act):
                continue
            rotated = True
            gg = np.where(act, g, 1.0)
            zeta = (b - a) / (2.0 * gg)
            t = np.sign(zeta) / (np.abs(zeta) + np.sqrt(1.0 + zeta * zeta))
            t = np.where(zeta == 0.0, 1.0, t)
            c = 1.0 / np.sqrt(1.0 + t * t)
            sn = c * t
            c = np.where(act, c, 1.0)[:, None]
            sn = np.where(act, sn, 0.0)[:, None]
            R[P], R[Q] = c * rp - sn * rq, sn * rp + c * rq
        if not rotated:
            break
    R = R[:m]
    norms = np.sqrt(np.einsum("ij,ij->i", R, R))
    order = sorted(range(m), key=lambda j: (-norms[j], j))
    sigma = norms[order]
    V = np.zeros((m, d))
    for k, j in enumerate(order):
        if norms[j] > 0.0:
            V[k] = R[j] / norms[j]
    return sigma, V, sweeps


def _svd_rows(X: np.ndarray, method: str = "lapack"):
    """Singular values (descending, padded to the row count) and right vectors.

    Returns ``(sigma, V)`` with ``V`` of shape ``(rows, d)``; rows of ``V``
    past ``min(rows, d)`` are zero (their singular value is zero too).
    ``method``: ``"lapack"`` (numpy's SVD, a library primitive) or
    ``"jacobi"`` (the oracle's own one-sided Jacobi, ``jacobi_svd_rows``).
    """
    m, d = X.shape
    if m == 0:
        return np.zeros(0), np.zeros((0, d))
    if method == "jacobi":
        sigma, V, _ = jacobi_svd_rows(X)
        return sigma, V
    _, s, vt = np.linalg.svd(X, full_matrices=False)
    k = s.shape[0]
    sigma = np.zeros(m)
    sigma[:k] = s
    V = np.zeros((m, d))
    V[:k] = vt
    return sigma, V


class FDOracle:
    """Stateful FP64 replay of the FD family over a row stream.

    ``mode="buffered"``: 2*ell-row buffer, fixed cadence (the GPU contract).
    ``mode="literal"``: Algorithm 1 exactly, ell-row sketch, zero rows free.
    ``record=True`` keeps, per reduction, the rows before (``C``), the
    spectrum, the new spectrum and the deltas, for the per-step lemma checks.
    """

    def __init__(self, d: int, ell: int, variant: str = "fd", alpha: float = 1.0,
                 mode: str = "buffered", record: bool = False, buffer_rows: int | None = None,
                 svd: str = "lapack"):
        if variant not in VARIANTS:
            raise ValueError(variant)
        if ell < 2 or d < 1:
            raise ValueError("need ell >= 2 and d >= 1")
        if variant in ("pfd", "fastpfd") and not (0.0 < alpha <= 1.0):
            raise ValueError("alpha must lie in (0, 1]")
        if mode not in ("buffered", "literal"):
            raise ValueError(mode)
        if svd not in ("lapack", "jacobi"):
            raise ValueError(svd)
        self.svd = svd
        self.d, self.ell, self.variant, self.mode = d, ell, variant, mode
        self.alpha = alpha if variant in ("pfd", "fastpfd") else 1.0
        if variant == "fastpfd":
            # the sketch is its own buffer (ell rows); a reduction leaves t-1 rows
            _, t = fast_pfd_split(ell, self.alpha)
            if t < 2:
                raise ValueError("Fast alpha-FD needs ell - ell*alpha/2 >= 2")
            if buffer_rows not in (None, ell):
                raise ValueError("Fast alpha-FD uses an ell-row buffer")
            self.cap, self.keep_rows = ell, t - 1
        else:
            # buffered FD: a buffer of c*ell rows (c >= 2; Fast FD of Sec. 2.3
            # with delta = sigma_ell^2) that always leaves ell-1 rows
            cap = 2 * ell if buffer_rows is None else int(buffer_rows)
            if mode == "buffered" and cap < 2 * ell:
                raise ValueError("the buffer holds at least 2*ell rows")
            self.cap, self.keep_rows = (cap if mode == "buffered" else ell), ell - 1
        self.buf = np.zeros((self.cap, d))
        self.m = 0                     # buffered: filled rows (zero rows included)
        self.normA2 = 0.0
        self.sum_delta = 0.0
        self.last_delta = 0.0
        self.removed = 0.0             # sum over reductions of sum_j (sigma^2 - sigma'^2)
        self.n_seen = 0
        self.reductions = 0
        self.record = record
        self.records = []

    # -- Algorithm 1, one reduction ------------------------------------
    def _reduce(self, X: np.ndarray, commit: bool):
        """SVD of the rows ``X``, ReduceRank, and the new rows ``S' V^T``.

        Returns ``(new_rows, deltas, removed)`` where ``new_rows`` lists the
        retained rows ``sigma'_j v_j`` ordered by ``sigma'`` descending
        (stable in the slot index).
        """
        sigma, V = _svd_rows(X, self.svd)
        # numerical-rank floor of the FP64 SVD (largest value x size x eps),
        # squared: masses at or below it are treated as exactly zero (SS)
        floor = (sigma[0] * max(X.shape) * np.finfo(np.float64).eps) ** 2 if sigma.size else 0.0
        sp, deltas = reduce_rank(sigma, self.ell, self.variant, self.alpha, floor)
        order = sorted((j for j in range(sp.shape[0]) if sp[j] > 0.0),
                       key=lambda j: (-sp[j], j))
        new_rows = np.array([sp[j] * V[j] for j in order]).reshape(len(order), self.d)
        removed = float(np.sum(sigma * sigma) - np.sum(sp * sp))
        if commit and self.record:
            self.records.append(dict(C=X.copy(), sigma=sigma, sigma_prime=sp,
                                     deltas=list(deltas), B=new_rows.copy()))
        return new_rows, deltas, removed

    def _commit(self, deltas, removed):
        self.reductions += 1
        self.sum_delta += float(sum(deltas))
        if deltas:
            self.last_delta = float(deltas[-1])
        self.removed += removed

    def append(self, rows):
        rows = np.asarray(rows)
        if rows.ndim == 1:
            rows = rows[None, :]
        if rows.shape[1] != self.d:
            raise ValueError("row width differs from d")
        rows = rows.astype(np.float64)   # exact widening from f32 / bf16-as-f32 / f64
        if self.mode == "literal":
            for a in rows:
                self._append_literal(a)
            return
        i, n = 0, rows.shape[0]
        while i < n:
            c = min(n - i, self.cap - self.m)
            chunk = rows[i:i + c]
            self.buf[self.m:self.m + c] = chunk
            for r in chunk:             # ||A||_F^2 summed in stream order
                self.normA2 += float(np.dot(r, r))
            self.m += c
            self.n_seen += c
            i += c
            if self.m == self.cap:
                new_rows, deltas, removed = self._reduce(self.buf[:self.m], True)
                self._commit(deltas, removed)
                self.buf[:] = 0.0
                self.buf[:new_rows.shape[0]] = new_rows
                self.m = self.keep_rows

    def _append_literal(self, a):
        self.normA2 += float(np.dot(a, a))
        self.n_seen += 1
        free = [r for r in range(self.cap) if not np.any(self.buf[r] != 0.0)]
        if not free:
            raise AssertionError("literal sketch has no free row")  # cannot happen
        self.buf[free[0]] = a
        if len(free) == 1:              # no zero-valued row left: reduce
            new_rows, deltas, removed = self._reduce(self.buf.copy(), True)
            self._commit(deltas, removed)
            self.buf[:] = 0.0
            self.buf[:new_rows.shape[0]] = new_rows

    def sketch(self):
        """Return ``(B, info)`` with ``B`` of shape ``(ell, d)``; non-destructive.

        Buffered mode flushes pending rows with one more reduction when more
        than ``ell-1`` rows are held (same index rules); literal mode returns
        the sketch as it stands (its last free row is zero).
        """
        info = dict(normA2=self.normA2, n_seen=self.n_seen)
        sum_delta, last_delta, removed, reductions = (
            self.sum_delta, self.last_delta, self.removed, self.reductions)
        B = np.zeros((self.ell, self.d))
        if self.mode == "literal":
            nz = [r for r in range(self.cap) if np.any(self.buf[r] != 0.0)]
            B[:len(nz)] = self.buf[nz]
        elif self.m > self.ell - 1:
            new_rows, deltas, rem = self._reduce(self.buf[:self.m].copy(), False)
            B[:new_rows.shape[0]] = new_rows
            sum_delta += float(sum(deltas))
            if deltas:
                last_delta = float(deltas[-1])
            removed += rem
            reductions += 1
        else:
            B[:self.m] = self.buf[:self.m]
        info.update(sum_delta=sum_delta, last_delta=last_delta, removed=removed,
                    reductions=reductions, normB2=float(np.sum(B * B)))
        return B, info


    def sketch_compensated(self):
        """Compensative FD (Sec. 3.1): ``(compensate(B, Delta), info)`` for the
        sketch ``B`` of ``sketch()`` and ``Delta = info["sum_delta"]`` (every
        delta subtracted, the final flush included). FD and PFD only: their
        sketches keep ``0 <= x^T (A^T A - B^T B) x <= Delta``."""
        if self.variant not in ("fd", "pfd"):
            raise ValueError("compensative FD is defined on FD and PFD sketches")
        B, info = self.sketch()
        return compensate(B, info["sum_delta"]), info

    def merge(self, other: "FDOracle"):
        """Fold ``other``'s stream into this sketch (merge of two sketches).

        The paper states the problem for streams that may be distributed
        (Sec. 1); a merge takes ``other``'s sketch (``other.sketch()``,
        non-destructive) and appends its rows to this stream, so that every
        later reduction treats them as ordinary rows. By the per-step bound
        of Lemma 1 (Sec. 3.1), applied to this stream and to ``other``'s,
        the result keeps 0 <= x^T (A^T A - B^T B) x <= (sum of all deltas)
        for the union of both streams. The counters carry ``other``'s:
        ``normA2`` counts ``other``'s rows instead of the appended sketch
        rows; ``other``'s deltas, removed mass, reductions and row count are
        added. Only the retained (nonzero) rows are appended: they come
        first in the sketch, and zero rows carry no mass but would take
        buffer slots.
        """
        if other.d != self.d:
            raise ValueError("row width differs")
        if other is self:
            raise ValueError("cannot merge a sketch into itself")
        B, info = other.sketch()
        nz = np.flatnonzero(np.any(B != 0.0, axis=1))
        rows = B[: (int(nz[-1]) + 1 if nz.size else 0)]
        na2, ns = self.normA2, self.n_seen
        self.append(rows)
        self.normA2 = na2 + info["normA2"]
        self.n_seen = ns + info["n_seen"]
        self.sum_delta += info["sum_delta"]
        self.removed += info["removed"]
        self.reductions += info["reductions"]


def fd_sketch(A, ell: int, variant: str = "fd", alpha: float = 1.0,
              mode: str = "buffered", record: bool = False, buffer_rows: int | None = None,
              svd: str = "lapack"):
    """Run the whole stream ``A`` (rows in order) and return ``(B, info)``.

    With ``record=True`` the per-reduction records are in ``info["records"]``.
    """
    A = np.asarray(A)
    o = FDOracle(A.shape[1], ell, variant, alpha, mode, record, buffer_rows, svd)
    o.append(A)
    B, info = o.sketch()
    if record:
        info["records"] = o.records
    return B, info


def _gram64(A, chunk: int = 8192):
    """``A^T A`` in float64, accumulated over row chunks."""
    A = np.asarray(A)
    d = A.shape[1]
    G = np.zeros((d, d))
    for i in range(0, A.shape[0], chunk):
        blk = A[i:i + chunk].astype(np.float64)
        G += blk.T @ blk
    return G


def cov_spectrum(A, B):
    """Eigenvalues (ascending) of ``A^T A - B^T B`` formed explicitly in FP64."""
    B = np.asarray(B, dtype=np.float64)
    M = _gram64(A) - B.T @ B
    return np.linalg.eigvalsh(0.5 * (M + M.T))


def cov_err(A, B, normA2: float | None = None) -> float:
    """``||A^T A - B^T B||_2 / ||A||_F^2`` (Sec. 1.1), spectral norm as max |lambda|."""
    lam = cov_spectrum(A, B)
    if normA2 is None:
        A64 = np.asarray(A)
        normA2 = 0.0
        for i in range(0, A64.shape[0], 8192):
            blk = A64[i:i + 8192].astype(np.float64)
            normA2 += float(np.sum(blk * blk))
    if normA2 == 0.0:
        return 0.0
    return float(max(abs(lam[0]), abs(lam[-1])) / normA2)


def _rank_floor(sigma, shape) -> float:
    """Numerical-rank floor of an FP64 SVD: largest value x size x eps."""
    return sigma[0] * max(shape) * np.finfo(np.float64).eps if sigma.size else 0.0


def compensate(B, sum_delta: float) -> np.ndarray:
    """Compensative FD (Sec. 3.1): write ``B = S' V^T`` (SVD) and return
    ``S-hat V^T`` with ``sigma-hat_j = sqrt(sigma'_j^2 + Delta)``.

    Reading: only the nonzero singular values (above the FP64 rank floor) are
    compensated. A zero singular value has no direction in ``B``, so the rows
    past the rank stay zero. Rows come out by ``sigma'`` descending.
    """
    B = np.asarray(B, dtype=np.float64)
    sigma, V = _svd_rows(B)
    r = int(np.sum(sigma > _rank_floor(sigma, B.shape)))
    out = np.zeros_like(B)
    out[:r] = np.sqrt(sigma[:r] ** 2 + float(sum_delta))[:, None] * V[:r]
    return out


def proj_err(A, B, k: int = 10) -> float:
    """proj-err (Sec. 1.1): ``||A - pi_{B_k}(A)||_F^2 / ||A - A_k||_F^2``.

    ``B_k`` spans the top ``k`` right singular vectors of ``B`` (fewer when
    ``B`` has rank below ``k``). The numerator sums, over row chunks of ``A``,
    the squared residual of each row after projection onto ``B_k``; the
    denominator is the sum of all but the ``k`` largest eigenvalues of
    ``A^T A`` (numpy ``eigvalsh``), i.e. ``||A - A_k||_F^2``. Returns 1.0
    when both are zero (``A`` of rank at most ``k``, captured exactly).
    """
    B = np.asarray(B, dtype=np.float64)
    sigma, V = _svd_rows(B)
    r = min(k, int(np.sum(sigma > _rank_floor(sigma, B.shape))))
    Vk = V[:r]
    A = np.asarray(A)
    num = 0.0
    for i in range(0, A.shape[0], 8192):
        X = A[i:i + 8192].astype(np.float64)
        R = X - (X @ Vk.T) @ Vk
        num += float(np.sum(R * R))
    lam = np.linalg.eigvalsh(_gram64(A))  # ascending
    den = float(np.sum(lam[:max(lam.shape[0] - k, 0)]))
    if den <= 0.0:
        return 1.0 if num <= 0.0 else math.inf
    return num / den
