"""Seeded synthetic row streams shaped like the paper's workloads.

This module only draws inputs; it holds none of the sketching arithmetic and
is shared, as the one common piece, by the GPU path's tests and benchmarks and
by the FP64 oracle's tests.

Generators
----------
* ``random_noisy``: the paper's *Random Noisy* matrix (Sec. 4, "Datasets"):
  ``A = S D U + F / zeta`` with ``S`` (n x m) and ``F`` (n x d) i.i.d. N(0,1),
  ``D = diag`` decreasing linearly from 1 to 0.1 over the ``m`` signal
  dimensions, ``U`` (m x d) with orthonormal rows (QR of a Gaussian matrix),
  ``zeta = 10``. Rows are drawn in fixed-size chunks, each from its own seeded
  stream, so any row range can be regenerated without the rest.
* ``two_subspace_stream``: a stream that is adversarial for iSVD: blocks of
  rows alternate between two orthogonal 20-dimensional subspaces; rows of the
  first have norm 10, rows of the second norm 1 plus a fixed component of norm
  0.5 along a direction orthogonal to both subspaces plus small i.i.d. noise
  (variance 1e-3).
* ``paper_adversarial``: the construction of Sec. 4 ("Adversarial"): unit rows
  from a 400-dimensional subspace, then unit rows from an orthogonal
  4-dimensional subspace.
* ``sparse_nonneg_rows``: sparse non-negative rows (2% density, U(0,1) values,
  row norm lognormal(0,1)) like a sparse recommendation matrix.
* ``batch_specs``: per-sketch (d, ell, n, seed) draws for many independent
  streams.
"""
from __future__ import annotations

import numpy as np

CHUNK_ROWS = 4096


def _rng(*key: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(np.random.SeedSequence(list(key))))


def orthonormal_rows(m: int, d: int, seed: int, tag: int = 1) -> np.ndarray:
    """An (m x d) matrix with orthonormal rows from the QR of a Gaussian d x m."""
    g = _rng(seed, tag, 0xC0FFEE).standard_normal((d, m))
    q, r = np.linalg.qr(g)
    q = q * np.sign(np.diag(r))[None, :]
    return np.ascontiguousarray(q.T)


def random_noisy(n: int, d: int, m: int = 30, zeta: float = 10.0, seed: int = 0,
                 dtype=np.float32, row_start: int = 0, row_stop: int | None = None,
                 d_hi: float = 1.0, d_lo: float = 0.1) -> np.ndarray:
    """Rows ``[row_start, row_stop)`` of the Random Noisy matrix, rounded to ``dtype``.

    ``dtype`` may be numpy float64/float32 or the string ``"bf16"`` (returns
    float32 values that are exactly representable in bfloat16, rounded to
    nearest even).
    """
    if row_stop is None:
        row_stop = n
    U = orthonormal_rows(m, d, seed)
    Dg = np.linspace(d_hi, d_lo, m) if m > 1 else np.array([d_hi])
    DU = Dg[:, None] * U
    out_dtype = np.float32 if dtype == "bf16" else dtype
    out = np.empty((row_stop - row_start, d), dtype=out_dtype)
    c0 = row_start // CHUNK_ROWS
    c1 = (row_stop + CHUNK_ROWS - 1) // CHUNK_ROWS
    for c in range(c0, c1):
        rows0 = c * CHUNK_ROWS
        cnt = min(CHUNK_ROWS, n - rows0)
        rng = _rng(seed, 2, c)
        S = rng.standard_normal((cnt, m))
        F = rng.standard_normal((cnt, d))
        blk = S @ DU + F / zeta
        lo = max(row_start, rows0)
        hi = min(row_stop, rows0 + cnt)
        part = blk[lo - rows0:hi - rows0]
        if dtype == "bf16":
            part = round_bf16(part)
        out[lo - row_start:hi - row_start] = part
    return out


def round_bf16(x: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even); returned as float32."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).reshape(f.shape)


def two_subspace_stream(n: int = 100_000, d: int = 1000, block: int = 2000,
                        dim: int = 20, seed: int = 2, dtype=np.float32) -> np.ndarray:
    """Alternating blocks from two orthogonal subspaces (first block: subspace 1)."""
    g = _rng(seed, 7).standard_normal((d, 2 * dim + 1))
    q, _ = np.linalg.qr(g)
    S1, S2, w = q[:, :dim], q[:, dim:2 * dim], q[:, 2 * dim]
    out = np.empty((n, d), dtype=dtype)
    nblocks = (n + block - 1) // block
    for b in range(nblocks):
        r0, r1 = b * block, min(n, (b + 1) * block)
        rng = _rng(seed, 8, b)
        coef = rng.standard_normal((r1 - r0, dim))
        if b % 2 == 0:
            rows = coef @ S1.T
            rows *= (10.0 / np.linalg.norm(rows, axis=1))[:, None]
        else:
            rows = coef @ S2.T
            rows *= (1.0 / np.linalg.norm(rows, axis=1))[:, None]
            rows += 0.5 * w[None, :]
            rows += rng.standard_normal((r1 - r0, d)) * np.sqrt(1e-3)
        out[r0:r1] = rows
    return out


def paper_adversarial(n: int = 10_000, d: int = 500, m1: int = 400, m2: int = 4,
                      seed: int = 5, dtype=np.float64) -> np.ndarray:
    """Unit rows from an m1-dim subspace, then unit rows from an orthogonal m2-dim one."""
    rng = _rng(seed, 9)
    q, _ = np.linalg.qr(rng.standard_normal((d, m1 + m2)))
    P1, P2 = q[:, :m1], q[:, m1:]
    n1 = n // 2
    Y = rng.standard_normal((n1, d)) @ P1 @ P1.T
    Z = rng.standard_normal((n - n1, d)) @ P2 @ P2.T
    A = np.vstack([Y, Z])
    A /= np.linalg.norm(A, axis=1)[:, None]
    return A.astype(dtype)


def sparse_nonneg_rows(n: int, d: int = 512, density: float = 0.02, seed: int = 4,
                       stream: int = 0) -> np.ndarray:
    """Sparse non-negative rows, values U(0,1), each row scaled to a lognormal norm."""
    rng = _rng(seed, 11, stream)
    mask = rng.random((n, d)) < density
    vals = rng.random((n, d)) * mask
    norms = np.linalg.norm(vals, axis=1)
    target = np.exp(rng.standard_normal(n))
    scale = np.divide(target, norms, out=np.zeros_like(norms), where=norms > 0)
    return (vals * scale[:, None]).astype(np.float32)


def batch_specs(count: int = 4096, seed: int = 3, d_range=(64, 1024),
                ell_range=(16, 64), n_range=(1000, 50_000)):
    """Per-sketch (d, ell, n, seed) for a batch of independent streams."""
    rng = _rng(seed, 13)
    d = rng.integers(d_range[0], d_range[1] + 1, size=count)
    ell = rng.integers(ell_range[0], ell_range[1] + 1, size=count)
    n = rng.integers(n_range[0], n_range[1] + 1, size=count)
    seeds = rng.integers(0, 2**31 - 1, size=count)
    return [dict(d=int(d[i]), ell=int(ell[i]), n=int(n[i]), seed=int(seeds[i]))
            for i in range(count)]


def low_rank_rows(n: int, d: int, rank: int, seed: int = 6, dtype=np.float64) -> np.ndarray:
    """Rows spanning exactly ``rank`` dimensions (for exact-recovery checks)."""
    rng = _rng(seed, 17)
    return (rng.standard_normal((n, rank)) @ rng.standard_normal((rank, d))).astype(dtype)


def random_noisy_device(n: int, d: int, m: int, seed: int, zeta: float = 10.0,
                        device="cuda", dtype=None, out=None):
    """Random Noisy rows generated on a CUDA device with PyTorch's generator
    (for streams too large to draw on the host); same recipe as
    ``random_noisy``: A = S D U + F / zeta, D from 1 to 0.1, U orthonormal
    rows. Rounded to ``dtype`` (default bfloat16). Returns an (n, d) tensor."""
    import torch
    dtype = torch.bfloat16 if dtype is None else dtype
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    # the d x m orthonormal factor is small: QR on the host (no device
    # linear-algebra library needed), Gaussian drawn from the device stream
    gauss = torch.randn(d, m, generator=g, device=device, dtype=torch.float32).cpu().double()
    q, r = torch.linalg.qr(gauss)
    q = (q * torch.sign(torch.diagonal(r))[None, :]).float().to(device)
    Dg = torch.linspace(1.0, 0.1, m, device=device) if m > 1 else torch.ones(1, device=device)
    DU = Dg[:, None] * q.T
    if out is None:
        out = torch.empty(n, d, device=device, dtype=dtype)
    step = 1 << 14
    for r0 in range(0, n, step):
        r1 = min(n, r0 + step)
        S = torch.randn(r1 - r0, m, generator=g, device=device, dtype=torch.float32)
        F = torch.randn(r1 - r0, d, generator=g, device=device, dtype=torch.float32)
        out[r0:r1] = (S @ DU + F / zeta).to(dtype)
    return out


def batch_streams_device(specs, device="cuda", dtype=None):
    """All streams of a batch in one device buffer: returns (flat tensor,
    list of (offset_elements, n, d)). Stream i follows ``random_noisy_device``
    with m = ell_i // 2 (at least 1) and seed specs[i]["seed"]."""
    import torch
    dtype = torch.bfloat16 if dtype is None else dtype
    sizes = [sp["n"] * sp["d"] for sp in specs]
    total = int(sum(sizes))
    flat = torch.empty(total, device=device, dtype=dtype)
    views = []
    off = 0
    for sp, sz in zip(specs, sizes):
        v = flat[off:off + sz].view(sp["n"], sp["d"])
        random_noisy_device(sp["n"], sp["d"], max(1, sp["ell"] // 2), sp["seed"], device=device,
                            dtype=dtype, out=v)
        views.append((off, sp["n"], sp["d"]))
        off += sz
    return flat, views
