"""ctypes binding of libfdsketch (C ABI in include/fdsketch.h).

Argument marshalling only: every step of the sketch update runs in the CUDA
kernels of the library. Tensors on a CUDA device are passed as device
pointers on PyTorch's current stream; numpy arrays and CPU tensors are passed
as host pointers (the library stages them through pinned memory). The library
is loaded on first use; if it has not been built, the call raises.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libfdsketch.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "fdsketch.h")

VARIANT = {"fd": 0, "pfd": 1, "ss": 2, "isvd": 3, "fastpfd": 4}
PREC = {"fp32": 0, "bf16x3": 1, "fp64": 2}
F32, BF16, F64 = 0, 1, 2
ERR = {0: "FD_OK", -1: "FD_EINVAL", -2: "FD_ENOMEM", -3: "FD_ECUDA", -4: "FD_ENOCONV",
       -5: "FD_EBUSY", -6: "FD_ETOOBIG"}

_lib = None


class FDError(RuntimeError):
    def __init__(self, code: int, where: str, text: str):
        super().__init__(f"{where}: {ERR.get(code, code)} ({text})")
        self.code = code


class Stats(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int64), ("ell", ctypes.c_int32), ("variant", ctypes.c_int32),
                ("alpha", ctypes.c_double), ("prec", ctypes.c_int32), ("pending", ctypes.c_int32),
                ("n_seen", ctypes.c_int64), ("reductions", ctypes.c_int64),
                ("noconv", ctypes.c_int64), ("norm_a2", ctypes.c_double),
                ("sum_delta", ctypes.c_double), ("last_delta", ctypes.c_double),
                ("removed", ctypes.c_double), ("max_sweeps", ctypes.c_double),
                ("sketch_sum_delta", ctypes.c_double), ("sketch_removed", ctypes.c_double),
                ("sketch_norm_b2", ctypes.c_double), ("eig_fallbacks", ctypes.c_int64)]


class Work(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int32), ("dtype", ctypes.c_int32), ("rows", ctypes.c_void_p),
                ("n", ctypes.c_int64), ("ld", ctypes.c_int64)]


def load():
    """Load libfdsketch.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built; run "
                           "`python -m paper_1501_06561_gb300.build` (nvcc, sm_103a)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "fd_create": [i64, i32, i32, dbl, i32, vp, ctypes.POINTER(vp)],
        "fd_create_buffered": [i64, i32, i32, dbl, i32, i32, vp, ctypes.POINTER(vp)],
        "fd_append": [vp, vp, i64, i64, i32, i32],
        "fd_sketch": [vp, vp, i32, i32],
        "fd_record_spectrum": [vp, i32],
        "fd_sketch_compensated": [vp, vp, i32, i32],
        "fd_merge": [vp, vp],
        "fd_merge_sketch": [vp, vp, i64, i64, i32, i32, ctypes.POINTER(Stats)],
        "fd_cov_err": [vp, vp, i64, i64, i32, i32, ctypes.POINTER(dbl)],
        "fd_proj_err": [vp, vp, i64, i64, i32, i32, i32, ctypes.POINTER(dbl)],
        "fd_cov_err_pair": [vp, i64, i64, i64, i32, vp, i64, i32, i32, vp,
                            ctypes.POINTER(dbl), ctypes.POINTER(dbl), ctypes.POINTER(dbl)],
        "fd_stats": [vp, ctypes.POINTER(Stats)],
        "fd_last_spectrum": [vp, ctypes.POINTER(dbl), ctypes.POINTER(dbl)],
        "fd_destroy": [vp],
        "fd_reset": [vp],
        "fd_profile": [vp, i32],
        "fd_kernel_times": [vp, ctypes.POINTER(i64), ctypes.POINTER(dbl)],
        "fd_strerror": [i32],
        "fd_batch_create": [i32, ctypes.POINTER(i64), ctypes.POINTER(i32), i32, dbl, i32, vp,
                            ctypes.POINTER(vp)],
        "fd_batch_append": [vp, ctypes.POINTER(Work), i32],
        "fd_batch_sketch": [vp, i32, vp, i32, i32],
        "fd_batch_stats": [vp, i32, ctypes.POINTER(Stats)],
        "fd_batch_sketch_all": [vp, vp, ctypes.POINTER(i64)],
        "fd_batch_reset": [vp],
        "fd_batch_uses_graph": [vp, ctypes.POINTER(i64)],
        "fd_cov_err_noalloc": [vp, i64, i64, i64, i32, vp, i64, i32, vp, ctypes.POINTER(dbl)],
        "fd_serve_create": [i32, i64, i32, i32, dbl, i64, i32, ctypes.POINTER(vp)],
        "fd_serve_submit": [vp, i32, vp, i64, ctypes.POINTER(i64)],
        "fd_serve_poll": [vp, ctypes.POINTER(i64), ctypes.POINTER(dbl), i32, ctypes.POINTER(i32)],
        "fd_serve_drain": [vp],
        "fd_serve_sketch": [vp, i32, vp, i32],
        "fd_serve_counters": [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64),
                              ctypes.POINTER(i64)],
        "fd_serve_destroy": [vp],
        "fd_batch_destroy": [vp],
        "fd_version": [],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_char_p if name in ("fd_strerror", "fd_version") else ctypes.c_int
    _lib = lib
    return lib


def header_functions(path: str = HEADER):
    """Names of the functions include/fdsketch.h declares."""
    txt = open(path).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(fd_\w+)\s*\(", txt)))


def _check(code: int, where: str):
    if code != 0:
        lib = load()
        raise FDError(code, where, lib.fd_strerror(code).decode())


def _stream_ptr(stream):
    if stream is not None:
        # a torch.cuda.Stream (or anything with a cuda_stream handle), or a raw handle
        return ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:  # pragma: no cover
        pass
    return ctypes.c_void_p(0)


def _as_rows(x):
    """(pointer, n, ld, dtype code, on_device, keepalive) for a 2-D array/tensor."""
    try:
        import torch
    except Exception:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(x, torch.Tensor):
        if x.dim() == 1:
            x = x.unsqueeze(0)
        if x.stride(1) != 1:
            x = x.contiguous()
        code = {torch.float32: F32, torch.bfloat16: BF16, torch.float64: F64}.get(x.dtype)
        if code is None:
            raise TypeError(f"unsupported dtype {x.dtype}")
        return (ctypes.c_void_p(x.data_ptr()), x.shape[0], x.stride(0), code,
                1 if x.is_cuda else 0, x)
    a = np.asarray(x)
    if a.ndim == 1:
        a = a[None, :]
    if a.dtype not in (np.float32, np.float64) or a.strides[1] != a.itemsize:
        a = np.ascontiguousarray(a, dtype=np.float64 if a.dtype == np.float64 else np.float32)
    code = F32 if a.dtype == np.float32 else F64
    return (ctypes.c_void_p(a.ctypes.data), a.shape[0], a.strides[0] // a.itemsize, code, 0, a)


class FDSketch:
    """One buffered FD sketch on the GPU (fd_create ... fd_destroy)."""

    def __init__(self, d: int, ell: int, variant: str = "fd", alpha: float = 1.0,
                 prec: str = "fp32", stream=None, buffer_rows: int | None = None):
        lib = load()
        self.d, self.ell, self.variant, self.prec = d, ell, variant, prec
        self.buffer_rows = buffer_rows or (ell if variant == "fastpfd" else 2 * ell)
        self._stream = _stream_ptr(stream)
        h = ctypes.c_void_p()
        if buffer_rows is None:
            _check(lib.fd_create(d, ell, VARIANT[variant], float(alpha), PREC[prec], self._stream,
                                 ctypes.byref(h)), "fd_create")
        else:
            _check(lib.fd_create_buffered(d, ell, VARIANT[variant], float(alpha), PREC[prec],
                                          int(buffer_rows), self._stream, ctypes.byref(h)),
                   "fd_create_buffered")
        self._h = h

    def append(self, rows):
        ptr, n, ld, code, dev, keep = _as_rows(rows)
        _check(load().fd_append(self._h, ptr, n, ld, code, dev), "fd_append")
        return keep

    def sketch(self, out=None, dtype=np.float64):
        """B (ell x d). With ``out`` a CUDA tensor the result is written there."""
        lib = load()
        if out is not None:
            import torch
            code = F64 if out.dtype == torch.float64 else F32
            _check(lib.fd_sketch(self._h, ctypes.c_void_p(out.data_ptr()), code, 1), "fd_sketch")
            return out
        B = np.empty((self.ell, self.d), dtype=dtype)
        code = F64 if B.dtype == np.float64 else F32
        _check(lib.fd_sketch(self._h, ctypes.c_void_p(B.ctypes.data), code, 0), "fd_sketch")
        return B

    def sketch_compensated(self, out=None, dtype=np.float64):
        """Compensative FD sketch (fd_sketch_compensated); FD and PFD only."""
        lib = load()
        if out is not None:
            import torch
            code = F64 if out.dtype == torch.float64 else F32
            _check(lib.fd_sketch_compensated(self._h, ctypes.c_void_p(out.data_ptr()), code, 1),
                   "fd_sketch_compensated")
            return out
        B = np.empty((self.ell, self.d), dtype=dtype)
        code = F64 if B.dtype == np.float64 else F32
        _check(lib.fd_sketch_compensated(self._h, ctypes.c_void_p(B.ctypes.data), code, 0),
               "fd_sketch_compensated")
        return B

    def merge(self, other: "FDSketch"):
        """Fold ``other``'s stream into this sketch (fd_merge)."""
        _check(load().fd_merge(self._h, other._h), "fd_merge")

    def merge_sketch(self, B, stats: dict):
        """Fold a sketch given as its rows ``B`` (up to the last nonzero row)
        and the counters ``stats`` (an fd_stats dict) into this one
        (fd_merge_sketch)."""
        ptr, n, ld, code, dev, keep = _as_rows(B)
        st = Stats()
        for f, _ in Stats._fields_:
            if f in stats:
                setattr(st, f, type(getattr(st, f))(stats[f]))
        _check(load().fd_merge_sketch(self._h, ptr, n, ld, code, dev, ctypes.byref(st)),
               "fd_merge_sketch")
        return keep

    def cov_err(self, A) -> float:
        ptr, n, ld, code, dev, keep = _as_rows(A)
        out = ctypes.c_double()
        _check(load().fd_cov_err(self._h, ptr, n, ld, code, dev, ctypes.byref(out)), "fd_cov_err")
        return out.value

    def proj_err(self, A, k: int = 10) -> float:
        """||A - pi_{B_k}(A)||_F^2 / ||A - A_k||_F^2 of the current sketch (fd_proj_err)."""
        ptr, n, ld, code, dev, keep = _as_rows(A)
        out = ctypes.c_double()
        _check(load().fd_proj_err(self._h, ptr, n, ld, code, dev, int(k), ctypes.byref(out)),
               "fd_proj_err")
        return out.value

    def stats(self) -> dict:
        s = Stats()
        _check(load().fd_stats(self._h, ctypes.byref(s)), "fd_stats")
        return {f: getattr(s, f) for f, _ in Stats._fields_}

    def record_spectrum(self, on: bool = True):
        """Keep the spectrum of each reduction for last_spectrum() (fd_record_spectrum)."""
        _check(load().fd_record_spectrum(self._h, 1 if on else 0), "fd_record_spectrum")

    def last_spectrum(self):
        L = self.buffer_rows
        a = np.zeros(L)
        b = np.zeros(L)
        _check(load().fd_last_spectrum(self._h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                       b.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
               "fd_last_spectrum")
        return a, b

    def reset(self):
        _check(load().fd_reset(self._h), "fd_reset")

    def profile(self, enable: bool = True):
        _check(load().fd_profile(self._h, 1 if enable else 0), "fd_profile")

    def kernel_times(self):
        """{class: (launches, device ms)} since profiling was enabled."""
        c = (ctypes.c_int64 * 4)()
        m = (ctypes.c_double * 4)()
        _check(load().fd_kernel_times(self._h, c, m), "fd_kernel_times")
        names = ("ingest", "gram", "eig", "rotate")
        return {names[i]: (int(c[i]), float(m[i])) for i in range(4)}

    def close(self):
        if getattr(self, "_h", None):
            load().fd_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def merge_tree(sketches):
    """Merge a list of sketches pairwise, level by level ((0,1), (2,3), ...),
    until one is left; returns it (the others keep their own state)."""
    level = list(sketches)
    while len(level) > 1:
        nxt = []
        for i in range(0, len(level) - 1, 2):
            level[i].merge(level[i + 1])
            nxt.append(level[i])
        if len(level) % 2:
            nxt.append(level[-1])
        level = nxt
    return level[0]


def cov_err_noalloc(A, B, stream=None):
    """cov-err of CUDA tensors A and B through fd_cov_err_noalloc (no device
    allocation inside the library; fixed workspace, d <= 1024)."""
    pa, n, lda, ca, da, ka = _as_rows(A)
    pb, rows, ldb, cb, db, kb = _as_rows(B)
    if not (da and db):
        raise ValueError("A and B must be CUDA tensors")
    d = A.shape[1]
    if ldb != d:  # the entry point reads B with leading dimension d
        kb = kb.contiguous()
        pb, rows, ldb, cb, db, kb = _as_rows(kb)
    out = ctypes.c_double()
    _check(load().fd_cov_err_noalloc(pa, n, d, lda, ca, pb, rows, cb, _stream_ptr(stream),
                                     ctypes.byref(out)), "fd_cov_err_noalloc")
    return out.value


def cov_err_pair(A, B, stream=None):
    """(cov-err, lambda_min, lambda_max) of A^T A - B^T B on the GPU."""
    lib = load()
    pa, n, lda, ca, da, ka = _as_rows(A)
    pb, rows, ldb, cb, db, kb = _as_rows(B)
    if da != db:
        raise ValueError("A and B must both be on the device or both on the host")
    d = (A.shape[1])
    if ldb != d:
        raise ValueError("B must be contiguous (leading dimension d)")
    c, lo, hi = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib.fd_cov_err_pair(pa, n, d, lda, ca, pb, rows, cb, da, _stream_ptr(stream),
                               ctypes.byref(c), ctypes.byref(lo), ctypes.byref(hi)),
           "fd_cov_err_pair")
    return c.value, lo.value, hi.value


class FDBatch:
    """Many independent sketches updated together (fd_batch_* calls)."""

    def __init__(self, ds, ells, variant: str = "fd", alpha: float = 1.0, prec: str = "fp32",
                 stream=None):
        lib = load()
        self.ds = [int(x) for x in ds]
        self.ells = [int(x) for x in ells]
        n = len(self.ds)
        d_arr = (ctypes.c_int64 * n)(*self.ds)
        e_arr = (ctypes.c_int32 * n)(*self.ells)
        h = ctypes.c_void_p()
        _check(lib.fd_batch_create(n, d_arr, e_arr, VARIANT[variant], float(alpha), PREC[prec],
                                   _stream_ptr(stream), ctypes.byref(h)), "fd_batch_create")
        self._h = h
        self._keep = []

    def append(self, blocks):
        """blocks: {sketch id: CUDA tensor of rows} (one block per sketch per call)."""
        blocks = {k: v for k, v in blocks.items() if v.shape[0] > 0}
        if not blocks:
            return []
        items = (Work * len(blocks))()
        keep = []
        for i, (sid, x) in enumerate(blocks.items()):
            ptr, n, ld, code, dev, k = _as_rows(x)
            if not dev:
                raise ValueError("batched rows must be CUDA tensors")
            items[i] = Work(int(sid), code, ptr, n, ld)
            keep.append(k)
        _check(load().fd_batch_append(self._h, items, len(blocks)), "fd_batch_append")
        self._keep = keep   # rows must stay alive until the stream passes the call
        return keep

    def sketch(self, sid: int, dtype=np.float64):
        B = np.empty((self.ells[sid], self.ds[sid]), dtype=dtype)
        code = F64 if B.dtype == np.float64 else F32
        _check(load().fd_batch_sketch(self._h, sid, ctypes.c_void_p(B.ctypes.data), code, 0),
               "fd_batch_sketch")
        return B

    def offsets(self):
        """Element offsets of every sketch in a sketch_all buffer, and its size."""
        offs, tot = [], 0
        for d, e in zip(self.ds, self.ells):
            offs.append(tot)
            tot += d * e
        return offs, tot

    def sketch_all(self, out):
        """All sketches into the CUDA float32 tensor `out` (size from offsets())."""
        offs, tot = self.offsets()
        if out.numel() < tot:
            raise ValueError("output buffer too small")
        arr = (ctypes.c_int64 * len(offs))(*offs)
        _check(load().fd_batch_sketch_all(self._h, ctypes.c_void_p(out.data_ptr()), arr),
               "fd_batch_sketch_all")
        return out

    def prepare(self, blocks):
        """Build the work-item array once for repeated appends of the same rows."""
        blocks = {k: v for k, v in blocks.items() if v.shape[0] > 0}
        items = (Work * len(blocks))()
        keep = []
        for i, (sid, x) in enumerate(blocks.items()):
            ptr, n, ld, code, dev, k = _as_rows(x)
            items[i] = Work(int(sid), code, ptr, n, ld)
            keep.append(k)
        return items, len(blocks), keep

    def append_prepared(self, prep):
        items, n, _ = prep
        _check(load().fd_batch_append(self._h, items, n), "fd_batch_append")

    def stats(self, sid: int) -> dict:
        s = Stats()
        _check(load().fd_batch_stats(self._h, sid, ctypes.byref(s)), "fd_batch_stats")
        return {f: getattr(s, f) for f, _ in Stats._fields_}

    def reset(self):
        _check(load().fd_batch_reset(self._h), "fd_batch_reset")

    def uses_graph(self):
        """(whether appends run as the captured CUDA graph, graph launches so far)."""
        n = ctypes.c_int64(0)
        rc = load().fd_batch_uses_graph(self._h, ctypes.byref(n))
        if rc < 0:
            _check(rc, "fd_batch_uses_graph")
        return bool(rc), int(n.value)

    def close(self):
        if getattr(self, "_h", None):
            load().fd_batch_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FDServer:
    """Continuous-batching request loop over `count` live sketches (fd_serve_*)."""

    def __init__(self, count: int, d: int, ell: int, variant: str = "fd", alpha: float = 1.0,
                 budget_bytes: int = 256 << 20, streams: int = 2):
        lib = load()
        self.count, self.d, self.ell = count, d, ell
        h = ctypes.c_void_p()
        _check(lib.fd_serve_create(count, d, ell, VARIANT[variant], float(alpha), int(budget_bytes),
                                   streams, ctypes.byref(h)), "fd_serve_create")
        self._h = h

    def submit(self, sid: int, rows):
        """Ticket, or None when the budget is full (FD_EBUSY: retry later)."""
        a = np.ascontiguousarray(rows, dtype=np.float32)
        t = ctypes.c_int64()
        rc = load().fd_serve_submit(self._h, sid, ctypes.c_void_p(a.ctypes.data), a.shape[0],
                                    ctypes.byref(t))
        if rc == -5:
            return None
        _check(rc, "fd_serve_submit")
        return t.value

    def poll(self, max_items: int = 65536):
        tk = (ctypes.c_int64 * max_items)()
        lat = (ctypes.c_double * max_items)()
        cnt = ctypes.c_int32()
        _check(load().fd_serve_poll(self._h, tk, lat, max_items, ctypes.byref(cnt)), "fd_serve_poll")
        return [(tk[i], lat[i]) for i in range(cnt.value)]

    def drain(self):
        _check(load().fd_serve_drain(self._h), "fd_serve_drain")

    def sketch(self, sid: int):
        B = np.empty((self.ell, self.d), dtype=np.float64)
        _check(load().fd_serve_sketch(self._h, sid, ctypes.c_void_p(B.ctypes.data), F64),
               "fd_serve_sketch")
        return B

    def counters(self):
        v = [ctypes.c_int64() for _ in range(4)]
        _check(load().fd_serve_counters(self._h, *[ctypes.byref(x) for x in v]), "fd_serve_counters")
        return dict(zip(("admitted", "busy", "launches", "rows_done"), [x.value for x in v]))

    def close(self):
        if getattr(self, "_h", None):
            load().fd_serve_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
