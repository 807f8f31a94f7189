"""C-ABI library checks that need no GPU: it loads, exports every function
include/fdsketch.h declares, and rejects bad arguments before touching CUDA."""
import ctypes
import os
import subprocess

import pytest

from paper_1501_06561_gb300 import fd
from paper_1501_06561_gb300 import build as fdbuild


@pytest.fixture(scope="module")
def lib():
    fdbuild.build()
    return fd.load()


def test_exports_every_declared_function(lib):
    declared = fd.header_functions()
    assert len(declared) >= 10
    out = subprocess.run(["nm", "-D", "--defined-only", fd.LIB_PATH], capture_output=True,
                         text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    missing = [f for f in declared if f not in exported]
    assert not missing, missing
    for f in declared:
        assert hasattr(lib, f)


def test_version_and_strerror(lib):
    assert b"sm_103a" in lib.fd_version()
    for code in (0, -1, -2, -4, -5):
        assert lib.fd_strerror(code)
    assert lib.fd_strerror(-99) == b"unknown error code"


@pytest.mark.parametrize("args", [
    (0, 4, 0, 1.0, 0),        # d < 1
    (10, 1, 0, 1.0, 0),       # ell < 2
    (10, 257, 0, 1.0, 0),     # 2*ell > 512
    (10, 4, 7, 1.0, 0),       # unknown variant
    (10, 4, 1, 0.0, 0),       # PFD alpha = 0
    (10, 4, 1, 1.5, 0),       # PFD alpha > 1
    (10, 4, 0, 1.0, 9),       # unknown precision
])
def test_create_rejects_bad_arguments(lib, args):
    h = ctypes.c_void_p()
    assert lib.fd_create(*args, None, ctypes.byref(h)) == -1
    assert not h.value


def test_null_handle_calls_are_rejected(lib):
    assert lib.fd_create(10, 4, 0, 1.0, 0, None, None) == -1
    assert lib.fd_append(None, None, 1, 10, 0, 0) == -1
    assert lib.fd_sketch(None, None, 0, 0) == -1
    assert lib.fd_stats(None, None) == -1
    assert lib.fd_destroy(None) == -1
    c = ctypes.c_double()
    assert lib.fd_cov_err(None, None, 1, 1, 0, 0, ctypes.byref(c)) == -1
    assert lib.fd_cov_err_pair(None, 1, 1, 1, 0, None, 1, 0, 0, None, ctypes.byref(c), None,
                               None) == -1


def test_binding_raises_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(fd, "_lib", None)
    monkeypatch.setattr(fd, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        fd.load()
