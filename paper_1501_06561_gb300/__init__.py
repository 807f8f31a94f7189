"""GB300-native buffered Frequent Directions (FD) sketching.

The sketching arithmetic lives in hand-written sm_103a CUDA kernels behind the
C ABI declared in ``include/fdsketch.h`` (library ``libfdsketch.so``, built
in-tree by ``paper_1501_06561_gb300.build``). ``paper_1501_06561_gb300.fd`` is
the thin ctypes binding with the same entry-point names; it loads the library
on first use and raises if it is missing (there is no CPU fallback).
``paper_1501_06561_gb300.workloads`` draws the seeded synthetic row streams.
"""
__all__ = ["fd", "workloads", "build"]
