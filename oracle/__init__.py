"""FP64 CPU oracle for the buffered Frequent Directions update (test infrastructure).

This package is test infrastructure. Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
it. The product path (``paper_1501_06561_gb300``) never imports, calls or links
anything here, and this package never imports the product path.
"""
from .fd_oracle import (  # noqa: F401
    VARIANTS,
    FDOracle,
    compensate,
    cov_err,
    cov_spectrum,
    fast_pfd_split,
    fd_sketch,
    jacobi_svd_rows,
    proj_err,
    reduce_rank,
    shrink_index_split,
)
