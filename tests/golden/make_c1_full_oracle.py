"""Writes c1_full_oracle.json: the FP64 oracle on the full Random Noisy stream
of 200,000 x 2,000 rows (k = 50 signal dimensions, zeta = 10, seed 1, FP32
rows) with ell = 100, buffered FD (Algorithm 1 with a 2*ell-row buffer,
Sec. 2.3). With --ell / --variant / --alpha it writes the same record for
another sketch size or rule of the C1 grid to c1_full_oracle_<variant>_ell<ell>.json
(PFD: Algorithm 2 with its alpha; iSVD: Sec. 2.1).

Stored: cov-err of the oracle's sketch (Sec. 1.1, d x d difference formed in
FP64), Delta = sum of every delta (Sec. 3.1, the final flush included),
||A||_F^2, ||B||_F^2, the removed mass, the reduction count and the singular
values of B. Only the seeded input generator and the oracle are called.

    python tests/golden/make_c1_full_oracle.py     # about 2-3 min on 8 cores
    python tests/golden/make_c1_full_oracle.py --ell 50
    python tests/golden/make_c1_full_oracle.py --ell 200
    python tests/golden/make_c1_full_oracle.py --variant pfd --alpha 0.2
    python tests/golden/make_c1_full_oracle.py --variant isvd
"""
import argparse
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import fd_oracle as O  # noqa: E402
from paper_1501_06561_gb300 import workloads as W  # noqa: E402

N, D, M, ZETA, SEED = 200_000, 2000, 50, 10.0, 1


def out_name(ell, variant):
    if (ell, variant) == (100, "fd"):
        return "c1_full_oracle.json"
    return f"c1_full_oracle_{variant}_ell{ell}.json"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--ell", type=int, default=100)
    ap.add_argument("--variant", default="fd", choices=["fd", "pfd", "isvd", "ss"])
    ap.add_argument("--alpha", type=float, default=1.0)
    args = ap.parse_args()
    ELL = args.ell
    A = W.random_noisy(N, D, m=M, zeta=ZETA, seed=SEED, dtype=np.float32, row_stop=N)
    o = O.FDOracle(D, ELL, args.variant, args.alpha)
    for i in range(0, N, 10_000):
        o.append(A[i:i + 10_000])
    B, info = o.sketch()
    ce = O.cov_err(A, B, info["normA2"])
    sig = np.linalg.svd(B, compute_uv=False)
    out = {
        "source": "tests/golden/make_c1_full_oracle.py (FP64 oracle; Alg. 1 buffered, Sec. 2.3; "
                  "cov-err Sec. 1.1; Delta Sec. 3.1)",
        "workload": dict(kind="random_noisy", n=N, d=D, m=M, zeta=ZETA, seed=SEED,
                         dtype="float32", ell=ELL, variant=args.variant, alpha=args.alpha),
        "cov_err": ce,
        "sum_delta": info["sum_delta"],
        "normA2": info["normA2"],
        "normB2": info["normB2"],
        "removed": info["removed"],
        "reductions": info["reductions"],
        "sigma": [float(s) for s in sig],
    }
    with open(os.path.join(HERE, out_name(ELL, args.variant)), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(json.dumps({k: v for k, v in out.items() if k != "sigma"}, indent=1))


if __name__ == "__main__":
    main()
