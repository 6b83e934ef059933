"""Write the golden fixture: oracle R, T on a fixed sample of the seeded
64-stack x 12-layer workload.  Calls only ``oracle/`` (and the seeded input
generator); rerun it only when the oracle's arithmetic changes for a reason
that the commit message names.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2111_13667_gb300 import workloads as W  # noqa: E402

STACKS = [0, 31, 63]
THETAS = [0, 4, 9]
LAMBDAS = [0, 50, 100, 150, 199]


def main():
    w = W.plain_fp64()
    sub = w.subset(STACKS)
    n = oracle.assemble_index(sub.n_direct, None, None, sub.n_lambda)
    R, T = oracle.coh_tmm_pols("sp", n, sub.d, sub.theta, sub.lam)
    pick = np.ix_(range(2), range(len(STACKS)), THETAS, LAMBDAS)
    out = {
        "workload": "plain_fp64 (seed 0): 64 stacks x 12 layers, 200 lambda in 400-800 nm x 10 theta in 0-80 deg",
        "written_by": "tests/golden/make_golden.py (FP64 C oracle, oracle/tmm_oracle.c)",
        "stacks": STACKS, "theta_index": THETAS, "lambda_index": LAMBDAS, "pols": "sp",
        "R": [[[[repr(float(v)) for v in row] for row in plane] for plane in pol] for pol in R[pick]],
        "T": [[[[repr(float(v)) for v in row] for row in plane] for plane in pol] for pol in T[pick]],
    }
    with open(os.path.join(HERE, "oracle_plain_fp64_sample.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
