"""Writes condition_scales.json: the off-diagonal scale s of the seeded
factor generator (strict triangle uniform(-1,1) * s / k, diagonal
1 + |N(0,1)|) at which the factor's 1-norm condition number, as the oracle
estimates it (Hager's method with Higham's refinements), reaches the target
kappa. The precision-form workloads (refined TRSM, split-product
comparisons) and the engine tests read these scales for their inputs.

Run from the repository root: python tests/golden/make_condition_scales.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2504_13821_gb300 import inputs  # noqa: E402

ORDERS = (1024, 4096, 8192, 16384, 32768)
TARGETS = (1e2, 1e4, 1e6)


def seed_for(k: int, target: float) -> int:
    return 3 * k + int(round(np.log10(target)))


def main():
    oracle.build()
    out = {"generator": "paper_2504_13821_gb300.inputs.tri_matrix, uplo L",
           "estimator": "oracle.cond_one_estimate (trans N, diag N)", "entries": []}
    for k in ORDERS:
        for t in TARGETS:
            seed = seed_for(k, t)
            s = oracle.scale_for_condition(k, t, seed=seed, steps=30)
            A = inputs.tri_matrix(k, "L", seed=seed, dtype=np.float64, scale=s)
            kappa = oracle.cond_one_estimate("L", "N", "N", A)
            out["entries"].append({"k": k, "target": t, "seed": seed, "scale": s,
                                   "kappa_estimate": kappa})
            print(k, t, seed, s, kappa, flush=True)
            # written after every entry: the large orders take minutes each
            with open(os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                   "condition_scales.json"), "w") as f:
                json.dump(out, f, indent=1)
                f.write("\n")


if __name__ == "__main__":
    main()
