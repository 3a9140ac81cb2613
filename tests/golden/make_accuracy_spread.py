"""Writes accuracy_spread.json: the stated error of the annealed solve, from
the FP64 oracle alone.

Case (the shape of the lifted 3D workload at a size the oracle solves): the
8-blob mixture vs its rigid copy, N = M = 1000, c = ||x - x'|| lifted by the
oracle's Kernel PCA to D = 32 (Prop. 2.3, Algorithm 4), uniform weights,
eps geometric 0.1 -> 1e-3 over 20 outer steps of 100 symmetric Sinkhorn
iterations (Algorithm 1 with Algorithm 3).

For each cost-tile precision the script runs the oracle's solve with fresh
uniform noise at the per-cell bound of that precision's exponent arithmetic
(helpers.noisy_cnt_gw), from three seeds, and records per outer step the
largest relative energy difference to the noiseless oracle.  That spread is
what the arithmetic of the precision implies for this solve; the GPU's
trajectory is held to it.

Calls only the oracle (and the seeded input generators):
    python tests/golden/make_accuracy_spread.py   (about 15 min on 8 cores)
"""

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
sys.path.insert(0, os.path.dirname(HERE))

import oracle as O  # noqa: E402
import workloads as W  # noqa: E402
from helpers import noisy_cnt_gw  # noqa: E402

N, D = 1000, 32
EPS0, EPS1, N_OUTER, N_INNER = 0.1, 1e-3, 20, 100
SEEDS = (1, 2, 3)
PRECS = {"fp32": 0, "f16x3": 3}


def case():
    r32 = lambda x: np.asarray(x, np.float32).astype(np.float64)
    w = W.gmm_rigid(N, seed=0)
    a = np.full(N, 1.0 / N)
    X = r32(O.lift(w["x"], a, "power", 1.0, D=D)["X"])
    Y = r32(O.lift(w["y"], a, "power", 1.0, D=D)["X"])
    return X, Y, r32(a)


def main():
    X, Y, a = case()
    ref = O.cnt_gw(a, a, X, Y, EPS0, N_OUTER, N_INNER, eps_final=EPS1, symmetric=True)
    E0 = np.array([h["E"] for h in ref["history"]])
    out = {"case": "gmm8-3d N=M=1000, ||x-x'|| Kernel PCA D=32, eps 0.1 -> 1e-3 geometric, "
                   "20 outer x 100 symmetric Sinkhorn",
           "E_oracle": E0.tolist(), "eps": [h["eps"] for h in ref["history"]],
           "seeds": list(SEEDS), "spread": {}}
    for name, prec in PRECS.items():
        worst = np.zeros(N_OUTER)
        per_seed = []
        for seed in SEEDS:
            h = noisy_cnt_gw(a, a, X, Y, EPS0, N_OUTER, N_INNER, prec, seed, eps_final=EPS1)
            rel = np.abs(np.array([r["E"] for r in h]) - E0) / np.abs(E0)
            per_seed.append(rel.tolist())
            worst = np.maximum(worst, rel)
            print(name, seed, " ".join(f"{v:.1e}" for v in rel), flush=True)
        out["spread"][name] = {"max": worst.tolist(), "per_seed": per_seed}
    with open(os.path.join(HERE, "accuracy_spread.json"), "w") as fh:
        json.dump(out, fh, indent=1)


if __name__ == "__main__":
    main()
