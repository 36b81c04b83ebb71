"""Write tests/golden/fullsize_relres.json: the oracle's relative residuals for
configs 3 and 4 at their full sizes and sketch widths.

This script calls only the oracle (oracle/) and the seeded inputs
(workloads/).  It runs on the CPU for several minutes and tens of GB of host
memory, so its output is committed and the GPU test reads it.

Cases (Algorithm 1 with the Rademacher R of seed 13, tau = 1e-8):
  config3  2D disc |x| <= 0.8, n = 256 (N = 65536, M = 131753), k = 4096;
  config4  2D Poisson on the star r = 0.6 + 0.15 cos(5 theta), n = 128,
           2048 boundary points with weight 10, k = 2048.
The widths are those the adaptive setup settles on (the rank of the
perturbation at tau = 1e-8 is about 14.6 n in the disc, about 1800 for the
star, so k = 2048 saturates the disc and k = 4096 does not).  For each case the
file holds the kept rank and the relative residual ||A x - b|| / ||b|| of the
workload's right-hand side after zero and one refinement step.

Usage: python tests/golden/make_fullsize_relres.py [config3|config4 ...]
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402
from oracle.az import AZ, relres  # noqa: E402
from oracle.operators import Operator  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fullsize_relres.json")
SEED = 13
TAU = 1e-8
WIDTH = {"config3": 4096, "config4": 2048}


def case(name):
    if name == "config3":
        p = W.config3(n=256, k=WIDTH[name])
        op = Operator(p.grid, p.mask)
        b = p.rhs()
    else:
        p = W.config4(n=128, nb=2048, k=WIDTH[name])
        op = Operator(p.grid, p.mask, "poisson", p.boundary, p.weight)
        b = op.collocation_rhs(p.rhs(), p.boundary_rhs())
    t0 = time.time()
    az = AZ(op, p.k, SEED, TAU, chunk=256)
    t1 = time.time()
    x0 = az.solve(b)
    r0 = float(relres(op, x0, b)[0])
    x1 = x0 + az.solve_once(b - op.A(x0))
    r1 = float(relres(op, x1, b)[0])
    return {"N": op.N, "M": op.M, "Mb": op.Mb, "k": p.k, "seed": SEED, "tau": TAU, "rank": az.rank,
            "sigma_max": float(az.sig[0]), "relres_refine0": r0, "relres_refine1": r1,
            "oracle_seconds": round(time.time() - t0, 1), "sketch_and_svd_seconds": round(t1 - t0, 1)}


def main(names):
    out = {}
    if os.path.exists(OUT):
        out = json.load(open(OUT))
    out["what"] = ("oracle Algorithm 1 (oracle.az.AZ) at full size: rank kept at tau and relative residual "
                   "of the workload right-hand side after 0 and 1 refinement steps; written by "
                   "tests/golden/make_fullsize_relres.py")
    for n in names:
        out[n] = case(n)
        print(n, out[n], flush=True)
        with open(OUT, "w") as f:
            json.dump(out, f, indent=1)


if __name__ == "__main__":
    main(sys.argv[1:] or ["config4", "config3"])
