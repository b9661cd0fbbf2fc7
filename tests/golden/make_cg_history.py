"""Write the FP64 oracle's CG residual histories used by the long-run solver tests.

Calls only oracle/ (and the seeded input generators): for each workload the oracle builds
the lattice and runs plain CG (Sec. 2; App. A: at most 500 iterations) on the symmetric
lattice operator (outputscale 1) + noise I, recording ||r_j|| / ||b|| of every column after
every iteration.  Output: one text file per workload with the iterations 1, 10, 20, ...,
max_iter (one row each: the iteration, then one value per column), '#' lines stating the
workload.

    python tests/golden/make_cg_history.py [--threads T] [--only NAME]

The oracle's results do not depend on the thread count.
"""

import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import OracleLattice, max_threads, set_threads  # noqa: E402
from paper_2106_06695_gb300 import synth  # noqa: E402

# name -> (n, d, seed, right-hand sides, description)
WORKLOADS = {
    "cg_history_n200k_d11": (
        200_000, 11, 2, "solve",
        "n=200,000 d=11: standardised 16-component GMM (seed 2), unit lengthscales, "
        "binomial stencil r=1, B = [y, 8 Rademacher probes] (k=9), noise 0.01"),
    "cg_history_n2M_d11": (
        2_000_000, 11, 4, "gauss16",
        "n=2,000,000 d=11: standardised 16-component GMM (seed 4), unit lengthscales, "
        "binomial stencil r=1, B = 16 columns N(0,1) (seed 4), noise 0.01"),
}
NOISE = 0.01
MAX_ITER = 500


def rhs(kind, X, seed):
    if kind == "solve":
        return synth.solve_rhs(X, seed, probes=8)
    return synth.gaussian_values(X.shape[0], 16, seed)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=max_threads())
    ap.add_argument("--only", default=None)
    args = ap.parse_args()
    set_threads(args.threads)
    for name, (n, d, seed, kind, desc) in WORKLOADS.items():
        if args.only and name != args.only:
            continue
        t0 = time.time()
        X = synth.gmm_points(n, d, seed)
        B = rhs(kind, X, seed).astype(np.float64)
        L = OracleLattice(X, np.ones(d, np.float32))
        _, iters, rel, hist = L.cg(B, NOISE, tol=0.0, max_iter=MAX_ITER, mode=2, history=True)
        rows = [1] + list(range(10, MAX_ITER + 1, 10))
        path = os.path.join(HERE, name + ".txt")
        with open(path, "w") as f:
            f.write("# FP64 oracle, plain CG on (K~ + noise I) x = b with the symmetric lattice\n")
            f.write("# operator (Sec. 2; Sec. 3.2; App. A: at most 500 iterations), tol 0 (every\n")
            f.write("# column runs all %d iterations); written by make_cg_history.py.\n" % MAX_ITER)
            f.write("# workload: %s; m = %d lattice vertices\n" % (desc, L.m))
            f.write("# columns: iteration, then ||r|| / ||b|| of each right-hand side\n")
            for j in rows:
                f.write("%d " % j + " ".join("%.6e" % v for v in hist[j - 1]) + "\n")
        print("%s: m=%d, final rel %s, %.0f s" % (name, L.m, np.array2string(rel, precision=3),
                                                 time.time() - t0), flush=True)


if __name__ == "__main__":
    main()
