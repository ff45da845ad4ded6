"""Writes tests/golden/stresslet_uniform_1e5_256.txt: the double-layer
(stresslet) periodic sum of Sec. 2.3 at 256 seeded targets of the uniform
N = 100,000 workload, from the CPU oracle alone (oracle/stresslet.py, direct
Ewald sum).  The GPU parity test of the combined apply at this size reads it
instead of re-running the oracle (about two minutes of numpy work).

Inputs: positions and forces of the named workload (workloads.make), q and n
iid N(0, 1) from numpy PCG64 seed 1009 (q first), targets 256 distinct indices
from seed 7, sorted.  xi = 5.5 only balances the oracle's real- and k-space
work; the sum does not depend on it.

Run from the repository root:  python tests/golden/make_stresslet_uniform_1e5.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import stresslet  # noqa: E402
from paper_2606_19059_gb300 import workloads  # noqa: E402

NAME = "uniform_1e5_tol1e-6_M128_P12"
OUT = os.path.join(ROOT, "tests", "golden", "stresslet_uniform_1e5_256.txt")


def inputs():
    kind, N, L, tol, M, P, seed = workloads.WORKLOADS[NAME]
    x, f = workloads.make(kind, N, seed, L)
    rng = np.random.default_rng(1009)
    q = rng.standard_normal((N, 3))
    n = rng.standard_normal((N, 3))
    idx = np.sort(np.random.default_rng(7).choice(N, 256, replace=False))
    return x, f, q, n, idx, L


def main():
    x, f, q, n, idx, L = inputs()
    u = stresslet.ewald(x, stresslet.densities(q, n), L, xi=5.5 / L, targets=idx)
    with open(OUT, "w") as fh:
        fh.write("# double-layer periodic sum (oracle/stresslet.py ewald, FP64) at 256 targets of the\n")
        fh.write(f"# {NAME} workload; q, n ~ N(0,1) from seed 1009; written by\n")
        fh.write("# tests/golden/make_stresslet_uniform_1e5.py\n")
        fh.write("# index ux uy uz\n")
        for i, row in zip(idx, u):
            fh.write(f"{int(i)} {float(row[0])!r} {float(row[1])!r} {float(row[2])!r}\n")


if __name__ == "__main__":
    main()
