"""Writes expected values that take the oracle minutes to compute, so the
GPU tests can compare against them. Calls only the oracle (and the shared
input generator). Run from the repository root:

    python tests/golden/make_golden.py
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import gen  # noqa: E402
import oracle  # noqa: E402


def main():
    t0 = time.time()
    t = gen.rmat(20, 16, seed=4)
    g = oracle.csr_from_tuples(t)
    count = oracle.tc(g)
    with open(os.path.join(HERE, "tc_rmat_s20.txt"), "w") as f:
        f.write("# Triangle count of R-MAT scale 20, edge factor 16, seed 4 (a=.57 b=.19 c=.19 d=.05,\n"
                "# symmetrised, self-loops and duplicates removed), by the oracle's node iterator\n"
                "# (Section 7.5 counts triangles as the reduction of the masked product).\n"
                "# Written by tests/golden/make_golden.py.\n")
        f.write(f"n: {g.n}\nm_stored: {g.m}\ntriangles: {count}\n")
    print(f"tc_rmat_s20: {count} ({time.time() - t0:.0f} s)")


if __name__ == "__main__":
    main()
