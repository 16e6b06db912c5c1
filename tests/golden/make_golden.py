"""Writes tests/golden/radii.txt from the CPU oracle only.

Run from the repository root:  python tests/golden/make_golden.py
The file lists, for each measured workload, the radius R that the oracle's
Eq. (22) solve (Appendix B.1) returns, as a hex float so it is exact.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1501_03545_gb300 import workloads  # noqa: E402


def main():
    lines = ["# name n alpha kbar R(hex) R(decimal) -- written by make_golden.py from oracle.solve_radius"]
    for w in workloads.ALL:
        R = oracle.solve_radius(w.n, w.alpha, w.kbar)
        lines.append("%s %d %r %r %s %.15f" % (w.name, w.n, w.alpha, w.kbar, float(R).hex(), R))
    with open(os.path.join(HERE, "radii.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
