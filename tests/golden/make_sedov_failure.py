"""Writes sedov_262144_failure.txt: the step at which the oracle's Sedov
run (262,144 points, seed 2, Courant number 0.3) first produces a cell with
non-positive mass or thermal energy, the time reached before it, and the
cell (caller's index).

The scheme has no floor (the paper names energy depletion in strong
rarefactions as a way a run can crash, Section 2.3); in this blast the
evacuated interior empties a cell within the first hundred steps.  The
library must fail at the same step, in the same cell, and keep the state of
the last good step.

Usage:  python tests/golden/make_sedov_failure.py   (about two minutes)
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O  # noqa: E402
from paper_1410_3219_gb300 import workloads as W  # noqa: E402


def main():
    wl = W.sedov(n=262144, seed=2)
    s = O.Sim(wl)
    k = 0
    while True:
        t_good = s.t
        try:
            s.step(0.05)
        except O.OracleError:
            break
        k += 1
        if s.t >= 0.05:
            raise SystemExit("no failure before t = 0.05")
    c = s.conserved()
    eth = c["E"] - 0.5 * (c["px"] ** 2 + c["py"] ** 2) / c["m"]
    bad = np.where((c["m"] <= 0) | (eth <= 0))[0]
    lines = [
        "# Oracle Sedov run, 262,144 points (seed 2), Courant number 0.3: the",
        "# first step that leaves a cell with non-positive mass or thermal",
        "# energy; written by make_sedov_failure.py.",
        f"failing_step {k + 1}",
        f"t_before {t_good:.17g}",
        "cells " + " ".join(str(int(i)) for i in bad),
    ]
    with open(os.path.join(HERE, "sedov_262144_failure.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")
    print("\n".join(lines))


if __name__ == "__main__":
    main()
