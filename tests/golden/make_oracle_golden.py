"""Writes oracle_plain32.json: the FP64 oracle's answer on the 32^3 lattice set-up (unit point source
at cell (16,16,16), kappa h = 0.1, vacuum boundaries, 16 Fibonacci directions; the R-type test geometry
of Sec. 3.1 without the chemistry). Calls only the oracle and the input generators; run from the
repository root:  python tests/golden/make_oracle_golden.py"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from synth import configs  # noqa: E402

SAMPLE = [0, 31, 1023, 16912, 16913, 16944, 17936, 20000, 32767]


def main():
    oracle.build()
    p = configs.plain32()
    r = oracle.solve(p.mesh, p.omega, p.weight, p.kappa_abs, p.emissivity, threads=4)
    rc, _, depth = oracle.levels(p.mesh, p.omega)
    assert rc == 0 and r["rc"] == 0
    depths = [int(x) for x in depth]
    out = {
        "what": "FP64 oracle on configs.plain32(): J and Gamma at sampled cells, total Gamma, escaped flux, "
                "depth of every direction",
        "cells": SAMPLE,
        "J": [float(r["J"][c, 0]) for c in SAMPLE],
        "Gamma": [float(r["Gamma"][c, 0]) for c in SAMPLE],
        "Gamma_total": float(np.sum(r["Gamma"])),
        "escaped": float(r["stats"]["escaped"]),
        "depths": depths,
    }
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_plain32.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
