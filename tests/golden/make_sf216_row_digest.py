"""Writes sf216_row_digest.json: a digest of one row of L.A computed by the FP64 oracle on the
216-atom spin-flip configuration (cubic cell a = 20.2 bohr, 108^3 grid, 25 Ha sphere of 49173
plane waves, 433 source-spin and 431 target-spin random orthonormal orbitals, 16 projected
trial vectors, exchange fraction 0.18, seed 0): the row (b = 0, v = 0) with all its 864 pair
convolutions, its norm, its contribution Re<x|(L x)> to omega_0, and 64 sampled coefficients.
The bench's 216-atom measurement compares its own row with it, so that the rate it reports
carries an error against the oracle without recomputing the row (about a minute of host time
and 26 GB of host memory) on every run. Calls only oracle/ and the input generator.

    python tests/golden/make_sf216_row_digest.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import tddft_oracle as O  # noqa: E402
from paper_2309_03513_b300 import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "sf216_row_digest.json")
ROW = (0, 0)


def digest() -> dict:
    n, a, ecut = 108, 20.2, 25.0
    npw = O.miller_sphere(n, a, ecut).shape[0]
    wl = synth.make_workload(n=n, a=a, ecut=ecut, npw=npw, nocc_src=433, nb=16, seed=0, spin_flip=True,
                             nocc_tgt=431)
    row = O.system_from_workload(wl).apply(wl.X, rows=[ROW])[0]
    x = wl.X[ROW]
    idx = np.linspace(0, npw - 1, 64).round().astype(int)
    return {
        "config": "108^3, a = 20.2 bohr, 25 Ha, spin-flip, nocc 433 up / 431 down, nb 16, alpha 0.18, seed 0 "
                  "(synth.make_workload defaults)",
        "npw": int(npw),
        "row": list(ROW),
        "norm": float(np.linalg.norm(row)),
        "omega_row": float(np.vdot(x, row).real),
        "samples": [[int(g), float(row[g].real), float(row[g].imag)] for g in idx],
    }


if __name__ == "__main__":
    d = digest()
    with open(OUT, "w") as fh:
        json.dump(d, fh, indent=1)
    print(OUT, d["norm"], d["omega_row"])
