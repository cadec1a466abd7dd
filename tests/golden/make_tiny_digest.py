"""Writes tiny_24_digest.json: a digest of the FP64 oracle on the tiny spin-conserving
configuration (cubic cell a = 10 bohr, 24^3 grid, 10 Ha sphere of 1503 plane waves, 8 random
orthonormal orbitals, 4 projected trial vectors, exchange fraction 0.18, kappa_x(0) = 2 pi R_c^2
with R_c = 5 bohr, seed 0), so that a later change of the oracle's arithmetic shows up in
tests/test_oracle_pins.py. Calls only oracle/ and the input generator; the paper prints no values
for the operator itself, so the digest is a regression fixture, not a pin to the paper.

    python tests/golden/make_tiny_digest.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import tddft_oracle as O  # noqa: E402
from paper_2309_03513_b300 import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiny_24_digest.json")
SAMPLES = [(0, 0, 0), (1, 3, 17), (2, 5, 400), (3, 7, 1502)]  # (b, v, G index)


def digest() -> dict:
    n, a, ecut = 24, 10.0, 10.0
    wl = synth.make_workload(n=n, a=a, ecut=ecut, npw=O.Grid(n, a, ecut).npw, nocc_src=8, nb=4, seed=0)
    S = O.system_from_workload(wl)
    LX = S.apply(wl.X)
    omega = np.einsum("bvg,bvg->b", wl.X.conj(), LX)
    return {
        "config": "24^3, a = 10 bohr, 10 Ha, nocc 8, nb 4, alpha 0.18, seed 0 (synth.make_workload defaults)",
        "npw": int(wl.phi_src.shape[1]),
        "omega": [float(w.real) for w in omega],
        "row_norms": [float(x) for x in np.linalg.norm(LX.reshape(4, -1), axis=1)],
        "samples": [[b, v, g, float(LX[b, v, g].real), float(LX[b, v, g].imag)] for b, v, g in SAMPLES],
    }


if __name__ == "__main__":
    with open(OUT, "w") as fh:
        json.dump(digest(), fh, indent=1)
    print("wrote", OUT)
