"""Write stored expected values for the parity tests.  Calls only the oracle and tbgen.

Usage: python tests/golden/make_golden.py
Writes tests/golden/w16_r125_k24.json: the oracle's S(E_F) on the full 24^3 mesh of the
W=16, N_R=125 random model (seed 0, E_F = 0, eta = 1e-3) plus the same at E_F in
{-1, -0.5, 0.5, 1} and eta = 1e-2.
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import tbgen  # noqa: E402
from oracle import kubo_oracle as O  # noqa: E402


def main():
    model, kmesh, E_F, etas, kT = tbgen.config("w16_r125_k24")
    E_F = np.array([-1.0, -0.5, 0.0, 0.5, 1.0])
    etas = np.array([1e-3, 1e-2])
    t0 = time.time()
    S = O.ahc(model.H_R, model.R, kmesh, E_F, etas=etas, kT=0.0)
    out = {
        "workload": "w16_r125_k24: W=16, R in {-2..2}^3, decay 1.0, seed 0, mesh 24^3",
        "writer": "tests/golden/make_golden.py (oracle only)",
        "E_F": E_F.tolist(), "etas": etas.tolist(), "kT": 0.0,
        "S": S.tolist(), "oracle_seconds": time.time() - t0,
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "w16_r125_k24.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path, S)


if __name__ == "__main__":
    main()
