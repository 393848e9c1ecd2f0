"""Write tests/golden/oracle_regression.json: observables of small cases
computed by the FP64 CPU oracle (oracle/ only).  The paper prints no
physical values for a worked example (its tables are running times), so these
are regression fixtures of the oracle, pinned by the closed-form and
invariant tests of tests/test_oracle_*.py, not values quoted from the paper.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

CASES = [
    # 64^3 on [-6.4, 6.4)^3, (1, 1.5, 2), g = 10, dt = 0.002, 1000 imaginary steps
    {"name": "imag3d-64^3-g10-1000", "kind": "cartesian", "shape": [64, 64, 64], "h": [0.2, 0.2, 0.2],
     "dt": 0.002, "trap": [1.0, 1.5, 2.0], "g": 10.0, "mode": 0, "steps": 1000},
    # 2D, 96 x 80, imaginary then real time
    {"name": "imag2d-96x80-g25-600", "kind": "cartesian", "shape": [96, 80, 1], "h": [0.15, 0.18, 1.0],
     "dt": 0.003, "trap": [1.0, 1.3, 0.0], "g": 25.0, "mode": 0, "steps": 600},
    {"name": "real3d-48x40x36-g30-300", "kind": "cartesian", "shape": [48, 40, 36], "h": [0.25, 0.25, 0.3],
     "dt": 0.002, "trap": [1.2, 1.0, 1.6], "g": 30.0, "mode": 1, "steps": 300},
    # axially symmetric, imaginary time
    {"name": "axial-64x128-g10-1000", "kind": "axial", "nr": 64, "nz": 128, "hr": 0.1, "hz": 0.1,
     "dt": 0.002, "gamma": 1.0, "lambda": 2.0, "g": 10.0, "mode": 0, "steps": 1000},
]


def run(c):
    if c["kind"] == "axial":
        p = oracle.AxialParams.make(c["nr"], c["nz"], c["hr"], c["hz"], c["dt"], c["gamma"],
                                    c["lambda"], c["g"], c["mode"])
        psi = oracle.axial_seed(p)
        oracle.axial_step(p, psi, c["steps"])
        return oracle.axial_observables(p, psi)
    p = oracle.Params.make(tuple(c["shape"]), tuple(c["h"]), c["dt"], *c["trap"], c["g"], c["mode"])
    psi = oracle.seed(p)
    oracle.step(p, psi, c["steps"])
    return oracle.observables(p, psi)


def main():
    out = {"source": "FP64 CPU oracle (oracle/sscn_ref.c), written by tests/golden/make_golden.py",
           "cases": []}
    for c in CASES:
        out["cases"].append(dict(c, observables=run(c)))
    with open(os.path.join(HERE, "oracle_regression.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
