"""Regression fixtures (tests/golden/oracle_regression.json, written by
tests/golden/make_golden.py from the oracle alone): the oracle reproduces
them (CPU), and the CUDA path matches them (GPU) at the FP64 parity bar."""
import json
import os

import pytest

import oracle
from paper_1206_1361_gb300 import gp
from tests.gpu_util import require_gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "oracle_regression.json")
CASES = json.load(open(GOLDEN))["cases"]
KEYS = ("norm", "mu", "energy", "rms_x", "rms_y", "rms_z", "rms_r")


def _oracle(c):
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


@pytest.mark.parametrize("c", CASES, ids=[c["name"] for c in CASES])
def test_oracle_reproduces_golden(c):
    got = _oracle(c)
    for k in KEYS:
        want = c["observables"][k]
        assert abs(got[k] - want) <= 1e-12 * max(1.0, abs(want)), k


@pytest.mark.gpu
@pytest.mark.parametrize("c", CASES, ids=[c["name"] for c in CASES])
def test_gpu_matches_golden(c):
    require_gpu()
    if c["kind"] == "axial":
        s = gp.Solver.axial(c["nr"], c["nz"], c["hr"], c["hz"], c["dt"], c["gamma"], c["lambda"],
                            c["g"], c["mode"])
    else:
        s = gp.Solver(tuple(c["shape"]), tuple(c["h"]), c["dt"], *c["trap"], c["g"], c["mode"])
    with s:
        s.load(None).step(c["steps"])
        obs = s.observables()
    for k in KEYS:
        want = c["observables"][k]
        assert abs(obs[k] - want) <= 1e-10 * max(1.0, abs(want)), (k, obs[k], want)
