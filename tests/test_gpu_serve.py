"""Serving-layer tests: continuous batching gives every request the same result
alone and in a mix, admission respects the memory cap, and the batched ground
states agree with sequential single-grid solves."""
import pytest

from paper_1206_1361_gb300 import gp
from paper_1206_1361_gb300.serve import Server, solve_batch, solve_sequential
from paper_1206_1361_gb300.workloads import Instance, Request, box_spacing
from tests.gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def make(shape, trap, g, arrival=0.0, kind="ground", qg=0.0, qsteps=0):
    h, dt = box_spacing(shape, trap, g)
    return Request(arrival, kind, Instance(shape, h, dt, trap, g), qg, qsteps)


REQS = [
    make((32, 48, 40), (1.0, 1.5, 2.0), 30.0, 0.0),
    make((48, 32, 1), (2.0, 1.0, 0.0), 60.0, 0.0, "quench", 50.0, 200),
    make((40, 40, 32), (3.0, 2.5, 1.0), 5.0, 0.01),
    make((64, 48, 32), (0.8, 1.2, 3.5), 120.0, 0.02, "quench", 110.0, 300),
    make((32, 32, 32), (1.0, 1.0, 1.0), 0.0, 0.03),
]


def by_key(results):
    return {(r.req.inst, r.req.kind): r for r in results}


def test_each_request_is_the_same_alone_and_in_the_mix():
    require_gpu()
    with Server(gp.GP_C64, cap_bytes=1 << 32) as s:
        mixed = by_key(s.run(REQS, realtime=False).results)
    assert len(mixed) == len(REQS)
    for req in REQS:
        with Server(gp.GP_C64, cap_bytes=1 << 32) as s:
            alone = s.run([req], realtime=False).results[0]
        m = mixed[(req.inst, req.kind)]
        assert alone.total_steps == m.total_steps
        assert alone.ground_steps == m.ground_steps
        for k in ("norm", "mu", "energy", "rms_x", "rms_y", "rms_z"):
            assert alone.obs[k] == m.obs[k], (req.kind, k)
        if req.kind == "quench":
            assert m.total_steps == m.ground_steps + req.quench_steps


def test_admission_never_exceeds_the_cap():
    require_gpu()
    fp = sorted(gp.gp_batch_footprint(r.inst.shape, gp.GP_C64) for r in REQS)
    cap = fp[-1] + fp[-2]                       # never room for three at once
    with Server(gp.GP_C64, cap_bytes=cap) as s:
        stats = s.run(REQS, realtime=True)
    assert len(stats.results) == len(REQS)
    assert stats.peak_bytes <= cap
    for r in stats.results:
        assert r.finished >= r.admitted >= r.arrival - 1e-9


def test_batched_ground_states_agree_with_sequential_solves():
    require_gpu()
    insts = [r.inst for r in REQS]
    batched = by_key(solve_batch(insts, gp.GP_C64).results)
    seq = by_key(solve_sequential([Request(0.0, "ground", i) for i in insts], gp.GP_C128,
                                  realtime=False).results)
    for inst in insts:
        b, s = batched[(inst, "ground")], seq[(inst, "ground")]
        # both converged to |dmu| < 1e-6 between checks; complex64 vs FP64
        assert abs(b.obs["mu"] - s.obs["mu"]) <= 2e-5 * abs(s.obs["mu"]), inst
        assert abs(b.obs["norm"] - 1) < 1e-6
