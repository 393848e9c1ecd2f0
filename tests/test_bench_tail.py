"""Host logic of the batch-tail report: the wall time after 90 % of the
instances finished, and the point-steps done in it with each instance's
steps spread evenly over its time in the batch."""
import os
import sys
from types import SimpleNamespace

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def res(points, steps, finished, admitted=0.0):
    return SimpleNamespace(req=SimpleNamespace(inst=SimpleNamespace(points=points)),
                           admitted=admitted, finished=finished, total_steps=steps)


def test_tail_of_ten_instances():
    # nine finish by t = 1, the last (1000 points, 400 steps) runs to t = 4
    rs = [res(100, 100, 0.5 + 0.05 * k) for k in range(9)] + [res(1000, 400, 4.0)]
    t = bench.batch_tail(SimpleNamespace(results=rs, wall=4.0), 0.9)
    assert t["tail_s"] == pytest.approx(4.0 - 0.9)
    assert t["share_of_wall"] == pytest.approx(3.1 / 4.0)
    assert t["instances_in_tail"] == 1
    # the last instance's steps spread over [0, 4]: 3.1 / 4 of them in the tail
    assert t["point_steps_per_s_in_tail"] == pytest.approx(1000 * 400 * (3.1 / 4.0) / 3.1)


def test_no_results():
    assert bench.batch_tail(SimpleNamespace(results=[], wall=1.0)) is None
