"""The continuous-batching loop's host logic (serve.Server) against a stand-in
batch, no GPU: admission under the memory cap, chunked launches that stop at
the next due convergence check, observables requested for the due instances
only, the check cadence K = max(10, ceil(0.05 / dt)), convergence, the quench
hand-over to real time, and the point-step count."""
import math

import pytest

from paper_1206_1361_gb300 import gp, serve, workloads


class StandInBatch:
    """Records the calls the server makes; mu of slot s after n imaginary
    steps is mu_inf + a exp(-r n), so |dmu| between checks falls below 1e-6
    after a predictable number of checks."""

    def __init__(self, precision, cap, stream=None):
        self.cap, self.used = int(cap), 0
        self.slots, self.free = {}, []
        self.launches, self.obs_calls, self.params = [], [], []
        self.checks = {}                # slot -> [(imaginary steps, mu)] at each check

    def add(self, shape, h, dt, g0, g1, g2, g, mode, psi=None):
        need = shape[0] * shape[1] * shape[2] * 8
        if self.used + need > self.cap:
            raise gp.GPError(gp.GP_EFULL, "cap")
        slot = self.free.pop(0) if self.free else len(self.slots)
        self.slots[slot] = {"need": need, "steps": 0, "imag": 0, "mode": mode, "dt": dt}
        self.used += need
        return slot

    def step(self, n):
        self.launches.append((n, sorted(self.slots)))
        for s in self.slots.values():
            s["steps"] += n
            if s["mode"] == gp.GP_IMAG:
                s["imag"] += n

    def observables(self, slots=None):
        assert slots is not None, "the server asks for the due instances only"
        self.obs_calls.append((list(slots), len(self.slots)))
        out = {}
        for k in slots:
            s = self.slots[k]
            mu = 2.0 + 0.5 * math.exp(-0.002 * s["imag"])
            self.checks.setdefault(k, []).append((s["imag"], mu))
            out[k] = {"mu": mu, "norm": 1.0, "step": s["steps"]}
        return out

    def set_params(self, slot, g, mode):
        self.params.append((slot, g, mode))
        self.slots[slot]["mode"] = mode

    def remove(self, slot):
        self.used -= self.slots.pop(slot)["need"]
        self.free.append(slot)

    def info(self):
        return len(self.slots), len(self.slots) + len(self.free), self.used

    def close(self):
        pass


@pytest.fixture
def stand_in(monkeypatch):
    made = []

    def factory(precision, cap, stream=None):
        b = StandInBatch(precision, cap, stream)
        made.append(b)
        return b

    monkeypatch.setattr(serve.gp, "Batch", factory)
    return made


def _inst(edge, dt):
    return workloads.Instance((edge, edge, edge), (0.1, 0.1, 0.1), dt, (1.0, 1.0, 1.0), 5.0)


def test_checks_ask_only_for_due_instances_and_count_point_steps(stand_in):
    reqs = [workloads.Request(0.0, "ground", _inst(16, dt)) for dt in (0.005, 0.002, 0.001)]
    with serve.Server(gp.GP_C64, cap_bytes=10 ** 9, chunk=10) as srv:
        stats = srv.run(reqs, realtime=False)
    b = stand_in[0]
    assert len(stats.results) == 3 and all(r.converged for r in stats.results)
    # every launch is whole chunks of 10 steps, at most 10 chunks
    assert all(n % 10 == 0 and 10 <= n <= 100 for n, _ in b.launches)
    # observables of a subset: never more than the instances then on the device,
    # and on some checks fewer (the three solves are due at different steps)
    assert all(0 < len(c) <= active for c, active in b.obs_calls)
    assert any(len(c) < active for c, active in b.obs_calls)
    # each solve is checked in the chunk after every multiple of its K (10,
    # 25, 50 steps) and stops at the first check whose |dmu| meets the
    # complex64 criterion; the slots are taken in admission order
    for slot, r in enumerate(sorted(stats.results, key=lambda q: reqs.index(q.req))):
        k = workloads.convergence_interval(r.req.inst.dt)
        seen = b.checks[slot]
        for j, (steps, _) in enumerate(seen, start=1):
            assert j * k <= steps < j * k + 10
        tol = lambda mu: max(serve.MU_TOL, 2.0 ** -22 * abs(mu))
        dmu = [abs(seen[j][1] - seen[j - 1][1]) for j in range(1, len(seen))]
        assert dmu[-1] < tol(seen[-1][1]) and all(d >= tol(seen[i + 1][1]) for i, d in enumerate(dmu[:-1]))
        assert r.ground_steps == r.total_steps == seen[-1][0]
    assert stats.point_steps == sum(n * len(active) * 16 ** 3 for n, active in b.launches)


def test_quench_switches_to_real_time_and_runs_its_steps(stand_in):
    inst = _inst(16, 0.005)
    req = workloads.Request(0.0, "quench", inst, quench_g=7.5, quench_steps=130)
    with serve.Server(gp.GP_C64, cap_bytes=10 ** 9, chunk=10) as srv:
        stats = srv.run([req], realtime=False)
    b = stand_in[0]
    (r,) = stats.results
    assert b.params == [(0, 7.5, gp.GP_REAL)]
    assert r.converged and r.total_steps - r.ground_steps >= 130
    assert r.total_steps - r.ground_steps < 130 + 10      # whole chunks past the quench length
    assert r.ground_obs is not None and r.obs is not None


def test_admission_waits_for_the_cap(stand_in):
    need = 16 ** 3 * 8
    reqs = [workloads.Request(0.0, "ground", _inst(16, 0.005)) for _ in range(5)]
    with serve.Server(gp.GP_C64, cap_bytes=2 * need, chunk=10) as srv:
        stats = srv.run(reqs, realtime=False)
    b = stand_in[0]
    assert len(stats.results) == 5
    assert max(len(active) for _, active in b.launches) == 2
    assert stats.peak_bytes <= 2 * need
