"""Many SSCN problems on one GPU: batched solves and a continuous-batching
server, both driven through the batch C ABI (gp_batch_*).

A request is an imaginary-time ground-state solve, run until the chemical
potential changes by less than 1e-6 between checks K = max(10, ceil(0.05/dt))
steps apart (complex64: by less than max(1e-6, 2^-22 |mu|), the resolution of
mu from an FP32 state), optionally followed by a quench: the resident ground
state continues in real time at a new g for a fixed number of steps.

A solve also ends, unconverged, at the step cap or when |dmu| has not reached
a new minimum for STALL_CHECKS checks in a row: where dt g max|psi|^2 is large
the explicit nonlinear step makes the imaginary-time iteration settle into a
cycle (mu alternating between two values) that no number of steps resolves.
A converging solve lowers |dmu| at every check and never meets that rule.

The server admits requests that have arrived, first come first served, as
long as the batch's memory cap can take their footprint; every instance on the
device advances together, chunk by chunk, in one persistent launch per chunk;
finished requests leave at a chunk boundary and free their memory, so newly
arrived ones join while others are mid-solve.  Each instance's arithmetic
depends only on its own parameters (see gp_batch), so a request's result is
the same alone and in any mix.

The sequential comparator solves the same requests one at a time on a
single-grid context (plain FP64 by default), in arrival order.
"""
import collections
import time
from dataclasses import dataclass, field

from . import gp
from .workloads import convergence_interval

MU_TOL = 1e-6
STALL_CHECKS = 100
# complex64 states carry FP32 rounding noise of ~1e-7 |mu| in the chemical
# potential, so the absolute criterion is floored there at 2^-22 |mu|.
MU_REL_FLOOR = {gp.GP_C64: 2.0 ** -22, gp.GP_C128: 0.0}


def mu_converged(mu, mu_prev, precision):
    if mu_prev is None:
        return False
    return abs(mu - mu_prev) < max(MU_TOL, MU_REL_FLOOR[precision] * abs(mu))


@dataclass
class Job:
    req: object
    slot: int
    t_admit: float
    phase: str = "ground"           # "ground", then "real" for quenches
    steps: int = 0                  # steps taken in the current phase
    total_steps: int = 0
    next_check: int = 0
    mu_prev: float = None
    obs: dict = None
    ground_obs: dict = None
    watch: object = None
    converged: bool = True
    stalled: bool = False


@dataclass
class Result:
    req: object
    arrival: float
    admitted: float
    finished: float
    ground_steps: int
    total_steps: int
    obs: dict
    ground_obs: dict = None
    converged: bool = True
    stalled: bool = False

    @property
    def latency(self):
        return self.finished - self.arrival


@dataclass
class ServeStats:
    results: list
    wall: float
    point_steps: int
    peak_bytes: int
    chunks: int = 0
    extra: dict = field(default_factory=dict)

    def summary(self):
        import numpy as np
        lat = np.array([r.latency for r in self.results]) if self.results else np.zeros(1)
        return {"requests": len(self.results), "wall_s": self.wall,
                "converged": sum(1 for r in self.results if r.converged),
                "stalled": sum(1 for r in self.results if r.stalled),
                "requests_per_s": len(self.results) / self.wall if self.wall else 0.0,
                "point_steps_per_s": self.point_steps / self.wall if self.wall else 0.0,
                "p50_latency_s": float(np.percentile(lat, 50)),
                "p99_latency_s": float(np.percentile(lat, 99)),
                "mean_latency_s": float(lat.mean()), "peak_bytes": self.peak_bytes,
                "chunks": self.chunks}


class StallWatch:
    """Tracks the best |dmu| of a solve and the checks since it last fell."""

    def __init__(self):
        self.best, self.since = float("inf"), 0

    def update(self, dmu):
        if dmu < self.best:
            self.best, self.since = dmu, 0
        else:
            self.since += 1
        return self.since >= STALL_CHECKS


def _instance_args(inst):
    return inst.shape, inst.h, inst.dt, inst.trap[0], inst.trap[1], inst.trap[2], inst.g


class Server:
    """Continuous batching over one gp_batch."""

    def __init__(self, precision=gp.GP_C64, cap_bytes=120 * 10 ** 9, chunk=10, max_chunks=10,
                 stream=None):
        self.precision = precision
        self.cap = int(cap_bytes)
        self.chunk = int(chunk)
        self.max_chunks = int(max_chunks)     # longest launch, for admission latency
        self.batch = gp.Batch(precision, self.cap, stream)

    def close(self):
        self.batch.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _admit(self, req, now):
        shape, h, dt, g0, g1, g2, g = _instance_args(req.inst)
        slot = self.batch.add(shape, h, dt, g0, g1, g2, g, gp.GP_IMAG, psi=None)
        return Job(req=req, slot=slot, t_admit=now, next_check=convergence_interval(dt),
                   watch=StallWatch())

    def run(self, requests, realtime=True, max_steps=200000, on_chunk=None):
        """Serve `requests` (with .arrival seconds).  realtime: requests become
        visible at their arrival time on the wall clock; otherwise all are
        queued at t = 0 (throughput mode).  Returns ServeStats."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        active = {}
        results = []
        t0 = time.perf_counter()
        now = 0.0
        point_steps = 0
        peak = 0
        chunks = 0
        while pending or active:
            now = time.perf_counter() - t0
            # admission: FIFO while the cap takes the next footprint
            while pending and (not realtime or pending[0].arrival <= now):
                try:
                    job = self._admit(pending[0], now)
                except gp.GPError as e:
                    if e.code == gp.GP_EFULL:
                        break
                    raise
                pending.popleft()
                active[job.slot] = job
            peak = max(peak, self.batch.info()[2])
            if not active:
                if pending:                       # idle until the next arrival
                    wait = pending[0].arrival - (time.perf_counter() - t0)
                    if wait > 0:
                        time.sleep(min(wait, 0.01))
                continue
            # run up to the next due check (whole chunks, at most max_chunks;
            # one chunk while requests wait, so they are admitted promptly)
            def to_due(j):
                if j.phase == "ground":
                    left = min(j.next_check, max_steps) - j.steps
                else:
                    left = j.req.quench_steps - j.steps
                return max(1, -(-left // self.chunk))
            n = min(to_due(j) for j in active.values())
            if pending:
                n = 1
            n = min(n, self.max_chunks) * self.chunk
            self.batch.step(n)
            chunks += 1
            for job in active.values():
                job.steps += n
                job.total_steps += n
                point_steps += job.req.inst.points * n
            due = [j for j in active.values()
                   if (j.phase == "ground" and j.steps >= j.next_check)
                   or (j.phase == "real" and j.steps >= j.req.quench_steps)
                   or j.total_steps >= max_steps]
            if not due:
                continue
            obs = self.batch.observables([j.slot for j in due])
            now = time.perf_counter() - t0
            done = []
            for j in due:
                o = obs[j.slot]
                if j.phase == "ground":
                    j.next_check += convergence_interval(j.req.inst.dt)
                    converged = mu_converged(o["mu"], j.mu_prev, self.precision)
                    stalled = (j.mu_prev is not None and not converged and
                               j.watch.update(abs(o["mu"] - j.mu_prev)))
                    j.mu_prev = o["mu"]
                    if converged or stalled or j.total_steps >= max_steps:
                        j.ground_obs = o
                        j.converged, j.stalled = converged, stalled
                        if j.req.kind == "quench" and converged:
                            self.batch.set_params(j.slot, j.req.quench_g, gp.GP_REAL)
                            j.phase = "real"
                            j.steps = 0
                        else:
                            j.obs = o
                            done.append(j)
                else:
                    j.obs = o
                    done.append(j)
            for j in done:
                self.batch.remove(j.slot)
                del active[j.slot]
                results.append(Result(j.req, j.req.arrival, j.t_admit, now,
                                      j.total_steps - (j.steps if j.phase == "real" else 0),
                                      j.total_steps, j.obs, j.ground_obs,
                                      j.converged, j.stalled))
            if on_chunk:
                on_chunk(chunks, len(active), len(pending))
        wall = time.perf_counter() - t0
        return ServeStats(results, wall, point_steps, peak, chunks)


def solve_batch(instances, precision=gp.GP_C64, chunk=10, max_steps=200000, cap_bytes=None):
    """Ground states of many instances at once (all queued at t = 0)."""
    from .workloads import Request
    reqs = [Request(0.0, "ground", inst) for inst in instances]
    cap = cap_bytes or sum(gp.gp_batch_footprint(i.shape, precision) for i in instances) + (1 << 20)
    with Server(precision, cap, chunk) as s:
        return s.run(reqs, realtime=False, max_steps=max_steps)


def solve_sequential(requests, precision=gp.GP_C128, realtime=True, max_steps=200000,
                     stream=None):
    """The same requests one at a time on a single-grid context, in arrival
    order (plain FP64 by default); latency includes the wait for the server."""
    results = []
    point_steps = 0
    t0 = time.perf_counter()
    for req in sorted(requests, key=lambda r: r.arrival):
        if realtime:
            wait = req.arrival - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
        start = time.perf_counter() - t0
        shape, h, dt, g0, g1, g2, g = _instance_args(req.inst)
        k = convergence_interval(dt)
        with gp.Solver(shape, h, dt, g0, g1, g2, g, gp.GP_IMAG, precision, stream) as s:
            s.load(None)
            steps, mu_prev, watch = 0, None, StallWatch()
            while True:
                s.step(k)
                steps += k
                o = s.observables()
                converged = mu_converged(o["mu"], mu_prev, precision)
                stalled = (mu_prev is not None and not converged and
                           watch.update(abs(o["mu"] - mu_prev)))
                mu_prev = o["mu"]
                if converged or stalled or steps >= max_steps:
                    break
            ground_obs, ground_steps = o, steps
            if req.kind == "quench" and converged:
                s.set_params(req.quench_g, gp.GP_REAL)
                s.step(req.quench_steps)
                steps += req.quench_steps
                o = s.observables()
        point_steps += req.inst.points * steps
        results.append(Result(req, req.arrival, start, time.perf_counter() - t0, ground_steps,
                              steps, o, ground_obs, converged, stalled))
    wall = time.perf_counter() - t0
    return ServeStats(results, wall, point_steps, 0)


def shard_requests(requests, world, rank, precision=gp.GP_C64):
    """Requests of one rank when `world` GPUs serve one stream: independent
    problems need no exchange, so each goes whole to the rank with the least
    footprint so far (greedy in arrival order, ties to the lower rank)."""
    load = [0] * world
    mine = []
    for r in sorted(requests, key=lambda q: q.arrival):
        target = min(range(world), key=lambda k: (load[k], k))
        load[target] += r.inst.points * (16 if precision == gp.GP_C128 else 8)
        if target == rank:
            mine.append(r)
    return mine
