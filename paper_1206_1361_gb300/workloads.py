"""Seeded synthetic workloads: grid shapes, spacings, trap frequencies, g, dt
and step counts of the benchmark and parity cases.  This module holds input
recipes only -- no step of the method's arithmetic -- so the CUDA path and
the CPU oracle can both draw their inputs from it.

The paper's runs used input files that are not available, so these
synthetic configurations stand in for them (program summaries v, xiv: the
fully anisotropic 3D imaginary- and real-time programs).
"""
import math
from dataclasses import dataclass, field


@dataclass(frozen=True)
class Case:
    name: str
    shape: tuple            # (nx, ny, nz)
    h: tuple                # (hx, hy, hz)
    dt: float
    trap: tuple             # (gamma, nu, lambda)
    g: float
    mode: int               # 0 imaginary, 1 real
    steps: int
    precision: int = 0      # 0 complex128, 1 complex64
    note: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def points(self):
        nx, ny, nz = self.shape
        return nx * ny * nz


# 64^3 on [-6.4, 6.4)^3, imaginary time from the normalised Gaussian seed.
SMALL_IMAG_64 = Case(
    name="imag3d-64^3-fp64", shape=(64, 64, 64), h=(0.2, 0.2, 0.2), dt=0.002,
    trap=(1.0, 1.5, 2.0), g=10.0, mode=0, steps=1000,
    note="imaginary time, 1000 steps, renormalised every step, Gaussian seed")

# 256^3 on [-12.8, 12.8)^3, real time after an imaginary-time ground state at
# g = 20, quenched to g = 18 (breathing); reports every 10 steps.
REAL_256 = Case(
    name="real3d-256^3-fp64", shape=(256, 256, 256), h=(0.1, 0.1, 0.1), dt=0.0005,
    trap=(1.0, math.sqrt(2.0), 2.0), g=18.0, mode=1, steps=2000,
    note="real time, 2000 steps, quench g 20 -> 18 from the imaginary-time ground state",
    extra={"g_ground": 20.0, "report_every": 10})

# 512 x 512 x 256, dx = 0.05, real time from the Gaussian seed at g = 50,
# complex64 psi and sweeps with FP64 reductions and tables.
PRECISION_512 = Case(
    name="real3d-512x512x256-c64", shape=(512, 512, 256), h=(0.05, 0.05, 0.05), dt=1e-4,
    trap=(1.0, 2.0, 4.0), g=50.0, mode=1, steps=1000, precision=1,
    note="real time from the Gaussian seed, complex64 psi, FP64 reductions")

# Grids whose xy-plane fits one CTA's shared memory (the fused x+y slab
# sweep): many small planes, psi larger than L2 (129 MB).
SLAB_C64 = Case(
    name="real3d-128x128x1024-c64", shape=(128, 128, 1024), h=(0.1, 0.1, 0.0125), dt=1e-4,
    trap=(1.0, 1.5, 2.0), g=10.0, mode=1, steps=200, precision=1,
    note="real time from the Gaussian seed, complex64, 128 x 128 planes")
SLAB_FP64 = Case(
    name="real3d-96x96x1024-fp64", shape=(96, 96, 1024), h=(0.1, 0.1, 0.0125), dt=1e-4,
    trap=(1.0, 1.5, 2.0), g=10.0, mode=1, steps=200,
    note="real time from the Gaussian seed, complex128, 96 x 96 planes")

CASES = {c.name: c for c in (SMALL_IMAG_64, REAL_256, PRECISION_512, SLAB_C64, SLAB_FP64)}


def convergence_interval(dt):
    """Steps between chemical-potential checks of an imaginary-time solve:
    max(10, ceil(0.05 / dt))."""
    return max(10, int(math.ceil(0.05 / dt)))


# ------------------------------------------------ batched and served problems
#
# Instance parameters are drawn with numpy's PCG64 from a fixed seed.  Spacing
# per axis: the box spans +-6 radii, R_k = max(R_TF,k, 1/sqrt(omega_k)) with
# the Thomas-Fermi radius R_TF,k = sqrt(2 mu_TF) / omega_k (mu_TF of the
# Thomas-Fermi density at unit norm), so h_k = 12 R_k / n_k; dt = 0.2 min h^2.

def thomas_fermi_mu(g, w):
    """Chemical potential of the Thomas-Fermi profile at N = 1 (input recipe:
    sets the box size).  3D: (15 g w1 w2 w3 / (4 pi))^(2/5) / 2; 2D:
    sqrt(g w1 w2 / pi)."""
    if len(w) == 3:
        return 0.5 * (15.0 * g * w[0] * w[1] * w[2] / (4.0 * math.pi)) ** 0.4
    return math.sqrt(g * w[0] * w[1] / math.pi)


def box_spacing(shape, trap, g):
    nx, ny, nz = shape
    w = trap if nz > 1 else trap[:2]
    mu = thomas_fermi_mu(g, w) if g > 0 else 0.0
    hs = []
    for n, wk in zip((nx, ny, nz)[:len(w)], w):
        r = max(math.sqrt(2.0 * mu) / wk, 1.0 / math.sqrt(wk))
        hs.append(12.0 * r / n)
    if nz == 1:
        hs.append(1.0)
    dt = 0.2 * min(hs[:len(w)]) ** 2
    return tuple(hs), dt


@dataclass(frozen=True)
class Instance:
    shape: tuple
    h: tuple
    dt: float
    trap: tuple
    g: float

    @property
    def points(self):
        return self.shape[0] * self.shape[1] * self.shape[2]


def batched_instances(seed=3, count=256):
    """256 imaginary-time problems: edges from {32, 48, 64, 96, 128}
    independently per axis, 25 % 2D (nz = 1), gamma, nu, lambda ~ U[0.5, 4],
    g ~ U[0, 200]."""
    import numpy as np
    rng = np.random.Generator(np.random.PCG64(seed))
    edges = (32, 48, 64, 96, 128)
    out = []
    for _ in range(count):
        two_d = rng.random() < 0.25
        nx, ny, nz = (int(rng.choice(edges)) for _ in range(3))
        if two_d:
            nz = 1
        trap = tuple(float(v) for v in rng.uniform(0.5, 4.0, 3))
        if two_d:
            trap = (trap[0], trap[1], 0.0)
        g = float(rng.uniform(0.0, 200.0))
        h, dt = box_spacing((nx, ny, nz), trap, g)
        out.append(Instance((nx, ny, nz), h, dt, trap, g))
    return out


@dataclass(frozen=True)
class Request:
    arrival: float          # seconds after the stream starts
    kind: str               # "ground" or "quench"
    inst: Instance
    quench_g: float = 0.0
    quench_steps: int = 0


def request_stream(seed=4, count=20000, rate=200.0):
    """Poisson arrivals (mean `rate` per second): 70 % ground-state solves,
    30 % quench runs.  Grid edges uniform over multiples of 16 in [48, 192]
    per axis, gamma, nu, lambda ~ U[0.5, 4], g ~ U[0, 500]; a quench continues
    the ground state in real time at g U[0.8, 1.2] for a multiple of 10 steps
    in [500, 5000]."""
    import numpy as np
    rng = np.random.Generator(np.random.PCG64(seed))
    edges = list(range(48, 193, 16))
    t = 0.0
    out = []
    for _ in range(count):
        t += float(rng.exponential(1.0 / rate))
        quench = rng.random() < 0.3
        shape = tuple(int(rng.choice(edges)) for _ in range(3))
        trap = tuple(float(v) for v in rng.uniform(0.5, 4.0, 3))
        g = float(rng.uniform(0.0, 500.0))
        h, dt = box_spacing(shape, trap, g)
        inst = Instance(shape, h, dt, trap, g)
        if quench:
            out.append(Request(t, "quench", inst, g * float(rng.uniform(0.8, 1.2)),
                               10 * int(rng.integers(50, 501))))
        else:
            out.append(Request(t, "ground", inst))
    return out
