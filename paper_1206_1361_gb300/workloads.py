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

CASES = {c.name: c for c in (SMALL_IMAG_64, REAL_256, PRECISION_512)}


def convergence_interval(dt):
    """Steps between chemical-potential checks of an imaginary-time solve:
    max(10, ceil(0.05 / dt))."""
    return max(10, int(math.ceil(0.05 / dt)))
