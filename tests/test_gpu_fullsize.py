"""GPU parity at the benchmark's full sizes, in the launch configuration the
benchmark times (the 10-step graph, an observables report every 10 steps,
the automatic sweep path):

* 256^3 FP64 and float-float: imaginary-time ground-state steps at g = 20,
  then the quench to g = 18 in real time for 2000 steps, element by element
  against the oracle (relative L2 of psi <= 1e-10; observables <= 1e-10;
  norm drift of both within the rounding bound);
* 512 x 512 x 256 complex64 real time from the Gaussian seed against the FP64
  oracle (relative L2 bound derived from FP32 rounding per pass; mu <= 1e-6);
* the 256 batched instances advanced together, sampled instances against
  their solo runs (bitwise) and against the oracle.

The oracle runs on every host core; these are the slowest GPU tests."""
import numpy as np
import pytest

import oracle
from paper_1206_1361_gb300 import gp
from paper_1206_1361_gb300.workloads import PRECISION_512, REAL_256, batched_instances
from tests.gpu_util import oracle_params, rel_l2, require_gpu

pytestmark = pytest.mark.gpu


_ORACLE_256 = {}


def oracle_real_256(prep):
    """The oracle's 256^3 quench (ground-state prep steps at g = 20, then 2000
    real-time steps at g = 18): final psi, observables and the norm after the
    quench; computed once per session and shared by both precisions."""
    if prep not in _ORACLE_256:
        c = REAL_256
        pi = oracle_params(c.shape, c.h, c.dt, c.trap, c.extra["g_ground"], 0)
        want = oracle.seed(pi)
        oracle.step(pi, want, prep)
        pr = oracle_params(c.shape, c.h, c.dt, c.trap, c.g, 1)
        n0 = oracle.observables(pr, want)["norm"]
        oracle.step(pr, want, c.steps)
        _ORACLE_256[prep] = (want, oracle.observables(pr, want), n0)
    return _ORACLE_256[prep]


@pytest.mark.parametrize("precision", [gp.GP_C128, gp.GP_CFF])
def test_real_256_quench_2000_steps_matches_oracle(precision):
    """The benchmark's workload and launch configuration (the 10-step graph,
    an observables report every 10 steps) on the FP64 form and on the
    float-float form, against the same oracle run."""
    require_gpu()
    c = REAL_256
    prep, every = 100, c.extra["report_every"]
    with gp.Solver(c.shape, c.h, c.dt, *c.trap, c.extra["g_ground"], gp.GP_IMAG, precision) as s:
        s.load(None).step(prep)
        s.set_params(c.g, gp.GP_REAL)
        for _ in range(c.steps // every):
            s.step(every)
            obs = s.observables()
        got = s.psi()
    want, ref, n0 = oracle_real_256(prep)
    assert rel_l2(got, want) <= 1e-10
    for k in ("norm", "mu", "energy", "rms_x", "rms_y", "rms_z", "rms_r"):
        assert abs(obs[k] - ref[k]) <= 1e-10 * abs(ref[k]), (k, obs[k], ref[k])
    # Real time conserves N up to the unitarity defect of the rounded
    # arithmetic: the stored LU factors reproduce I - kappa L with a
    # Hermitian part off by ~2 ulp, which the Cayley step u = (2 (I - kappa
    # L)^-1 - I) psi turns into a norm change of up to ~4 ulp per sweep,
    # and the phase factor's modulus is off by ~2 ulp.  Those defects are
    # fixed, so on a slowly varying state they add up linearly in the steps
    # (both sides drift ~1.5e-15 per step here).  The float-float form's unit
    # is 2^-48 (tables split from FP64, hi + lo pairs) instead of 2^-52.
    unit = 2.0 ** -48 if precision == gp.GP_CFF else 2.0 ** -52
    bound = c.steps * (3 * 4 + 2) * unit
    assert abs(obs["norm"] - n0) <= bound and abs(ref["norm"] - n0) <= 2.0 ** -52 / unit * bound, \
        (obs["norm"] - n0, ref["norm"] - n0)


def test_precision_512_complex64_matches_fp64_oracle():
    """FP32 storage rounds psi once per pass (3 sweeps, with the phase fused
    into the first), 2^-24 relative each; over n steps the rounding errors
    add at most linearly: relative L2 <= n * 4 * 2^-23 (a factor 2 for the
    complex modulus).  mu within 1e-6 relative."""
    require_gpu()
    c = PRECISION_512
    steps = 20
    with gp.Solver(c.shape, c.h, c.dt, *c.trap, c.g, gp.GP_REAL, gp.GP_C64) as s:
        s.load(None)
        for _ in range(steps // 10):
            s.step(10)
            obs = s.observables()
        got = s.psi()
    assert got.dtype == np.complex64
    p = oracle_params(c.shape, c.h, c.dt, c.trap, c.g, 1)
    want = oracle.seed(p)
    oracle.step(p, want, steps)
    err = rel_l2(got.astype(np.complex128), want)
    assert err <= steps * 4 * 2.0 ** -23, err
    ref = oracle.observables(p, want)
    assert abs(obs["mu"] - ref["mu"]) <= 1e-6 * abs(ref["mu"]), (obs["mu"], ref["mu"])
    assert abs(obs["norm"] - ref["norm"]) <= 1e-6


def test_batched_256_instances_sampled_against_solo_and_oracle():
    require_gpu()
    insts = batched_instances()
    steps = 30
    sample = (0, 77, 255)
    with gp.Batch(gp.GP_C64) as b:
        slots = [b.add(i.shape, i.h, i.dt, *i.trap, i.g, gp.GP_IMAG) for i in insts]
        b.step(steps)
        mix = {k: b.psi(slots[k]) for k in sample}
        obs_mix = b.observables()
    for k in sample:
        i = insts[k]
        with gp.Batch(gp.GP_C64) as b:
            slot = b.add(i.shape, i.h, i.dt, *i.trap, i.g, gp.GP_IMAG)
            b.step(steps)
            alone = b.psi(slot)
        assert np.array_equal(alone, mix[k]), k
        p = oracle_params(i.shape, i.h, i.dt, i.trap, i.g, 0)
        want = oracle.seed(p)
        oracle.step(p, want, steps)
        assert rel_l2(mix[k].astype(np.complex128), want) <= steps * 4 * 2.0 ** -23, k
        ref = oracle.observables(p, want)
        assert abs(obs_mix[slots[k]]["mu"] - ref["mu"]) <= 1e-6 * max(1.0, abs(ref["mu"])), k


def test_real_256_strang_modulated_matches_oracle():
    """The symmetric splitting with g(t) = 18 + 4 cos(30 t) on the benchmark
    grid, 100 real-time steps from a short imaginary-time prep, through the
    graph: psi within 1e-10 of the oracle."""
    require_gpu()
    c = REAL_256
    with gp.Solver(c.shape, c.h, c.dt, *c.trap, c.extra["g_ground"], gp.GP_IMAG) as s:
        s.load(None).step(20)
        s.set_params(c.g, gp.GP_REAL).set_splitting(gp.GP_SPLIT_STRANG).set_modulation(4.0, 30.0)
        s.step(100)
        got = s.psi()
    pi = oracle_params(c.shape, c.h, c.dt, c.trap, c.extra["g_ground"], 0)
    want = oracle.seed(pi)
    oracle.step(pi, want, 20)
    pr = oracle_params(c.shape, c.h, c.dt, c.trap, c.g, 1)
    oracle.step_ext(pr, want, 100, 20, True, 4.0, 30.0)
    assert rel_l2(got, want) <= 1e-10


def test_axial_bench_case_matches_oracle():
    """The bench's axial case (1024 x 2048, h = 0.0125, trap (1, 4), g = 100,
    real time from the seed) on the segmented-window path, 30 steps."""
    require_gpu()
    nr, nz, h, dt, g = 1024, 2048, 0.0125, 1e-4, 100.0
    with gp.Solver.axial(nr, nz, h, h, dt, 1.0, 4.0, g, gp.GP_REAL) as s:
        assert gp.gp_sweep_paths(s.ctx)[:2] == (gp.GP_PATH_WINDOW, gp.GP_PATH_WINDOW)
        s.load(None).step(30)
        got, obs = s.psi(), s.observables()
    p = oracle.AxialParams.make(nr, nz, h, h, dt, 1.0, 4.0, g, 1)
    want = oracle.axial_seed(p)
    oracle.axial_step(p, want, 30)
    assert rel_l2(got, want) <= 1e-11
    ref = oracle.axial_observables(p, want)
    for k in ("norm", "mu", "energy", "rms_x", "rms_z"):
        assert abs(obs[k] - ref[k]) <= 1e-11 * abs(ref[k]), k


@pytest.mark.parametrize("shape,h", [((8192, 3, 3), (0.002, 1.0, 1.0)), ((3, 8192, 4), (1.0, 0.002, 0.9)),
                                     ((3, 4, 8192), (1.0, 0.9, 0.002))])
def test_longest_lines(shape, h):
    """Lines of the maximum edge (8192 points) along each axis."""
    require_gpu()
    rng = np.random.default_rng(6)
    nx, ny, nz = shape
    psi0 = (rng.standard_normal((nz, ny, nx)) + 1j * rng.standard_normal((nz, ny, nx))) * 0.3
    psi0[:, :, 0] = 0
    psi0[:, 0, :] = 0
    psi0[0] = 0
    for mode in (gp.GP_REAL, gp.GP_IMAG):
        p = oracle_params(shape, h, 0.001, (1.0, 1.5, 2.0), 3.0, mode)
        want = psi0.copy()
        oracle.step(p, want, 5)
        for prec, dtype, tol in ((gp.GP_C128, np.complex128, 1e-12),
                                 (gp.GP_C64, np.complex64, 5 * 4 * 2.0 ** -23)):
            with gp.Solver(shape, h, 0.001, 1.0, 1.5, 2.0, 3.0, mode, prec) as s:
                s.load(psi0.astype(dtype)).step(5)
                got = s.psi().astype(np.complex128)
            assert rel_l2(got, want) <= tol, (mode, prec)
