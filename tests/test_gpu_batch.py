"""GPU tests of the batch engine (gp_batch_*): every instance against the
oracle, results identical alone and in a mix (the per-instance
decomposition and reductions depend only on the instance), continuous
add/remove between steps, quench, memory cap and size limits."""
import numpy as np
import pytest

import oracle
from paper_1206_1361_gb300 import gp
from tests.gpu_util import oracle_params, rel_l2, require_gpu

pytestmark = pytest.mark.gpu

# (shape, h, dt, trap, g, mode)
INSTANCES = [
    ((32, 48, 40), (0.3, 0.25, 0.2), 0.004, (1.0, 1.5, 2.0), 8.0, 0),
    ((70, 33, 1), (0.2, 0.3, 1.0), 0.003, (0.7, 1.2, 0.0), 5.0, 1),
    ((40, 24, 56), (0.25, 0.35, 0.2), 0.002, (2.0, 0.8, 1.5), 3.0, 1),
    ((96, 64, 1), (0.15, 0.2, 1.0), 0.002, (1.0, 2.0, 0.0), 40.0, 0),
    ((48, 48, 48), (0.25, 0.25, 0.25), 0.003, (1.0, 1.0, 1.0), 0.0, 0),
    # odd nx: y tiles move point by point, z tiles as 16-byte column pieces
    ((33, 20, 18), (0.3, 0.3, 0.35), 0.004, (1.2, 1.0, 1.4), 6.0, 1),
    # lines of 96 points or more take the 4-segment solve on 8-line tiles:
    # kappa_x = 1 (windows wider than a segment, clipped at the line's ends)
    ((100, 20, 1), (0.05, 0.3, 1.0), 0.01, (1.0, 1.0, 0.0), 5.0, 0),
    # 96-point y lines with odd nx (point by point), 96-point z lines (column
    # pieces), x rows of 130 points (pitch 130) and 98-point y lines in real
    # time
    ((33, 96, 20), (0.3, 0.1, 0.35), 0.002, (1.2, 1.0, 1.4), 6.0, 1),
    ((24, 20, 96), (0.3, 0.3, 0.08), 0.003, (1.0, 1.0, 1.5), 4.0, 0),
    ((130, 98, 1), (0.08, 0.1, 1.0), 5e-4, (1.0, 1.5, 0.0), 20.0, 1),
]


def rand_state(shape, seed):
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    a = (rng.standard_normal((nz, ny, nx)) + 1j * rng.standard_normal((nz, ny, nx))) * 0.3
    a[:, :, 0] = 0
    a[:, 0, :] = 0
    if nz > 1:
        a[0] = 0
    return a


def add(b, spec, psi=None, mode=None):
    shape, h, dt, w, g, m = spec
    return b.add(shape, h, dt, *w, g, mode=m if mode is None else mode, psi=psi)


def oracle_run(spec, psi0, steps):
    shape, h, dt, w, g, mode = spec
    p = oracle_params(shape, h, dt, w, g, mode)
    want = psi0.astype(np.complex128).copy()
    oracle.step(p, want, steps)
    return p, want


@pytest.mark.parametrize("precision,dtype,tol", [(gp.GP_C128, np.complex128, 1e-12),
                                                 (gp.GP_C64, np.complex64, 3e-6)])
def test_batch_instances_match_oracle(precision, dtype, tol):
    require_gpu()
    steps = 9
    with gp.Batch(precision) as b:
        slots, starts = [], []
        for n, spec in enumerate(INSTANCES):
            psi0 = rand_state(spec[0], 50 + n)
            starts.append(psi0)
            slots.append(add(b, spec, psi0.astype(dtype)))
        b.step(steps)
        obs = b.observables()
        for spec, slot, psi0 in zip(INSTANCES, slots, starts):
            p, want = oracle_run(spec, psi0, steps)
            got = b.psi(slot)
            assert rel_l2(got, want) <= tol, spec
            ref = oracle.observables(p, want)
            # FP64: 1e-10 on every observable; complex64: the form's bar,
            # mu within 1e-6, and N, E, rms within 1e-6 as well
            otol = 1e-10 if precision == gp.GP_C128 else 1e-6
            for k in ("norm", "mu", "energy", "rms_r"):
                assert abs(obs[slot][k] - ref[k]) <= otol * abs(ref[k]), (spec, k, obs[slot][k], ref[k])
            assert obs[slot]["step"] == steps


@pytest.mark.parametrize("precision", [gp.GP_C128, gp.GP_C64])
@pytest.mark.parametrize("which", [2, 3, 9])
def test_alone_and_in_the_mix_are_identical(precision, which):
    require_gpu()
    dtype = np.complex128 if precision == gp.GP_C128 else np.complex64
    spec = INSTANCES[which]
    psi0 = rand_state(spec[0], 7).astype(dtype)
    with gp.Batch(precision) as alone:
        s = add(alone, spec, psi0)
        alone.step(12)
        a = alone.psi(s)
        oa = alone.observables()[s]
    with gp.Batch(precision) as mix:
        for n, other in enumerate(INSTANCES):
            if other is not spec:
                add(mix, other, rand_state(other[0], 90 + n).astype(dtype))
        s = add(mix, spec, psi0)
        mix.step(5)
        extra = add(mix, INSTANCES[0])          # joins mid-run
        mix.step(7)
        mix.remove(extra)
        m = mix.psi(s)
        om = mix.observables()[s]
    assert np.array_equal(a, m)
    for k in ("norm", "mu", "energy", "rms_x", "rms_y", "rms_z"):
        assert oa[k] == om[k], k


def test_continuous_batching_leaves_running_instances_untouched():
    require_gpu()
    spec0, spec1 = INSTANCES[0], INSTANCES[3]
    with gp.Batch(gp.GP_C128) as b:
        s0 = add(b, spec0)
        b.step(4)
        s1 = add(b, spec1)
        b.step(6)
        b.remove(s0)
        s2 = add(b, spec0)                      # reuses the freed slot id
        assert s2 == s0
        b.step(3)
        got1 = b.psi(s1)
        assert b.observables()[s2]["step"] == 3
    p = oracle_params(*spec1)
    want = oracle.seed(p)
    oracle.step(p, want, 9)
    assert rel_l2(got1, want) <= 1e-12


@pytest.mark.parametrize("which", [0, 3])
def test_batch_quench_matches_oracle(which):
    """Ground state, then real time from it: the mode switch swaps the
    tables (and the segment-solve windows) of a running instance."""
    require_gpu()
    spec = INSTANCES[which]
    with gp.Batch(gp.GP_C128) as b:
        s = add(b, spec, mode=gp.GP_IMAG)
        b.step(30)
        b.set_params(s, 6.5, gp.GP_REAL)
        b.step(20)
        got = b.psi(s)
    shape, h, dt, w, g, _ = spec
    pi = oracle_params(shape, h, dt, w, g, 0)
    want = oracle.seed(pi)
    oracle.step(pi, want, 30)
    pr = oracle_params(shape, h, dt, w, 6.5, 1)
    oracle.step(pr, want, 20)
    assert rel_l2(got, want) <= 1e-12


def test_observables_of_a_subset_equal_the_full_pass():
    """gp_batch_observables_of: the listed slots only, each identical to its
    entry of the pass over every instance."""
    require_gpu()
    with gp.Batch(gp.GP_C64) as b:
        slots = [add(b, spec, rand_state(spec[0], 30 + n).astype(np.complex64))
                 for n, spec in enumerate(INSTANCES)]
        b.step(4)
        full = b.observables()
        pick = [slots[5], slots[0], slots[9]]
        part = b.observables(pick)
        assert list(part) == pick
        for s in pick:
            assert part[s] == full[s]
        assert b.observables([]) == {}
        b.remove(slots[2])
        with pytest.raises(gp.GPError) as e:
            b.observables([slots[1], slots[2]])
        assert e.value.code == gp.GP_EINVAL


def test_batch_cap_and_limits():
    require_gpu()
    need = gp.gp_batch_footprint((64, 64, 64), gp.GP_C64)
    with gp.Batch(gp.GP_C64, cap_bytes=int(need * 2.5)) as b:
        b.add((64, 64, 64), (0.2, 0.2, 0.2), 0.002, 1, 1, 1, 1.0)
        b.add((64, 64, 64), (0.2, 0.2, 0.2), 0.002, 1, 1, 1, 1.0)
        with pytest.raises(gp.GPError) as e:
            b.add((64, 64, 64), (0.2, 0.2, 0.2), 0.002, 1, 1, 1, 1.0)
        assert e.value.code == gp.GP_EFULL
        active, _, used = b.info()
        assert active == 2 and used == 2 * need
        with pytest.raises(gp.GPError) as e:
            b.add((600, 8, 8), (0.2, 0.2, 0.2), 0.002, 1, 1, 1, 1.0)
        assert e.value.code == gp.GP_EINVAL


def test_complex64_real_time_conserves_norm():
    """Real time is unitary: with the complex64 coefficients carried as hi +
    lo FP32 pairs computed for the FP32 kappa, the norm drift over 2000 steps
    stays at the level of random FP32 rounding (the plain FP32 roundings of
    the tables drifted ~3e-4 in 1000 steps)."""
    require_gpu()
    shape, h, dt = (128, 96, 64), (0.1, 0.12, 0.15), 2.5e-4
    with gp.Solver(shape, h, dt, 1.0, 2.0, 4.0, 50.0, gp.GP_REAL, gp.GP_C64) as s:
        s.load(None)
        n0 = s.observables()["norm"]
        s.step(2000)
        n1 = s.observables()["norm"]
        assert s.paths()[0] == gp.GP_PATH_TMA
    assert abs(n1 / n0 - 1) <= 1e-6
    with gp.Batch(gp.GP_C64) as b:
        slot = b.add((96, 64, 48), (0.15, 0.2, 0.25), 5e-4, 1.0, 2.0, 4.0, 50.0, gp.GP_REAL)
        n0 = b.observables()[slot]["norm"]
        b.step(2000)
        n1 = b.observables()[slot]["norm"]
    assert abs(n1 / n0 - 1) <= 1e-6


def test_dependency_wait_budget_times_out_and_recovers():
    """Failure detection of the persistent kernel without a fault: a
    dependency-wait budget of 0 makes the first wait that is not satisfied at
    once (a y-sweep item popped while its instance's x items are still
    running) give up; the kernel's warps leave, the next synchronising call
    reports GP_ETIMEOUT once, and with the budget restored a reloaded
    instance steps exactly like the oracle."""
    require_gpu()
    spec = ((128, 128, 64), (0.15, 0.15, 0.2), 0.002, (1.0, 1.5, 2.0), 10.0, 0)
    with gp.Batch(gp.GP_C128) as b:
        slot = add(b, spec)
        b.set_wait_ns(0).step(3)
        with pytest.raises(gp.GPError) as e:
            gp.gp_batch_sync(b.b)
        assert e.value.code == gp.GP_ETIMEOUT
        gp.gp_batch_sync(b.b)                      # reported once
        with pytest.raises(gp.GPError) as e:
            b.set_wait_ns(-1)
        assert e.value.code == gp.GP_EINVAL
        b.set_wait_ns(2 * 10 ** 9)
        gp.gp_batch_load(b.b, slot, None)
        b.step(5)
        got = b.psi(slot)
    shape, h, dt, w, g, mode = spec
    p = oracle_params(shape, h, dt, w, g, mode)
    want = oracle.seed(p)
    oracle.step(p, want, 5)
    assert rel_l2(got, want) <= 1e-12
