"""GPU parity of the fused x+y slab sweep (GP_PATH_SLAB: a z-plane held in
shared memory -- by one CTA, or split at the middle row over a 2-CTA cluster
when one CTA cannot hold it -- calcnu and the x sweep
on its rows, the y sweep on its columns) against the oracle and against the
separate sweeps.  Shapes cover odd and even edges, nx != ny, planes that fill
several warps with a ragged last warp, both plane placements, the largest
planes that fit, and both modes; the symmetric splitting and a modulated g
ride on the slab's x sweep."""
import numpy as np
import pytest

import oracle
from paper_1206_1361_gb300 import gp
from tests.gpu_util import oracle_params, rel_l2, require_gpu

pytestmark = pytest.mark.gpu

W3 = (1.0, 1.5, 2.0)


def rand_state(shape, seed, dtype=np.complex128):
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    a = (rng.standard_normal((nz, ny, nx)) + 1j * rng.standard_normal((nz, ny, nx))) * 0.3
    a[:, :, 0] = 0
    a[:, 0, :] = 0
    a[0] = 0
    return a.astype(dtype)


def run(shape, h, dt, g, mode, steps, psi0, precision, path, strang=False, g1=0.0, om=0.0):
    with gp.Solver(shape, h, dt, *W3, g, mode, precision) as s:
        s.set_path(path)
        if strang:
            s.set_splitting(gp.GP_SPLIT_STRANG)
        if g1:
            s.set_modulation(g1, om)
        paths = s.paths()
        s.load(psi0)
        for n in steps:
            s.step(n)
        return s.psi(), s.observables(), paths


SHAPES = [
    ((40, 24, 12), (0.25, 0.3, 0.35)),
    ((33, 50, 9), (0.3, 0.2, 0.4)),       # odd nx, nx < ny: ragged last warp in both phases
    ((64, 64, 16), (0.2, 0.2, 0.3)),
    ((120, 7, 5), (0.1, 0.6, 0.5)),       # long rows, short columns
    ((3, 3, 3), (0.5, 0.5, 0.5)),         # one unknown per line
]


@pytest.mark.parametrize("shape,h", SHAPES)
@pytest.mark.parametrize("mode", [gp.GP_IMAG, gp.GP_REAL])
def test_slab_fp64_matches_oracle(shape, h, mode):
    require_gpu()
    dt, g = 0.004, 6.0
    psi0 = rand_state(shape, 41)
    got, _, paths = run(shape, h, dt, g, mode, [9], psi0, gp.GP_C128, gp.GP_PATH_SLAB)
    assert paths[:2] == (gp.GP_PATH_SLAB, gp.GP_PATH_SLAB)
    want = psi0.copy()
    oracle.step(oracle_params(shape, h, dt, W3, g, mode), want, 9)
    assert rel_l2(got, want) <= 1e-12


@pytest.mark.parametrize("shape,h", SHAPES)
@pytest.mark.parametrize("mode", [gp.GP_IMAG, gp.GP_REAL])
def test_slab_complex64_matches_oracle(shape, h, mode):
    require_gpu()
    dt, g = 0.004, 6.0
    psi0 = rand_state(shape, 42)
    got, _, _ = run(shape, h, dt, g, mode, [9], psi0.astype(np.complex64), gp.GP_C64,
                    gp.GP_PATH_SLAB)
    want = psi0.copy()
    oracle.step(oracle_params(shape, h, dt, W3, g, mode), want, 9)
    assert rel_l2(got, want) <= 3e-6


# planes larger than one CTA's shared memory: split over a 2-CTA cluster
SPLIT = [
    ((130, 120, 4), (0.1, 0.12, 0.3), gp.GP_C128),    # 120 x 131 x 16 B = 251 KB: fits only split
    ((131, 125, 3), (0.12, 0.1, 0.4), gp.GP_C128),    # odd nx and ny
    ((172, 171, 4), (0.08, 0.08, 0.4), gp.GP_C64),    # 171 x 173 x 8 B = 237 KB: odd ny
    ((180, 176, 3), (0.08, 0.08, 0.5), gp.GP_C64),    # 253 KB: fits only split
]


@pytest.mark.parametrize("shape,h,prec", SPLIT)
@pytest.mark.parametrize("mode", [gp.GP_IMAG, gp.GP_REAL])
def test_split_plane_matches_oracle(shape, h, prec, mode):
    require_gpu()
    dt, g = 0.002, 6.0
    dtype = np.complex128 if prec == gp.GP_C128 else np.complex64
    psi0 = rand_state(shape, 43)
    got, _, paths = run(shape, h, dt, g, mode, [5, 4], psi0.astype(dtype), prec, gp.GP_PATH_SLAB)
    assert paths[:2] == (gp.GP_PATH_SLAB, gp.GP_PATH_SLAB)
    want = psi0.copy()
    oracle.step(oracle_params(shape, h, dt, W3, g, mode), want, 9)
    assert rel_l2(got, want) <= (1e-12 if prec == gp.GP_C128 else 3e-6)


@pytest.mark.parametrize("mode", [gp.GP_IMAG, gp.GP_REAL])
def test_slab_agrees_with_separate_sweeps_over_many_steps(mode):
    require_gpu()
    shape, h, dt, g = (48, 40, 32), (0.25, 0.25, 0.25), 0.003, 15.0
    psi0 = rand_state(shape, 5)
    a, oa, _ = run(shape, h, dt, g, mode, [100, 100], psi0, gp.GP_C128, gp.GP_PATH_SLAB)
    b, ob, _ = run(shape, h, dt, g, mode, [100, 100], psi0, gp.GP_C128, gp.GP_PATH_EXACT)
    assert rel_l2(a, b) <= 1e-12
    for k in ("norm", "mu", "energy", "rms_r"):
        assert abs(oa[k] - ob[k]) <= 1e-11 * abs(ob[k]), k


@pytest.mark.parametrize("mode", [gp.GP_IMAG, gp.GP_REAL])
def test_slab_with_strang_and_modulated_g(mode):
    require_gpu()
    shape, h, dt = (36, 44, 20), (0.25, 0.25, 0.3), 0.003
    g, g1, om = 12.0, 9.0, 40.0
    psi0 = rand_state(shape, 6)
    got, _, _ = run(shape, h, dt, g, mode, [7, 13], psi0, gp.GP_C128, gp.GP_PATH_SLAB, True, g1, om)
    want = oracle.step_ext(oracle_params(shape, h, dt, W3, g, mode), psi0.copy(), 20, 0, True, g1, om)
    assert rel_l2(got, want) <= 1e-12


def test_largest_one_cta_fp64_plane_and_eligibility():
    require_gpu()
    # 120 x 120 complex128: 120 rows of 121 points x 16 B = 232320 B, just under 227 KB
    shape, h, dt, g = (120, 120, 4), (0.1, 0.1, 0.4), 5e-4, 3.0
    psi0 = rand_state(shape, 7)
    got, _, paths = run(shape, h, dt, g, gp.GP_REAL, [4], psi0, gp.GP_C128, gp.GP_PATH_SLAB)
    assert paths[:2] == (gp.GP_PATH_SLAB, gp.GP_PATH_SLAB)
    want = psi0.copy()
    oracle.step(oracle_params(shape, h, dt, W3, g, gp.GP_REAL), want, 4)
    assert rel_l2(got, want) <= 1e-12
    for shape in ((256, 256, 4), (64, 64, 1), (300, 8, 4)):   # too large, 2D, edge > 256
        with gp.Solver(shape, (0.1, 0.1, 0.1), 1e-3, *W3, 1.0, gp.GP_REAL, gp.GP_C128) as s:
            with pytest.raises(gp.GPError) as e:
                s.set_path(gp.GP_PATH_SLAB)
            assert e.value.code == gp.GP_EINVAL


def test_slab_saves_one_launch_per_step():
    require_gpu()
    with gp.Solver((32, 32, 32), (0.3, 0.3, 0.3), 1e-3, *W3, 1.0, gp.GP_IMAG, gp.GP_C64) as s:
        k0, _ = gp.gp_launches_per_step(s.ctx)
        s.set_path(gp.GP_PATH_SLAB)
        k1, _ = gp.gp_launches_per_step(s.ctx)
        assert k1 == k0 - 1
        assert gp.gp_get_option(s.ctx, gp.GP_OPT_SWEEP_PATH) == gp.GP_PATH_SLAB
