"""GPU parity of the symmetric (Strang) splitting and of the modulated
interaction g(t) = g + g1 cos(omega t) against the oracle's step_ext, on
random states and ragged multi-tile grids, through the 10-step graph and
plain launches, on every sweep path and both precisions."""
import numpy as np
import pytest

import oracle
from paper_1206_1361_gb300 import gp
from tests.gpu_util import oracle_params, rel_l2, require_gpu

pytestmark = pytest.mark.gpu

W3 = (1.0, 1.5, 2.0)
SHAPES = [
    ((33, 130, 17), (0.3, 0.1, 0.5)),
    ((200, 7, 140), (0.08, 1.2, 0.1)),
    ((65, 131, 1), (0.2, 0.15, 1.0)),
]


def rand_state(shape, seed):
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    a = (rng.standard_normal((nz, ny, nx)) + 1j * rng.standard_normal((nz, ny, nx))) * 0.3
    a[:, :, 0] = 0
    a[:, 0, :] = 0
    if nz > 1:
        a[0] = 0
    return np.ascontiguousarray(a)


def gpu_run(shape, h, dt, g, mode, chunks, psi0, strang, g1=0.0, om=0.0, precision=gp.GP_C128,
            path=None):
    dtype = np.complex128 if precision == gp.GP_C128 else np.complex64
    with gp.Solver(shape, h, dt, *W3, g, mode, precision) as s:
        if path is not None:
            s.set_path(path)
        s.set_splitting(gp.GP_SPLIT_STRANG if strang else gp.GP_SPLIT_LIE)
        if g1:
            s.set_modulation(g1, om)
        s.load(psi0.astype(dtype))
        for n in chunks:
            s.step(n)
        return s.psi(), s.observables()


def oracle_run(shape, h, dt, g, mode, steps, psi0, strang, g1=0.0, om=0.0):
    p = oracle_params(shape, h, dt, W3, g, mode)
    return oracle.step_ext(p, psi0.copy(), steps, 0, strang, g1, om)


@pytest.mark.parametrize("shape,h", SHAPES)
@pytest.mark.parametrize("mode", [gp.GP_REAL, gp.GP_IMAG])
def test_strang_matches_oracle(shape, h, mode):
    require_gpu()
    psi0 = rand_state(shape, 21)
    got, _ = gpu_run(shape, h, 0.004, 7.0, mode, [12], psi0, True)
    want = oracle_run(shape, h, 0.004, 7.0, mode, 12, psi0, True)
    assert rel_l2(got, want) <= 1e-12


@pytest.mark.parametrize("strang", [False, True])
@pytest.mark.parametrize("mode", [gp.GP_REAL, gp.GP_IMAG])
def test_modulated_g_matches_oracle_across_calls_and_graph_replays(strang, mode):
    require_gpu()
    shape, h, dt = (48, 40, 36), (0.25, 0.25, 0.25), 0.003
    g, g1, om = 12.0, 9.0, 40.0
    psi0 = rand_state(shape, 4)
    got, obs = gpu_run(shape, h, dt, g, mode, [7, 20, 3], psi0, strang, g1, om)
    want = oracle_run(shape, h, dt, g, mode, 30, psi0, strang, g1, om)
    assert rel_l2(got, want) <= 1e-12
    # mu and E with g(t) at t = 30 dt
    p = oracle_params(shape, h, dt, W3, g + g1 * np.cos(om * 30 * dt), mode)
    ref = oracle.observables(p, want)
    for k in ("norm", "mu", "energy", "rms_r"):
        assert abs(obs[k] - ref[k]) <= 1e-11 * abs(ref[k]), k
    assert obs["step"] == 30


def test_modulation_with_zero_omega_is_a_constant_shift():
    require_gpu()
    shape, h, dt = (40, 36, 32), (0.25, 0.25, 0.25), 0.004
    psi0 = rand_state(shape, 8)
    a, _ = gpu_run(shape, h, dt, 5.0, gp.GP_REAL, [15], psi0, True, 3.0, 0.0)
    want = oracle_run(shape, h, dt, 8.0, gp.GP_REAL, 15, psi0, True)
    assert rel_l2(a, want) <= 1e-12


@pytest.mark.parametrize("path", [gp.GP_PATH_TMA, gp.GP_PATH_EXACT])
@pytest.mark.parametrize("mode", [gp.GP_REAL, gp.GP_IMAG])
def test_complex64_strang_and_modulation(path, mode):
    require_gpu()
    shape, h, dt = (64, 48, 40), (0.2, 0.25, 0.3), 0.002
    psi0 = rand_state(shape, 13)
    steps = 24
    got, _ = gpu_run(shape, h, dt, 6.0, mode, [steps], psi0, True, 4.0, 25.0,
                     precision=gp.GP_C64, path=path)
    want = oracle_run(shape, h, dt, 6.0, mode, steps, psi0, True, 4.0, 25.0)
    assert got.dtype == np.complex64
    assert rel_l2(got.astype(np.complex128), want) <= steps * 4 * 2.0 ** -23


def test_launch_accounting_and_option_round_trip():
    require_gpu()
    with gp.Solver((24, 20, 18), (0.4, 0.4, 0.4), 0.01, *W3, 2.0, gp.GP_IMAG) as s:
        assert gp.gp_get_option(s.ctx, gp.GP_OPT_SPLITTING) == gp.GP_SPLIT_LIE
        base = gp.gp_launches_per_step(s.ctx)[0]
        s.set_splitting(gp.GP_SPLIT_STRANG)
        assert gp.gp_get_option(s.ctx, gp.GP_OPT_SPLITTING) == gp.GP_SPLIT_STRANG
        assert gp.gp_launches_per_step(s.ctx)[0] == base + 2
        s.set_modulation(1.0, 3.0)
        assert gp.gp_launches_per_step(s.ctx)[0] == base + 3
        with pytest.raises(gp.GPError):
            gp.gp_set_option(s.ctx, gp.GP_OPT_SPLITTING, 7)
        with pytest.raises(gp.GPError):
            gp.gp_set_modulation(s.ctx, float("nan"), 1.0)


def test_autotune_restores_the_modulation_clock():
    require_gpu()
    shape, h, dt = (64, 64, 48), (0.2, 0.2, 0.25), 0.002
    psi0 = rand_state(shape, 17)
    with gp.Solver(shape, h, dt, *W3, 10.0, gp.GP_REAL, gp.GP_C128) as s:
        s.set_splitting(gp.GP_SPLIT_STRANG).set_modulation(5.0, 30.0)
        s.load(psi0)
        s.step(10)
        gp.gp_autotune(s.ctx, 2)
        s.step(10)
        got = s.psi()
    want = oracle_run(shape, h, dt, 10.0, gp.GP_REAL, 20, psi0, True, 5.0, 30.0)
    assert rel_l2(got, want) <= 1e-12
