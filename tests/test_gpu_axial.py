"""GPU parity of the axially symmetric form psi(rho, z) against the oracle:
random states on ragged grids in both modes, the seed and the observables,
a 1000-step imaginary-time ground state, the symmetric splitting with a
modulated g, weighted-norm conservation, load/store and argument checks."""
import numpy as np
import pytest

import oracle
from paper_1206_1361_gb300 import gp
from tests.gpu_util import rel_l2, require_gpu

pytestmark = pytest.mark.gpu

GRIDS = [(37, 50, 0.2, 0.15), (130, 21, 0.05, 0.4), (3, 3, 0.9, 0.8), (64, 200, 0.1, 0.07)]


def rand_state(nr, nz, seed):
    rng = np.random.default_rng(seed)
    a = (rng.standard_normal((nz, nr)) + 1j * rng.standard_normal((nz, nr))) * 0.3
    a[0] = 0
    return np.ascontiguousarray(a)


def params(nr, nz, hr, hz, dt, g, mode, gamma=1.0, lam=2.0):
    return oracle.AxialParams.make(nr, nz, hr, hz, dt, gamma, lam, g, mode)


def solver(nr, nz, hr, hz, dt, g, mode, gamma=1.0, lam=2.0):
    return gp.Solver.axial(nr, nz, hr, hz, dt, gamma, lam, g, mode)


@pytest.mark.parametrize("nr,nz,hr,hz", GRIDS)
@pytest.mark.parametrize("mode", [gp.GP_REAL, gp.GP_IMAG])
def test_random_state_steps_match_oracle(nr, nz, hr, hz, mode):
    require_gpu()
    dt, g = 0.004, 7.0
    psi0 = rand_state(nr, nz, 23)
    with solver(nr, nz, hr, hz, dt, g, mode) as s:
        s.load(psi0).step(12)
        got = s.psi()
    want = oracle.axial_step(params(nr, nz, hr, hz, dt, g, mode), psi0.copy(), 12)
    assert rel_l2(got, want) <= 1e-12


def test_seed_and_observables_match_oracle():
    require_gpu()
    nr, nz, hr, hz = 48, 80, 0.15, 0.12
    with solver(nr, nz, hr, hz, 0.01, 9.0, gp.GP_IMAG, 1.3, 2.2) as s:
        s.load(None)
        got, obs = s.psi(), s.observables()
    p = params(nr, nz, hr, hz, 0.01, 9.0, 0, 1.3, 2.2)
    want = oracle.axial_seed(p)
    assert rel_l2(got, want) <= 1e-13
    ref = oracle.axial_observables(p, want)
    for k, v in ref.items():
        assert abs(obs[k] - v) <= 1e-12 * max(1.0, abs(v)), k


def test_ground_state_1000_imaginary_steps():
    require_gpu()
    nr, nz, hr, hz, dt, g = 64, 128, 0.1, 0.1, 0.002, 20.0
    with solver(nr, nz, hr, hz, dt, g, gp.GP_IMAG) as s:
        s.load(None).step(1000)
        got, obs = s.psi(), s.observables()
    p = params(nr, nz, hr, hz, dt, g, 0)
    want = oracle.axial_seed(p)
    oracle.axial_step(p, want, 1000)
    assert rel_l2(got, want) <= 1e-10
    ref = oracle.axial_observables(p, want)
    for k, v in ref.items():
        assert abs(obs[k] - v) <= 1e-10 * abs(v), k


@pytest.mark.parametrize("mode", [gp.GP_REAL, gp.GP_IMAG])
def test_strang_and_modulation_match_oracle(mode):
    require_gpu()
    nr, nz, hr, hz, dt = 40, 66, 0.2, 0.2, 0.003
    psi0 = rand_state(nr, nz, 5)
    with solver(nr, nz, hr, hz, dt, 10.0, mode) as s:
        s.set_splitting(gp.GP_SPLIT_STRANG).set_modulation(6.0, 35.0)
        s.load(psi0)
        s.step(13)
        s.step(12)
        got = s.psi()
    want = oracle.axial_step(params(nr, nz, hr, hz, dt, 10.0, mode), psi0.copy(), 25, 0, True,
                             6.0, 35.0)
    assert rel_l2(got, want) <= 1e-12


def test_real_time_conserves_the_weighted_norm():
    require_gpu()
    with solver(50, 70, 0.2, 0.2, 0.005, 25.0, gp.GP_REAL) as s:
        s.load(rand_state(50, 70, 2))
        n0 = s.observables()["norm"]
        s.step(500)
        assert abs(s.observables()["norm"] / n0 - 1) <= 500 * 2e-15


def test_load_keeps_the_axis_and_zeroes_the_axial_boundary():
    require_gpu()
    a = np.ones((9, 8), np.complex128)
    with solver(8, 9, 0.5, 0.5, 0.01, 0.0, gp.GP_IMAG) as s:
        s.load(a)
        b = s.psi()
    assert np.all(b[0] == 0) and np.all(b[1:] == 1)


def test_arguments():
    require_gpu()
    with pytest.raises(gp.GPError):
        gp.gp_create_axial(2, 10, 0.1, 0.1, 0.01, 1, 1, 0, 0, gp.GP_C128)
    with pytest.raises(gp.GPError):
        gp.gp_create_axial(10, 10, 0.1, 0.1, 0.01, 1, 1, 0, 0, gp.GP_C64)
    with pytest.raises(gp.GPError):
        gp.gp_create_axial(10, 10, -0.1, 0.1, 0.01, 1, 1, 0, 0, gp.GP_C128)
    assert gp.gp_footprint_axial(100, 200) > 100 * 200 * 32


# grids long enough for the segmented-window sweeps (>= 2 cores per line)
WIN_GRIDS = [(300, 420, 0.05, 0.06), (700, 130, 0.02, 0.1)]


@pytest.mark.parametrize("nr,nz,hr,hz", WIN_GRIDS)
@pytest.mark.parametrize("mode", [gp.GP_REAL, gp.GP_IMAG])
def test_segmented_window_sweeps_match_oracle_and_exact(nr, nz, hr, hz, mode):
    require_gpu()
    dt, g = 0.004, 9.0
    psi0 = rand_state(nr, nz, 31)
    with solver(nr, nz, hr, hz, dt, g, mode) as s:
        assert gp.gp_sweep_paths(s.ctx)[:2] == (gp.GP_PATH_WINDOW, gp.GP_PATH_WINDOW)
        s.load(psi0).step(12)
        got = s.psi()
    with solver(nr, nz, hr, hz, dt, g, mode) as s:
        s.set_path(gp.GP_PATH_EXACT)
        assert gp.gp_sweep_paths(s.ctx)[:2] == (gp.GP_PATH_EXACT, gp.GP_PATH_EXACT)
        s.load(psi0).step(12)
        exact = s.psi()
    want = oracle.axial_step(params(nr, nz, hr, hz, dt, g, mode), psi0.copy(), 12)
    assert rel_l2(got, want) <= 1e-12
    assert rel_l2(got, exact) <= 1e-13


@pytest.mark.parametrize("mode", [gp.GP_REAL, gp.GP_IMAG])
def test_segmented_window_strang_modulation_and_norm(mode):
    require_gpu()
    nr, nz, hr, hz, dt = 320, 300, 0.04, 0.05, 0.002
    psi0 = rand_state(nr, nz, 8)
    with solver(nr, nz, hr, hz, dt, 20.0, mode) as s:
        s.set_splitting(gp.GP_SPLIT_STRANG).set_modulation(5.0, 40.0)
        s.load(psi0)
        n0 = s.observables()["norm"]
        s.step(17)
        got, obs = s.psi(), s.observables()
    want = oracle.axial_step(params(nr, nz, hr, hz, dt, 20.0, mode), psi0.copy(), 17, 0, True,
                             5.0, 40.0)
    assert rel_l2(got, want) <= 1e-12
    if mode == gp.GP_REAL:
        assert abs(obs["norm"] / n0 - 1) <= 17 * 2e-15
