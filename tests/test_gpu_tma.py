"""GPU parity of the TMA-pipelined, windowed sweep path against the oracle
and against the exact one-line-per-thread path.  The window bound
|c'|^(C+1) (C = 16 complex64, 8 complex128) is checked by the library; cases
here sit inside it.  Shapes span several 128-line tiles, ragged tiles, odd
lengths (chunk tails) and 2D."""
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
    if nz > 1:
        a[0] = 0
    return a.astype(dtype)


def run(shape, h, dt, g, mode, steps, psi0, precision, path):
    with gp.Solver(shape, h, dt, *W3, g, mode, precision) as s:
        s.set_path(path)
        paths = s.paths()
        s.load(psi0)
        s.step(steps)
        return s.psi(), s.observables(), paths


SHAPES = [
    ((130, 33, 20), (0.1, 0.2, 0.15)),     # ragged tiles in y, z
    ((96, 200, 17), (0.12, 0.1, 0.2)),
    ((34, 18, 129), (0.2, 0.3, 0.1)),
    ((258, 130, 1), (0.08, 0.1, 1.0)),    # 2D
    ((6, 6, 6), (0.5, 0.5, 0.5)),
]


@pytest.mark.parametrize("shape,h", SHAPES)
@pytest.mark.parametrize("mode", [gp.GP_IMAG, gp.GP_REAL])
def test_tma_fp64_matches_oracle(shape, h, mode):
    require_gpu()
    dt, g = 2.5e-4, 5.0          # kappa <= 0.01: |c'|^9 < 2^-55
    psi0 = rand_state(shape, 31)
    got, _, paths = run(shape, h, dt, g, mode, 6, psi0, gp.GP_C128, gp.GP_PATH_TMA)
    assert all(p == gp.GP_PATH_TMA for p in paths[: 3 if shape[2] > 1 else 2])
    want = psi0.copy()
    oracle.step(oracle_params(shape, h, dt, W3, g, mode), want, 6)
    assert rel_l2(got, want) <= 1e-12


@pytest.mark.parametrize("shape,h", SHAPES)
@pytest.mark.parametrize("mode", [gp.GP_IMAG, gp.GP_REAL])
def test_tma_complex64_matches_exact_path_and_oracle(shape, h, mode):
    require_gpu()
    dt, g = 1e-3, 5.0
    psi0 = rand_state(shape, 32)
    tma, _, paths = run(shape, h, dt, g, mode, 6, psi0.astype(np.complex64), gp.GP_C64,
                        gp.GP_PATH_AUTO)
    even = shape[0] % 2 == 0
    assert (paths[0] == gp.GP_PATH_TMA) == even     # complex64 rows need 16-byte strides
    exact, _, _ = run(shape, h, dt, g, mode, 6, psi0.astype(np.complex64), gp.GP_C64,
                      gp.GP_PATH_EXACT)
    want = psi0.copy()
    oracle.step(oracle_params(shape, h, dt, W3, g, mode), want, 6)
    assert rel_l2(tma, exact) <= 2e-6
    assert rel_l2(tma, want) <= 2e-6
    assert rel_l2(exact, want) <= 2e-6


def test_tma_rejected_when_the_window_bound_fails():
    require_gpu()
    shape, h = (64, 64, 64), (0.05, 0.05, 0.05)
    with gp.Solver(shape, h, 0.05, *W3, 0.0, gp.GP_REAL, gp.GP_C64) as s:   # kappa = 5
        assert s.paths()[0] == gp.GP_PATH_EXACT
        with pytest.raises(gp.GPError) as e:
            s.set_path(gp.GP_PATH_TMA)
        assert e.value.code == gp.GP_EINVAL


def test_tma_complex64_1000_imaginary_steps_mu_within_1e6():
    """64^3 imaginary time through the TMA path: mu within 1e-6 of the FP64
    oracle after 1000 steps."""
    require_gpu()
    shape, h, dt, g = (64, 64, 64), (0.2, 0.2, 0.2), 0.002, 10.0
    with gp.Solver(shape, h, dt, *W3, g, gp.GP_IMAG, gp.GP_C64) as s:
        assert s.paths() == (gp.GP_PATH_TMA,) * 3
        s.load(None).step(1000)
        obs = s.observables()
    p = oracle_params(shape, h, dt, W3, g, 0)
    want = oracle.seed(p)
    oracle.step(p, want, 1000)
    ref = oracle.observables(p, want)
    assert abs(obs["mu"] - ref["mu"]) <= 1e-6 * ref["mu"]
    assert abs(obs["energy"] - ref["energy"]) <= 1e-6 * ref["energy"]


def test_tma_complex64_1000_real_time_steps_against_the_oracle():
    """The precision form's real-time regime (trap (1, 2, 4), g = 50, dt / 4h^2 =
    0.01 as at 512 x 512 x 256) on a 96 x 80 x 64 grid, 1000 steps from the
    Gaussian seed through the TMA path: mu, E, N and the rms widths within 1e-6
    of the FP64 oracle."""
    require_gpu()
    shape, h, dt, g, w = (96, 80, 64), (0.1, 0.1, 0.1), 4e-4, 50.0, (1.0, 2.0, 4.0)
    with gp.Solver(shape, h, dt, *w, g, gp.GP_REAL, gp.GP_C64) as s:
        assert s.paths() == (gp.GP_PATH_TMA,) * 3
        s.load(None).step(1000)
        obs = s.observables()
    p = oracle_params(shape, h, dt, w, g, 1)
    want = oracle.seed(p)
    oracle.step(p, want, 1000)
    ref = oracle.observables(p, want)
    for k, v in ref.items():
        assert abs(obs[k] - v) <= 1e-6 * abs(v), (k, obs[k], v)


@pytest.mark.parametrize("mode", [gp.GP_REAL, gp.GP_IMAG])
@pytest.mark.parametrize("precision,dtype,tol", [(gp.GP_C128, np.complex128, 1e-12),
                                                 (gp.GP_C64, np.complex64, 2e-6)])
def test_every_tile_shape_matches_oracle(precision, dtype, tol, mode):
    """Every tile shape, the tensor-memory ring shapes included, on ragged
    tiles (66 and 130 lines against 32 K per CTA) in both modes (imaginary
    time: the norm partials and the renormalisation too)."""
    require_gpu()
    shape, h, dt, g = (130, 66, 40), (0.1, 0.12, 0.15), 2.5e-4, 5.0
    psi0 = rand_state(shape, 41)
    want = psi0.copy()
    oracle.step(oracle_params(shape, h, dt, W3, g, mode), want, 5)
    for sh in range(gp.gp_tile_shapes(precision)):
        with gp.Solver(shape, h, dt, *W3, g, mode, precision) as s:
            gp.gp_set_option(s.ctx, gp.GP_OPT_TILE_SHAPE, sh)
            s.set_path(gp.GP_PATH_TMA)
            assert gp.gp_get_option(s.ctx, gp.GP_OPT_TILE_SHAPE) == sh
            s.load(psi0.astype(dtype)).step(5)
            assert rel_l2(s.psi(), want) <= tol, sh
