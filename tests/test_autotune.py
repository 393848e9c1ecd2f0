"""Autotuner: picks an eligible kernel, leaves the state untouched, caches
the choice on disk and reapplies it."""
import numpy as np
import pytest

import oracle
from paper_1206_1361_gb300 import autotune, gp
from tests.gpu_util import oracle_params, rel_l2, require_gpu


def test_problem_key_separates_what_decides_the_kernel():
    k1 = autotune.problem_key((64, 64, 64), (0.2, 0.2, 0.2), 0.002, 1, 0)
    assert k1 != autotune.problem_key((64, 64, 64), (0.2, 0.2, 0.2), 0.002, 0, 0)
    assert k1 != autotune.problem_key((64, 64, 64), (0.2, 0.2, 0.2), 0.02, 1, 0)
    assert autotune.problem_key((64, 64, 64), (0.2, 0.2, 0.2), 0.0021, 1, 0) == \
        autotune.problem_key((64, 64, 64), (0.2, 0.2, 0.2), 0.00210001, 1, 0)
    assert "64x64x1" in autotune.problem_key((64, 64, 1), (0.2, 0.2, 1.0), 0.002, 1, 1)


@pytest.mark.gpu
def test_autotune_keeps_state_and_caches(tmp_path):
    require_gpu()
    shape, h, dt, w = (96, 64, 48), (0.15, 0.2, 0.25), 0.001, (1.0, 1.5, 2.0)
    rng = np.random.default_rng(2)
    psi0 = (rng.standard_normal((48, 64, 96)) + 1j * rng.standard_normal((48, 64, 96))) * 0.3
    psi0[:, :, 0] = psi0[:, 0, :] = psi0[0] = 0
    cache = str(tmp_path / "tune.json")
    for prec, dtype, tol in ((gp.GP_C64, np.complex64, 3e-6), (gp.GP_C128, np.complex128, 1e-12)):
        with gp.Solver(shape, h, dt, *w, 4.0, gp.GP_REAL, prec) as s:
            s.load(psi0.astype(dtype)).step(3)
            before = s.psi()
            first = autotune.tune(s, h, dt, gp.GP_REAL, steps=3, path=cache)
            assert not first["cached"] and first["path"] in (gp.GP_PATH_EXACT, gp.GP_PATH_TMA, gp.GP_PATH_SLAB)
            assert np.array_equal(s.psi(), before)
            assert s.observables()["step"] == 3
            s.step(4)
            got = s.psi()
        want = psi0.copy()
        oracle.step(oracle_params(shape, h, dt, w, 4.0, 1), want, 7)
        assert rel_l2(got, want) <= tol
        with gp.Solver(shape, h, dt, *w, 4.0, gp.GP_REAL, prec) as s:
            again = autotune.tune(s, h, dt, gp.GP_REAL, path=cache)
            assert again["cached"] and again["path"] == first["path"]
            assert gp.gp_get_option(s.ctx, gp.GP_OPT_TILE_SHAPE) == first["shape"]
