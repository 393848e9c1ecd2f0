"""gp_sweep_noalloc: one Crank-Nicolson sweep on a caller-owned device buffer
for callers that cannot allocate device memory (code running inside another
framework's operator with only the buffers it was handed, or loops that cannot
take cudaMalloc's device-wide synchronisation).  Its scratch lives in a static
device array, so this file checks it against the context path (gp_step) and
against the oracle's sweep on every axis and mode, on two calls in a row, and
that grids beyond the array are refused.  Collected
last on purpose: it must pass alone in a fresh process and after every other
test."""
import numpy as np
import pytest

import oracle
from paper_1206_1361_gb300 import gp
from tests.gpu_util import rel_l2, require_gpu

pytestmark = pytest.mark.gpu


def rand_state(shape, seed, dtype):
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    a = (rng.standard_normal((nz, ny, nx)) + 1j * rng.standard_normal((nz, ny, nx))) * 0.3
    a[:, :, 0] = 0
    a[:, 0, :] = 0
    if nz > 1:
        a[0] = 0
    return a.astype(dtype)


@pytest.mark.parametrize("precision,dtype", [(gp.GP_C128, np.complex128),
                                             (gp.GP_C64, np.complex64)])
@pytest.mark.parametrize("shape", [(48, 40, 36), (70, 33, 1)])
def test_noalloc_sweeps_match_gp_step_on_two_calls(precision, dtype, shape):
    """With no trap and g = 0 one real-time SSCN step of a context is exactly
    the x, y (and z) sweeps, so the two paths must agree."""
    require_gpu()
    import torch
    h, dt = (0.3, 0.25, 0.2), 0.01
    psi0 = rand_state(shape, 5, dtype)
    dev = torch.from_numpy(psi0.copy()).cuda()
    stream = torch.cuda.Stream()
    axes = (0, 1, 2) if shape[2] > 1 else (0, 1)
    with gp.Solver(shape, h, dt, 0.0, 0.0, 0.0, 0.0, gp.GP_REAL, precision) as s:
        s.set_path(gp.GP_PATH_EXACT)      # the kernel gp_sweep_noalloc is a variant of
        s.load(psi0)
        for _call in range(2):
            s.step(1)
            want = s.psi()
            for ax in axes:
                gp.gp_sweep_noalloc(dev, shape, ax, h[ax], dt, gp.GP_REAL, precision, stream)
            stream.synchronize()
            got = dev.cpu().numpy()
            assert rel_l2(got, want) <= 1e-12


@pytest.mark.parametrize("precision,dtype,tol", [
    (gp.GP_C128, np.complex128, 1e-12),
    # complex64: the FP32 roundings of a few dozen operations per point of one
    # sweep, 2^-24 each
    (gp.GP_C64, np.complex64, 32 * 2.0 ** -24)])
@pytest.mark.parametrize("mode", [gp.GP_IMAG, gp.GP_REAL])
def test_noalloc_each_axis_matches_the_oracle_sweep(precision, dtype, tol, mode):
    """Each axis, both modes: one sweep of gp_sweep_noalloc against the FP64
    oracle's sweep (calclux / calcluy / calcluz) of the same state, on two
    calls in a row (the second call reuses the array the first one wrote)."""
    require_gpu()
    import torch
    shape, h, dt = (40, 36, 30), (0.3, 0.25, 0.2), 0.01
    psi0 = rand_state(shape, 11, dtype)
    p = oracle.Params.make(shape, h, dt, 1.0, 1.0, 1.0, 0.0, mode)
    stream = torch.cuda.Stream()
    for ax in (0, 1, 2):
        want = psi0.astype(np.complex128)
        oracle.sweep(p, ax, want)
        for _call in range(2):
            dev = torch.from_numpy(psi0.copy()).cuda()
            gp.gp_sweep_noalloc(dev, shape, ax, h[ax], dt, mode, precision, stream)
            stream.synchronize()
            got = dev.cpu().numpy().astype(np.complex128)
            assert rel_l2(got, want) <= tol, (ax, mode)


def test_noalloc_imaginary_time_sweep_matches_dense_solve():
    require_gpu()
    import torch
    shape, h, dt = (12, 10, 9), 0.4, 0.05
    psi0 = rand_state(shape, 8, np.complex128)
    dev = torch.from_numpy(psi0.copy()).cuda()
    gp.gp_sweep_noalloc(dev, shape, 1, h, dt, gp.GP_IMAG, gp.GP_C128)
    torch.cuda.synchronize()
    m = shape[1] - 1
    lap = np.diag(-2.0 * np.ones(m)) + np.diag(np.ones(m - 1), 1) + np.diag(np.ones(m - 1), -1)
    k = dt / (4 * h * h)
    c = np.linalg.solve(np.eye(m) - k * lap, np.eye(m) + k * lap)
    want = psi0.copy()
    want[:, 1:, :] = np.einsum("ij,kjx->kix", c, psi0[:, 1:, :])
    assert rel_l2(dev.cpu().numpy(), want) <= 1e-12


def test_noalloc_rejects_grids_beyond_the_static_scratch():
    require_gpu()
    import torch
    dev = torch.zeros(8, dtype=torch.complex128, device="cuda")
    with pytest.raises(gp.GPError) as e:
        gp.gp_sweep_noalloc(dev, (128, 128, 128), 0, 0.1, 0.01, gp.GP_REAL, gp.GP_C128)
    assert e.value.code == gp.GP_EINVAL
    assert "static scratch" in gp.gp_last_error(None)
    with pytest.raises(gp.GPError):
        gp.gp_sweep_noalloc(dev, (8, 8, 1), 2, 0.1, 0.01, gp.GP_REAL, gp.GP_C128)
