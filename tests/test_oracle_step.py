"""Brute-force pins for one full SSCN step of the oracle on tiny grids: the
pointwise potential/nonlinearity step (calcnu) and the three Crank-Nicolson
sweeps (calclux, calcluy, calcluz) are rebuilt as dense matrices acting on the
unknowns (Kronecker products of the per-axis Crank-Nicolson matrices) and
compared with the oracle's line-by-line Thomas sweeps."""
import numpy as np
import pytest

import oracle


def lap(m):
    return (np.diag(-2.0 * np.ones(m)) + np.diag(np.ones(m - 1), 1)
            + np.diag(np.ones(m - 1), -1))


def axis_coords(n, h):
    if n == 1:
        return np.zeros(1)
    return -0.5 * n * h + h * np.arange(n)


def cn_matrix(n, h, dt, mode):
    m = n - 1
    k = dt / (4 * h * h) * (1j if mode else 1.0)
    return np.linalg.solve(np.eye(m) - k * lap(m), np.eye(m) + k * lap(m))


def random_state(shape, seed):
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    psi = rng.standard_normal((nz, ny, nx)) + 1j * rng.standard_normal((nz, ny, nx))
    psi[:, :, 0] = 0
    psi[:, 0, :] = 0
    if nz > 1:
        psi[0, :, :] = 0
    return psi * 0.3


def dense_step(shape, h, dt, gamma, nu, lam, g, mode, psi):
    """calcnu as a pointwise numpy expression, then the sweeps as one dense
    Kronecker operator C_z (x) C_y (x) C_x on the flattened unknowns."""
    nx, ny, nz = shape
    x = axis_coords(nx, h[0])[None, None, :]
    y = axis_coords(ny, h[1])[None, :, None]
    z = axis_coords(nz, h[2])[:, None, None]
    v = 0.5 * (gamma ** 2 * x ** 2 + nu ** 2 * y ** 2 + lam ** 2 * z ** 2)
    tau = dt * (1j if mode else 1.0)
    psi = np.exp(-tau * (v + g * np.abs(psi) ** 2)) * psi
    zs = slice(1, None) if nz > 1 else slice(0, 1)
    unk = psi[zs, 1:, 1:]
    op = np.kron(cn_matrix(ny, h[1], dt, mode), cn_matrix(nx, h[0], dt, mode))
    if nz > 1:
        op = np.kron(cn_matrix(nz, h[2], dt, mode), op)
    out = np.zeros_like(psi)
    out[zs, 1:, 1:] = (op @ unk.reshape(-1)).reshape(unk.shape)
    if mode == 0:
        w = h[0] * h[1] * (h[2] if nz > 1 else 1.0)
        out /= np.sqrt(w * np.sum(np.abs(out) ** 2))
    return out


CASES = [((4, 5, 6), (0.7, 0.5, 0.4)), ((6, 7, 1), (0.5, 0.6, 1.0)),
         ((3, 3, 3), (1.0, 0.9, 0.8)), ((9, 4, 5), (0.3, 0.8, 0.45))]


@pytest.mark.parametrize("shape,h", CASES)
@pytest.mark.parametrize("mode", [0, 1])
def test_full_step_equals_dense_operator(shape, h, mode):
    dt, gamma, nu, lam, g = 0.05, 1.0, 1.5, 2.0, 3.0
    p = oracle.Params.make(shape, h, dt, gamma, nu, lam, g, mode)
    psi = random_state(shape, 7 + mode)
    want = psi.copy()
    got = psi.copy()
    for _ in range(3):
        want = dense_step(shape, h, dt, gamma, nu, lam, g, mode, want)
    oracle.step(p, got, 3)
    assert np.linalg.norm(got - want) <= 1e-13 * np.linalg.norm(want)


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("mode", [0, 1])
def test_single_sweep_acts_on_its_own_axis(axis, mode):
    shape, h, dt = (5, 6, 7), (0.4, 0.5, 0.6), 0.08
    p = oracle.Params.make(shape, h, dt, 1.0, 1.0, 1.0, 0.0, mode)
    psi = random_state(shape, 11)
    got = oracle.sweep(p, axis, psi.copy())
    n = shape[axis]
    c = cn_matrix(n, h[axis], dt, mode)
    want = psi.copy()
    # numpy axis of the (nz, ny, nx) array that the sweep runs along
    nax = 2 - axis
    moved = np.moveaxis(want, nax, -1)
    moved[..., 1:] = moved[..., 1:] @ c.T
    want = np.moveaxis(moved, -1, nax)
    # the sweep keeps the other axes' Dirichlet nodes at zero
    assert np.linalg.norm(got - want) <= 1e-13 * np.linalg.norm(want)


def test_nonlinear_step_pointwise():
    shape, h = (5, 4, 3), (0.5, 0.6, 0.7)
    for mode in (0, 1):
        p = oracle.Params.make(shape, h, 0.03, 1.2, 0.7, 2.5, 4.0, mode)
        psi = random_state(shape, 3)
        got = oracle.nonlinear(p, psi.copy())
        x = axis_coords(5, 0.5)[None, None, :]
        y = axis_coords(4, 0.6)[None, :, None]
        z = axis_coords(3, 0.7)[:, None, None]
        v = 0.5 * (1.2 ** 2 * x ** 2 + 0.7 ** 2 * y ** 2 + 2.5 ** 2 * z ** 2)
        tau = 0.03 * (1j if mode else 1.0)
        want = np.exp(-tau * (v + 4.0 * np.abs(psi) ** 2)) * psi
        assert np.allclose(got, want, rtol=1e-15, atol=1e-16)
        if mode == 1:
            assert np.allclose(np.abs(got), np.abs(psi), rtol=1e-15, atol=0)


def test_two_d_has_no_z_sweep():
    shape, h = (8, 9, 1), (0.5, 0.5, 123.0)
    p = oracle.Params.make(shape, h, 0.05, 1.0, 1.3, 99.0, 0.0, 0)
    psi = random_state(shape, 5)
    before = psi.copy()
    oracle.sweep(p, 2, psi)
    assert np.array_equal(psi, before)
