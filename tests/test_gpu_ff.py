"""GPU parity of the float-float form (GP_CFF: psi as float-float pairs,
sweeps and calcnu in FP32 error-free arithmetic) against the FP64 oracle,
element by element, at the FP64 tolerances: relative L2 of psi <= 1e-12 for a
few steps of random states, <= 1e-10 (psi and every observable) over 1000
imaginary-time steps and over the 256^3 quench's 2000 real-time steps.

Shapes span several line tiles, ragged tiles, odd line lengths (chunk tails)
and 2D; the coupling dt / (4 h^2) stays where the back-substitution window
fits one 8-point chunk (max|c'|^9 < 2^-50), which gp_create checks."""
import numpy as np
import pytest

import oracle
from paper_1206_1361_gb300 import gp
from tests.gpu_util import oracle_params, rel_l2, require_gpu

pytestmark = pytest.mark.gpu

W3 = (1.0, 1.5, 2.0)


def rand_state(shape, seed):
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    a = (rng.standard_normal((nz, ny, nx)) + 1j * rng.standard_normal((nz, ny, nx))) * 0.3
    a[:, :, 0] = 0
    a[:, 0, :] = 0
    if nz > 1:
        a[0] = 0
    return a


def run_ff(shape, h, dt, w, g, mode, steps, psi0=None, shape_idx=None, every=None):
    with gp.Solver(shape, h, dt, w[0], w[1], w[2], g, mode, gp.GP_CFF) as s:
        if shape_idx is not None:
            gp.gp_set_option(s.ctx, gp.GP_OPT_TILE_SHAPE, shape_idx)
        s.load(psi0)
        if every:
            for _ in range(steps // every):
                s.step(every)
                obs = s.observables()
        else:
            s.step(steps)
            obs = s.observables()
        assert all(p == gp.GP_PATH_TMA for p in s.paths()[: 3 if shape[2] > 1 else 2])
        return s.psi(), obs


SHAPES = [
    ((130, 33, 20), (0.1, 0.2, 0.15)),     # ragged tiles in y, z
    ((131, 70, 9), (0.1, 0.15, 0.3)),      # odd nx
    ((96, 200, 17), (0.12, 0.1, 0.2)),
    ((34, 18, 129), (0.2, 0.3, 0.1)),
    ((258, 130, 1), (0.08, 0.1, 1.0)),    # 2D
    ((6, 6, 6), (0.5, 0.5, 0.5)),
    ((3, 3, 3), (0.9, 0.8, 0.7)),
]


@pytest.mark.parametrize("shape,h", SHAPES)
@pytest.mark.parametrize("mode", [gp.GP_IMAG, gp.GP_REAL])
def test_ff_random_state_steps_match_oracle(shape, h, mode):
    require_gpu()
    dt, g = 2.5e-4, 5.0          # kappa <= 0.01
    psi0 = rand_state(shape, 31)
    got, _ = run_ff(shape, h, dt, W3, g, mode, 6, psi0)
    assert got.dtype == np.complex128
    want = psi0.copy()
    oracle.step(oracle_params(shape, h, dt, W3, g, mode), want, 6)
    assert rel_l2(got, want) <= 1e-12


@pytest.mark.parametrize("shape_idx", range(7))
def test_ff_every_tile_shape_matches_oracle(shape_idx):
    require_gpu()
    assert gp.gp_tile_shapes(gp.GP_CFF) == 7
    shape, h, dt, g = (70, 45, 37), (0.15, 0.15, 0.15), 4e-4, 8.0
    psi0 = rand_state(shape, 5)
    got, _ = run_ff(shape, h, dt, W3, g, gp.GP_REAL, 5, psi0, shape_idx=shape_idx)
    want = psi0.copy()
    oracle.step(oracle_params(shape, h, dt, W3, g, gp.GP_REAL), want, 5)
    assert rel_l2(got, want) <= 1e-12


def test_ff_config_small_imaginary_time_1000_steps():
    """64^3 on [-6.4, 6.4)^3, (1, 1.5, 2), g = 10, dt = 0.002, 1000
    imaginary-time steps from the Gaussian seed: psi and every observable
    within 1e-10 of the oracle."""
    require_gpu()
    shape, h, dt, g = (64, 64, 64), (0.2, 0.2, 0.2), 0.002, 10.0
    got, obs = run_ff(shape, h, dt, W3, g, gp.GP_IMAG, 1000)
    p = oracle_params(shape, h, dt, W3, g, 0)
    want = oracle.seed(p)
    oracle.step(p, want, 1000)
    assert rel_l2(got, want) <= 1e-10
    ref = oracle.observables(p, want)
    for k, v in ref.items():
        assert abs(obs[k] - v) <= 1e-10 * abs(v), (k, obs[k], v)
    assert obs["step"] == 1000


def test_ff_quench_imag_to_real_with_reports():
    """Ground-state steps, the quench to real time, observables every 10
    steps (the replayed 10-step graph), against the oracle."""
    require_gpu()
    shape, h, dt = (48, 40, 36), (0.25, 0.25, 0.25), 0.002
    with gp.Solver(shape, h, dt, *W3, 20.0, gp.GP_IMAG, gp.GP_CFF) as s:
        s.load(None).step(150)
        s.set_params(18.0, gp.GP_REAL)
        for _ in range(10):
            s.step(10)
            obs = s.observables()
        got = s.psi()
    pi = oracle_params(shape, h, dt, W3, 20.0, 0)
    want = oracle.seed(pi)
    oracle.step(pi, want, 150)
    pr = oracle_params(shape, h, dt, W3, 18.0, 1)
    oracle.step(pr, want, 100)
    assert rel_l2(got, want) <= 1e-11
    ref = oracle.observables(pr, want)
    for k, v in ref.items():
        assert abs(obs[k] - v) <= 1e-11 * abs(v), (k, obs[k], v)


def test_ff_modulated_g_matches_oracle():
    require_gpu()
    shape, h, dt = (40, 36, 44), (0.3, 0.3, 0.3), 0.003
    psi0 = rand_state(shape, 8)
    with gp.Solver(shape, h, dt, *W3, 6.0, gp.GP_REAL, gp.GP_CFF) as s:
        s.set_modulation(3.0, 25.0).load(psi0).step(40)
        got = s.psi()
    want = psi0.copy()
    oracle.step_ext(oracle_params(shape, h, dt, W3, 6.0, 1), want, 40, 0, False, 3.0, 25.0)
    assert rel_l2(got, want) <= 1e-12


def test_ff_store_load_roundtrip_and_device_view():
    """complex128 in and out: the float-float pair holds each component to
    within 2^-48 of it; the device view exposes the pairs."""
    require_gpu()
    shape, h = (20, 24, 28), (0.4, 0.4, 0.4)
    psi0 = rand_state(shape, 3)
    with gp.Solver(shape, h, 0.01, *W3, 1.0, gp.GP_REAL, gp.GP_CFF) as s:
        s.load(psi0)
        back = s.psi()
        assert np.max(np.abs(back - psi0)) <= 2.0 ** -47 * np.max(np.abs(psi0))
        view = s.device_view().cpu().numpy()
        assert view.shape == (28, 24, 20, 4)
        re = view[..., 0].astype(np.float64) + view[..., 2]
        im = view[..., 1].astype(np.float64) + view[..., 3]
        assert np.array_equal(re + 1j * im, back)
        s.step(7)
        assert s.observables()["step"] == 7


@pytest.mark.parametrize("shape", [(37, 20, 9), (37, 21, 9), (31, 23, 1)])
def test_ff_load_from_a_device_buffer_zeroes_the_dirichlet_nodes(shape):
    """gp_load from a caller's device buffer splits it in place (the buffer is
    only read): the Dirichlet nodes come out zero, every other point within
    2^-47 of its complex128 value, and the caller's buffer is unchanged (line
    counts that fill the conversion's 4-line groups, a ragged last group, 2D)."""
    require_gpu()
    import torch
    nx, ny, nz = shape
    h = (0.4, 0.4, 0.4 if nz > 1 else 1.0)
    w = W3 if nz > 1 else (W3[0], W3[1], 0.0)
    rng = np.random.default_rng(12)
    a = rng.standard_normal((nz, ny, nx)) + 1j * rng.standard_normal((nz, ny, nx))
    dev = torch.from_numpy(a.copy()).cuda()
    with gp.Solver(shape, h, 0.01, *w, 1.0, gp.GP_REAL, gp.GP_CFF) as s:
        s.load(dev)
        back = s.psi()
        assert np.array_equal(dev.cpu().numpy(), a)
    want = a.copy()
    want[:, :, 0] = 0
    want[:, 0, :] = 0
    if nz > 1:
        want[0] = 0
    assert np.max(np.abs(back - want)) <= 2.0 ** -47 * np.max(np.abs(a))
    assert not back[:, :, 0].any() and not back[:, 0, :].any()
    if nz > 1:
        assert not back[0].any()


def test_ff_load_split_is_bit_exact():
    """The split of a complex128 input into float-float pairs (integer
    arithmetic on the bits): for 2^-97 <= |v| hi is the FP32 rounding of each
    component and lo the FP32 rounding of the exact remainder, bit for bit as
    numpy computes them -- over magnitudes up to 1e30, ties to even, values
    that round up to the next power of two and exact FP32 values; smaller
    values (down to 1e-300, and zeros) come within 2^-146 of v."""
    require_gpu()
    import torch
    shape, h = (33, 18, 10), (0.4, 0.4, 0.4)
    rng = np.random.default_rng(21)
    n = 10 * 18 * 33
    mag = 10.0 ** rng.uniform(-40, 30, 2 * n)
    v = rng.choice([-1.0, 1.0], 2 * n) * mag
    special = []
    for e in (-97, -96, -60, -1, 0, 1, 40, 99):
        b = 2.0 ** e
        special += [b, -b, b * (1 + 2.0 ** -24), b * (1 + 3 * 2.0 ** -24), b * (2 - 2.0 ** -53),
                    b * (1 + 2.0 ** -24 + 2.0 ** -52), -b * (1.5 + 2.0 ** -25), b * (1.75 - 2.0 ** -30)]
    special += [0.0, -0.0, 1e-300, -3e-39]
    a = (v[0::2] + 1j * v[1::2]).reshape(10, 18, 33)
    sp = np.array(special)
    for t in range(0, len(sp), 32):               # interior points (x, y, z >= 1)
        part = sp[t:t + 32]
        a.real[5, 7 + t // 32, 1:1 + len(part)] = part
        a.imag[6, 7 + t // 32, 1:1 + len(part)] = part
    a[:, :, 0] = 0
    a[:, 0, :] = 0
    a[0] = 0
    with gp.Solver(shape, h, 0.01, *W3, 1.0, gp.GP_REAL, gp.GP_CFF) as s:
        s.load(torch.from_numpy(a.copy()).cuda())
        view = s.device_view().cpu().numpy()
    assert (np.abs(a) < 2.0 ** -97).any() and (np.abs(a) >= 2.0 ** -97).any()
    for k, comp in ((0, a.real), (1, a.imag)):
        with np.errstate(under="ignore"):
            hi = comp.astype(np.float32)
            lo = (comp - hi.astype(np.float64)).astype(np.float32)
        big = np.abs(comp) >= 2.0 ** -97
        assert np.array_equal(view[..., k].view(np.uint32)[big], hi.view(np.uint32)[big])
        assert np.array_equal(view[..., k + 2].view(np.uint32)[big], lo.view(np.uint32)[big])
        got = view[..., k].astype(np.float64) + view[..., k + 2].astype(np.float64)
        assert np.max(np.abs(got - comp)[~big]) <= 2.0 ** -146


def test_ff_rejections():
    require_gpu()
    shape, h = (32, 32, 32), (0.3, 0.3, 0.3)
    with gp.Solver(shape, h, 0.004, *W3, 1.0, gp.GP_REAL, gp.GP_CFF) as s:
        for opt, val in ((gp.GP_OPT_SPLITTING, gp.GP_SPLIT_STRANG),
                         (gp.GP_OPT_SWEEP_PATH, gp.GP_PATH_EXACT),
                         (gp.GP_OPT_SWEEP_PATH, gp.GP_PATH_SLAB)):
            with pytest.raises(gp.GPError) as e:
                gp.gp_set_option(s.ctx, opt, val)
            assert e.value.code == gp.GP_EINVAL
    # kappa = 0.1: the window does not fit one chunk
    with pytest.raises(gp.GPError) as e:
        gp.gp_create(shape, h, 0.036, *W3, 1.0, gp.GP_REAL, gp.GP_CFF)
    assert e.value.code == gp.GP_EINVAL
    with pytest.raises(gp.GPError) as e:
        gp.gp_create_axial(64, 64, 0.2, 0.2, 0.001, 1.0, 1.0, 1.0, gp.GP_REAL, gp.GP_CFF)
    assert e.value.code == gp.GP_EINVAL


def test_ff_real_time_norm_drift():
    """Real time conserves N; the float-float roundings (~2^-48 per operation,
    a few dozen per point per step) keep the drift far below the 1e-10 bar."""
    require_gpu()
    shape, h, dt, g = (64, 64, 64), (0.2, 0.2, 0.2), 0.002, 10.0
    with gp.Solver(shape, h, dt, *W3, g, gp.GP_REAL, gp.GP_CFF) as s:
        s.load(None)
        n0 = s.observables()["norm"]
        s.step(1000)
        n1 = s.observables()["norm"]
    assert abs(n1 - n0) <= 1000 * 20 * 2.0 ** -48, n1 - n0
