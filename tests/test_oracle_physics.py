"""Physics pins for the oracle: closed forms, exact separable solutions,
invariants and limits of the GP equation that a wrong kappa (scale or sign), a
wrong grid convention, a dropped term in the energy or a wrong renormalisation
would violate.  Program summaries v, vi (imaginary time: stationary states) and
xiv, xv (real time: dynamics) describe what the two propagations produce."""
import math

import numpy as np
import pytest

import oracle


def lap(m):
    return (np.diag(-2.0 * np.ones(m)) + np.diag(np.ones(m - 1), 1)
            + np.diag(np.ones(m - 1), -1))


def coords(n, h):
    return -0.5 * n * h + h * np.arange(n)


def step_matrix_1d(n, h, dt, w, mode):
    """One g = 0 step restricted to one axis: M = C diag(exp(-tau w^2 x^2 / 2))
    on the n-1 unknowns; the 3D g = 0 step is the Kronecker product of three."""
    m = n - 1
    tau = dt * (1j if mode else 1.0)
    k = tau / (4 * h * h)
    c = np.linalg.solve(np.eye(m) - k * lap(m), np.eye(m) + k * lap(m))
    x = coords(n, h)[1:]
    return c @ np.diag(np.exp(-tau * 0.5 * w * w * x * x)), x


def top_eigvec(mat):
    ev, vec = np.linalg.eig(mat)
    v = vec[:, np.argmax(np.abs(ev))]
    v = v / v[np.argmax(np.abs(v))]
    return np.real_if_close(v, tol=1e6)


def full(v):
    return np.concatenate([[0.0], v])


def energy_1d(v, x, h, w):
    f = np.concatenate([[0.0], v, [0.0]])
    return (0.5 * np.sum(np.abs(np.diff(f)) ** 2) / h ** 2
            + np.sum(0.5 * w * w * x * x * np.abs(v) ** 2)) / np.sum(np.abs(v) ** 2)


def run_to_ground_state(p, steps):
    psi = oracle.seed(p)
    oracle.step(p, psi, steps)
    return psi


# ---------------------------------------------------------------- g = 0

G0_SHAPE, G0_H, G0_DT, G0_W = (40, 36, 32), (0.25, 0.25, 0.25), 0.01, (1.0, 1.5, 2.0)


@pytest.fixture(scope="module")
def g0_ground():
    p = oracle.Params.make(G0_SHAPE, G0_H, G0_DT, *G0_W, 0.0, 0)
    return p, run_to_ground_state(p, 1600)


def test_g0_ground_state_is_outer_product_of_1d_eigenvectors(g0_ground):
    p, psi = g0_ground
    vecs = []
    for n, h, w in zip(G0_SHAPE, G0_H, G0_W):
        m, _ = step_matrix_1d(n, h, G0_DT, w, 0)
        vecs.append(full(top_eigvec(m)))
    want = np.einsum("k,j,i->kji", vecs[2], vecs[1], vecs[0])
    want = want / np.sqrt(np.prod(G0_H) * np.sum(want ** 2))
    assert np.linalg.norm(psi - want) <= 1e-10 * np.linalg.norm(want)


def test_g0_energy_is_sum_of_1d_energies_and_near_closed_form(g0_ground):
    p, psi = g0_ground
    obs = oracle.observables(p, psi)
    sep = 0.0
    for n, h, w in zip(G0_SHAPE, G0_H, G0_W):
        m, x = step_matrix_1d(n, h, G0_DT, w, 0)
        sep += energy_1d(top_eigvec(m), x, h, w)
    assert abs(obs["energy"] - sep) <= 1e-11
    assert abs(obs["mu"] - obs["energy"]) <= 1e-12          # g = 0: mu == E
    # continuum (gamma + nu + lambda)/2 with the 3-point stencil's O(h^2) shift
    closed = sum(G0_W) / 2 - G0_H[0] ** 2 * sum(w * w for w in G0_W) / 32
    assert abs(obs["energy"] - closed) <= 2e-4
    assert abs(obs["norm"] - 1.0) <= 1e-13


def test_g0_rms_sizes_approach_oscillator_lengths(g0_ground):
    p, psi = g0_ground
    obs = oracle.observables(p, psi)
    for key, w in zip(("rms_x", "rms_y", "rms_z"), G0_W):
        assert abs(obs[key] - 1 / math.sqrt(2 * w)) <= 0.01 / math.sqrt(2 * w)
    assert abs(obs["rms_r"] ** 2 - sum(obs[k] ** 2 for k in ("rms_x", "rms_y", "rms_z"))) < 1e-13


def test_g0_real_time_is_separable():
    """Real-time g = 0: psi_n = (M_x^n a) (x) (M_y^n b) (x) (M_z^n c) for a
    separable start, here a Gaussian of the wrong widths (it breathes)."""
    shape, h, dt, w = (24, 28, 20), (0.35, 0.3, 0.4), 0.01, (1.0, 1.4, 0.8)
    seed_p = oracle.Params.make(shape, h, dt, 2.0, 0.7, 1.5, 0.0, 1)
    p = oracle.Params.make(shape, h, dt, *w, 0.0, 1)
    psi = oracle.seed(seed_p)
    steps = 300
    oracle.step(p, psi, steps)
    parts = []
    for n, hk, wk, sk in zip(shape, h, w, (2.0, 0.7, 1.5)):
        m, x = step_matrix_1d(n, hk, dt, wk, 1)
        a = np.exp(-0.5 * sk * x * x)
        parts.append(full(np.linalg.matrix_power(m, steps) @ a))
    want = np.einsum("k,j,i->kji", parts[2], parts[1], parts[0])
    s0 = oracle.seed(seed_p)
    raw = np.einsum("k,j,i->kji", *[full(np.exp(-0.5 * sk * coords(n, hk)[1:] ** 2))
                                    for n, hk, sk in zip(shape[::-1], h[::-1], (1.5, 0.7, 2.0))])
    want = want * (s0[1, 1, 1] / raw[1, 1, 1])
    assert np.linalg.norm(psi - want) <= 1e-11 * np.linalg.norm(want)


# ---------------------------------------------------------- invariants

def test_real_time_conserves_norm_to_roundoff():
    shape, h = (32, 28, 24), (0.3, 0.3, 0.3)
    p = oracle.Params.make(shape, h, 0.002, 1.0, 1.5, 2.0, 50.0, 1)
    seed_p = oracle.Params.make(shape, h, 0.002, 1.3, 1.0, 2.5, 0.0, 1)
    psi = oracle.seed(seed_p)
    n0 = oracle.norm(p, psi)
    steps = 400
    oracle.step(p, psi, steps)
    # round-off only: a few ulps per step (a wrong kappa or phase drifts ~1e-3)
    assert abs(oracle.norm(p, psi) / n0 - 1) <= 1e-15 * steps


def test_ground_state_mirror_symmetry():
    shape, h = (48, 40, 32), (0.3, 0.3, 0.3)
    p = oracle.Params.make(shape, h, 0.005, 1.0, 1.5, 2.0, 20.0, 0)
    psi = run_to_ground_state(p, 300)
    core = psi[1:, 1:, 1:]
    scale = np.abs(core).max()
    for ax in range(3):
        assert np.abs(core - np.flip(core, axis=ax)).max() <= 1e-12 * scale


def test_imaginary_time_keeps_unit_norm_and_lowers_energy():
    shape, h = (32, 32, 32), (0.3, 0.3, 0.3)
    p = oracle.Params.make(shape, h, 0.004, 1.0, 1.5, 2.0, 10.0, 0)
    psi = oracle.seed(p)
    e_prev = oracle.observables(p, psi)["energy"]
    for _ in range(5):
        oracle.step(p, psi, 20)
        obs = oracle.observables(p, psi)
        assert abs(obs["norm"] - 1) <= 1e-13
        assert obs["energy"] <= e_prev + 1e-14
        e_prev = obs["energy"]


def test_real_time_ground_state_rotates_as_exp_minus_i_mu_t():
    """A stationary state evolves as psi(t) = exp(-i mu t) psi(0): pins the
    sign convention i dpsi/dt = H psi of the real-time propagation."""
    shape, h, dt = (32, 28, 24), (0.3, 0.3, 0.3), 0.002
    pi = oracle.Params.make(shape, h, dt, 1.0, 1.5, 2.0, 5.0, 0)
    psi = run_to_ground_state(pi, 3000)
    mu = oracle.observables(pi, psi)["mu"]
    pr = oracle.Params.make(shape, h, dt, 1.0, 1.5, 2.0, 5.0, 1)
    phi = psi.copy()
    steps = 200
    oracle.step(pr, phi, steps)
    # the projection on the start state; the Lie splitting makes the
    # imaginary-time fixed point stationary only up to O(dt), hence the slack
    ov = np.vdot(psi, phi) / np.vdot(psi, psi)
    assert abs(abs(ov) - 1) < 1e-3
    assert abs(np.angle(ov) + mu * dt * steps) < 0.02 * mu * dt * steps


def virial(p, psi):
    kin, pot, inter = oracle.energy_parts(p, psi)
    dims = 3 if p.nz > 1 else 2
    return (2 * kin - 2 * pot + dims * inter) / (kin + pot + inter)


def test_virial_theorem_converges_at_second_order():
    """2 E_kin - 2 E_pot + 3 E_int = 0 for the ground state (3D); the discrete
    residual (O(h^2) from the stencil plus O(dt) from the Lie splitting, with
    dt tied to h^2) must shrink ~4x when h halves (2D keeps the test cheap)."""
    res = []
    for h, n in ((0.4, 40), (0.2, 80)):
        dt = 0.25 * h * h
        p = oracle.Params.make((n, n, 1), (h, h, h), dt, 1.0, 1.5, 0.0, 30.0, 0)
        psi = run_to_ground_state(p, int(20 / dt))
        res.append(abs(virial(p, psi)))
    assert 3.5 < res[0] / res[1] < 4.5
    assert res[1] < 3e-3


def test_virial_3d():
    shape, h = (40, 40, 40), (0.3, 0.3, 0.3)
    p = oracle.Params.make(shape, h, 0.01, 1.0, 1.5, 2.0, 40.0, 0)
    psi = run_to_ground_state(p, 1500)
    assert abs(virial(p, psi)) < 1e-2


def test_thomas_fermi_limit_2d():
    """mu / mu_TF -> 1 from above as g grows, with 2D mu_TF = sqrt(g gamma nu
    / pi); the excess falls roughly like 1/g (the kinetic energy of the
    surface layer).  Started from the Thomas-Fermi profile to converge fast."""
    gamma, nu, n = 1.0, 1.5, 96
    excess = []
    for g in (300.0, 1e3, 3e3):
        mu_tf = math.sqrt(g * gamma * nu / math.pi)
        h = 2.5 * math.sqrt(2 * mu_tf) / min(gamma, nu) / n
        dt = min(0.25 * h * h, 0.05 / mu_tf)
        p = oracle.Params.make((n, n, 1), (h, h, h), dt, gamma, nu, 0.0, g, 0)
        x = coords(n, h)
        v = 0.5 * (gamma ** 2 * x[None, :] ** 2 + nu ** 2 * x[:, None] ** 2)
        psi = np.sqrt(np.maximum(mu_tf - v, 0) / g).astype(np.complex128)[None]
        psi[:, 0, :] = 0
        psi[:, :, 0] = 0
        psi /= math.sqrt(h * h * np.sum(np.abs(psi) ** 2))
        oracle.step(p, psi, 3 * int(2 / dt))
        excess.append(oracle.observables(p, psi)["mu"] / mu_tf - 1)
    assert excess[0] > excess[1] > excess[2] > 0
    assert excess[2] < 3e-3
    assert 5 < excess[0] / excess[2] < 12


def test_thomas_fermi_limit_3d():
    """3D: mu / mu_TF -> 1 from above as g grows, mu_TF = (15 g gamma nu lambda
    / (4 pi))^(2/5) / 2, on 64^3 boxes of +-1.25 R_TF started from the
    Thomas-Fermi profile: the excess falls monotonically, is below 3 % at
    g = 1e4 and shrinks by a factor 3 - 8 over the decade of g (the leading
    correction, the kinetic energy of the surface layer, scales like
    (omega / mu)^2 ln(mu / omega), ~4.5x here)."""
    w, n = (1.0, 1.25, 1.5), 64
    excess = []
    for g in (1e3, 3e3, 1e4):
        mu_tf = 0.5 * (15.0 * g * w[0] * w[1] * w[2] / (4 * math.pi)) ** 0.4
        h = 2.5 * math.sqrt(2 * mu_tf) / min(w) / n
        dt = min(0.25 * h * h, 0.05 / mu_tf)
        p = oracle.Params.make((n, n, n), (h, h, h), dt, *w, g, 0)
        x = coords(n, h)
        v = 0.5 * (w[0] ** 2 * x[None, None, :] ** 2 + w[1] ** 2 * x[None, :, None] ** 2 +
                   w[2] ** 2 * x[:, None, None] ** 2)
        psi = np.sqrt(np.maximum(mu_tf - v, 0) / g).astype(np.complex128)
        psi[:, :, 0] = 0
        psi[:, 0, :] = 0
        psi[0] = 0
        psi /= math.sqrt(h ** 3 * np.sum(np.abs(psi) ** 2))
        oracle.step(p, psi, 3 * int(2 / dt))
        excess.append(oracle.observables(p, psi)["mu"] / mu_tf - 1)
    assert excess[0] > excess[1] > excess[2] > 0
    assert excess[2] <= 0.03
    assert 3 < excess[0] / excess[2] < 8


# ------------------------------------------------ observables on a Gaussian

def test_observables_of_the_analytic_gaussian():
    """The seed is the continuum g = 0 ground state: rms_k = 1/sqrt(2 w_k),
    E_pot = E_kin = (gamma+nu+lambda)/4 and E_int = g/2 sqrt(gamma nu lambda)
    / (2 pi)^(3/2), the sums converging spectrally except the O(h^2) kinetic
    stencil, whose error must drop 4x when h halves."""
    w, g = (1.0, 1.5, 2.0), 7.0
    kin_err = []
    for h, n in ((0.25, 64), (0.125, 128)):
        p = oracle.Params.make((n, n, n), (h, h, h), 0.01, *w, g, 0)
        psi = oracle.seed(p)
        obs = oracle.observables(p, psi)
        kin, pot, inter = oracle.energy_parts(p, psi)
        assert abs(obs["norm"] - 1) < 1e-12       # 2M-term serial sum
        for key, wk in zip(("rms_x", "rms_y", "rms_z"), w):
            assert abs(obs[key] - 1 / math.sqrt(2 * wk)) < 1e-10
        assert abs(pot - sum(w) / 4) < 1e-10
        assert abs(inter - 0.5 * g * math.sqrt(np.prod(w)) / (2 * math.pi) ** 1.5) < 1e-10
        assert abs(obs["energy"] - (kin + pot + inter)) < 1e-12
        assert abs(obs["mu"] - (kin + pot + 2 * inter)) < 1e-12
        kin_err.append(abs(kin - sum(w) / 4))
    assert 3.5 < kin_err[0] / kin_err[1] < 4.5


def test_two_d_observables():
    w, g, h, n = (1.0, 2.0), 3.0, 0.2, 80
    p = oracle.Params.make((n, n, 1), (h, h, 5.0), 0.01, w[0], w[1], 9.0, g, 0)
    psi = oracle.seed(p)
    obs = oracle.observables(p, psi)
    assert abs(obs["norm"] - 1) < 1e-13
    assert obs["rms_z"] == 0.0
    assert abs(obs["rms_x"] - 1 / math.sqrt(2)) < 1e-10
    assert abs(obs["rms_y"] - 0.5) < 1e-10
    kin, pot, inter = oracle.energy_parts(p, psi)
    assert abs(pot - 0.75) < 1e-10
    assert abs(inter - 0.5 * g * math.sqrt(2.0) / (2 * math.pi)) < 1e-10
