"""Pins of the oracle's axially symmetric discretisation (psi(rho, z); the
paper's axially symmetric programs, summaries vii, viii, xvi, xvii):

* the variable-coefficient tridiagonal solve against a dense LAPACK solve;
* one radial and one axial sweep against dense Crank-Nicolson operators built
  here from rho_{i +- 1/2} / rho_i directly;
* the g = 0 ground state is the outer product of the top eigenvectors of
  the radial and axial one-step matrices, and E -> gamma + lambda / 2;
* real time conserves the rho-weighted norm (and not the plain sum);
* a trap with gamma = nu solved on the Cartesian 3D grid gives the same
  mu, E and rms sizes to the discretisation error (an independent
  discretisation of the same problem);
* Gaussian moments converge at second order in h; the Thomas-Fermi limit;
* the symmetric splitting is time-reversible in real time."""
import numpy as np
import pytest

import oracle


def ax(nr, nz, hr, hz, dt, g, mode, gamma=1.0, lam=2.0):
    return oracle.AxialParams.make(nr, nz, hr, hz, dt, gamma, lam, g, mode)


def rand_state(nr, nz, seed):
    rng = np.random.default_rng(seed)
    a = (rng.standard_normal((nz, nr)) + 1j * rng.standard_normal((nz, nr))) * 0.3
    a[0] = 0
    return np.ascontiguousarray(a)


def radial_matrix(n, h):
    """T = h^2 L: (T psi)_i = [rho_{i+1/2}(psi_{i+1} - psi_i) - rho_{i-1/2}(psi_i - psi_{i-1})] / rho_i."""
    rho = (np.arange(n) + 0.5) * h
    T = np.zeros((n, n))
    for i in range(n):
        lo, hi = rho[i] - h / 2, rho[i] + h / 2
        T[i, i] = -(lo + hi) / rho[i]
        if i > 0:
            T[i, i - 1] = lo / rho[i]
        if i + 1 < n:
            T[i, i + 1] = hi / rho[i]
    return T


@pytest.mark.parametrize("m", [1, 2, 5, 64])
@pytest.mark.parametrize("kappa", [0.37 + 0j, 0.21j])
def test_variable_tridiagonal_solve_matches_lapack(m, kappa):
    rng = np.random.default_rng(m)
    a, c = rng.uniform(0.2, 1.0, m), rng.uniform(1.0, 1.8, m)
    b = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    A = np.eye(m, dtype=complex) * (1 + 2 * kappa)
    for i in range(m):
        if i > 0:
            A[i, i - 1] = -kappa * a[i]
        if i + 1 < m:
            A[i, i + 1] = -kappa * c[i]
    want = np.linalg.solve(A, b)
    got = oracle.tridiag_solve(kappa, a, c, b)
    assert np.linalg.norm(got - want) <= 1e-13 * np.linalg.norm(want)


@pytest.mark.parametrize("mode", [0, 1])
def test_sweeps_match_dense_operators(mode):
    nr, nz, hr, hz, dt = 9, 7, 0.4, 0.5, 0.03
    p = ax(nr, nz, hr, hz, dt, 0.0, mode)
    psi0 = rand_state(nr, nz, 3)
    kr = dt / (4 * hr * hr) * (1j if mode else 1)
    T = radial_matrix(nr, hr)
    Cr = np.linalg.solve(np.eye(nr) - kr * T, np.eye(nr) + kr * T)
    got = oracle.axial_sweep(p, 0, psi0.copy())
    assert np.linalg.norm(got - psi0 @ Cr.T) <= 1e-13 * np.linalg.norm(psi0)
    kz = dt / (4 * hz * hz) * (1j if mode else 1)
    L = np.diag(-2.0 * np.ones(nz - 1)) + np.diag(np.ones(nz - 2), 1) + np.diag(np.ones(nz - 2), -1)
    Cz = np.linalg.solve(np.eye(nz - 1) - kz * L, np.eye(nz - 1) + kz * L)
    want = psi0.copy()
    want[1:] = Cz @ psi0[1:]
    got = oracle.axial_sweep(p, 1, psi0.copy())
    assert np.linalg.norm(got - want) <= 1e-13 * np.linalg.norm(psi0)


def test_g0_ground_state_is_the_separable_eigenvector():
    nr, nz, hr, hz, dt, gam, lam = 24, 33, 0.25, 0.25, 0.01, 1.3, 2.1
    p = ax(nr, nz, hr, hz, dt, 0.0, 0, gam, lam)
    psi = oracle.axial_seed(p)
    oracle.axial_step(p, psi, 6000)
    rho = (np.arange(nr) + 0.5) * hr
    z = -nz * hz / 2 + np.arange(nz) * hz

    def top(C, v):
        w, V = np.linalg.eig(C @ np.diag(v))
        return np.real(V[:, np.argmax(np.abs(w))])

    kr, kz = dt / (4 * hr * hr), dt / (4 * hz * hz)
    T = radial_matrix(nr, hr)
    Cr = np.linalg.solve(np.eye(nr) - kr * T, np.eye(nr) + kr * T)
    er = top(Cr, np.exp(-dt * 0.5 * gam ** 2 * rho ** 2))
    L = np.diag(-2.0 * np.ones(nz - 1)) + np.diag(np.ones(nz - 2), 1) + np.diag(np.ones(nz - 2), -1)
    Cz = np.linalg.solve(np.eye(nz - 1) - kz * L, np.eye(nz - 1) + kz * L)
    ez = top(Cz, np.exp(-dt * 0.5 * lam ** 2 * z[1:] ** 2))
    want = np.zeros((nz, nr))
    want[1:] = np.outer(ez, er)
    want *= np.sign(want[nz // 2, 0]) / np.sqrt(2 * np.pi * hr * hz * np.sum(rho * want ** 2))
    got = np.real(psi) * np.sign(np.real(psi[nz // 2, 0]))
    assert np.linalg.norm(got - want) <= 1e-10 * np.linalg.norm(want)
    # E -> gamma + lambda / 2 at second order in h (same box, dt)
    errs = [abs(oracle.axial_observables(p, psi)["energy"] - (gam + lam / 2))]
    p2 = ax(2 * nr, 2 * nz, hr / 2, hz / 2, dt, 0.0, 0, gam, lam)
    psi2 = oracle.axial_seed(p2)
    oracle.axial_step(p2, psi2, 6000)
    errs.append(abs(oracle.axial_observables(p2, psi2)["energy"] - (gam + lam / 2)))
    assert 3.2 <= errs[0] / errs[1] <= 4.8, errs


@pytest.mark.parametrize("strang", [False, True])
def test_real_time_conserves_the_weighted_norm(strang):
    nr, nz = 20, 24
    p = ax(nr, nz, 0.3, 0.3, 0.01, 15.0, 1)
    psi = rand_state(nr, nz, 11)
    n0, s0 = oracle.axial_norm(p, psi), np.sum(np.abs(psi) ** 2)
    oracle.axial_step(p, psi, 300, 0, strang, 4.0, 9.0)
    assert abs(oracle.axial_norm(p, psi) / n0 - 1) <= 300 * 1e-15
    assert abs(np.sum(np.abs(psi) ** 2) / s0 - 1) >= 1e-6       # the weight matters


def test_matches_the_cartesian_solver_for_a_symmetric_trap():
    g, dt = 20.0, 0.005
    pa = ax(32, 64, 0.2, 0.2, dt, g, 0, 1.0, 2.0)
    psi = oracle.axial_seed(pa)
    oracle.axial_step(pa, psi, 2000)
    oa = oracle.axial_observables(pa, psi)
    pc = oracle.Params.make((64, 64, 64), (0.2, 0.2, 0.2), dt, 1.0, 1.0, 2.0, g, 0)
    pcart = oracle.seed(pc)
    oracle.step(pc, pcart, 2000)
    oc = oracle.observables(pc, pcart)
    for k in ("mu", "energy", "rms_x", "rms_z", "rms_r"):
        assert abs(oa[k] - oc[k]) <= 5e-3 * abs(oc[k]), (k, oa[k], oc[k])


def test_gaussian_moments_converge_at_second_order():
    gam, lam = 1.2, 1.7
    errs = []
    for h in (0.2, 0.1, 0.05):
        nr, nz = int(8 / h), int(12 / h)
        p = ax(nr, nz, h, h, 0.01, 0.0, 0, gam, lam)
        o = oracle.axial_observables(p, oracle.axial_seed(p))
        errs.append(abs(o["rms_x"] ** 2 - 1 / (2 * gam)))
        assert abs(o["rms_z"] ** 2 - 1 / (2 * lam)) <= 1e-12
        assert abs(o["norm"] - 1) <= 1e-12
    assert 3.5 <= errs[0] / errs[1] <= 4.5 and 3.5 <= errs[1] / errs[2] <= 4.5, errs


def test_thomas_fermi_limit():
    gam, lam = 1.0, 1.5
    ratios = []
    for g in (200.0, 1000.0, 5000.0):
        mu_tf = 0.5 * (15 * g * gam * gam * lam / (4 * np.pi)) ** 0.4
        r = np.sqrt(2 * mu_tf) / min(gam, lam) * 1.4
        h = r / 40
        p = ax(int(r / h), int(2 * r / h), h, h, 0.2 * h * h, g, 0, gam, lam)
        psi = oracle.axial_seed(p)
        oracle.axial_step(p, psi, 3000)
        ratios.append(oracle.axial_observables(p, psi)["mu"] / mu_tf)
    assert ratios[0] > ratios[1] > ratios[2] > 1.0, ratios
    assert ratios[2] - 1 <= 0.03, ratios


def test_strang_is_time_reversible():
    nr, nz, dt = 12, 14, 0.05
    psi0 = rand_state(nr, nz, 7)
    s = oracle.axial_step(ax(nr, nz, 0.4, 0.4, dt, 8.0, 1), psi0.copy(), 1, 0, True)
    s = oracle.axial_step(ax(nr, nz, 0.4, 0.4, -dt, 8.0, 1), s, 1, 0, True)
    assert np.linalg.norm(s - psi0) <= 1e-13 * np.linalg.norm(psi0)
