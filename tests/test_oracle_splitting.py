"""Pins of the oracle's Strang splitting and modulated g(t) = g + g1 cos(omega t)
(the symmetric splitting and the harmonic modulation of the scattering
length that the paper's cited applications use):

* the interval integral of g against numerical quadrature;
* Strang is time-reversible in real time (one step with dt, then one with
  -dt, returns the state to round-off) and the plain order is not;
* global order in dt in real time, with a modulated g: Strang 2, plain
  (Lie) 1;
* the time bookkeeping: n steps equal n1 + n2 steps started at step n1;
* real-time norm conservation with both extensions;
* imaginary time: both fixed points converge to the dt -> 0 ground state at
  first order (renormalising does not commute with the nonlinear step), the
  symmetric one with a much smaller error (renormalised before its second
  half step)."""
import numpy as np
import pytest

import oracle

W3 = (1.0, 1.5, 2.0)


def params(shape, h, dt, g, mode, w=W3):
    return oracle.Params.make(shape, h, dt, *w, g, mode)


def rand_state(shape, seed):
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    a = (rng.standard_normal((nz, ny, nx)) + 1j * rng.standard_normal((nz, ny, nx))) * 0.3
    a[:, :, 0] = 0
    a[:, 0, :] = 0
    if nz > 1:
        a[0] = 0
    return np.ascontiguousarray(a)


@pytest.mark.parametrize("g,g1,om,ta,tb", [(5.0, 3.0, 15.0, 0.1, 0.37), (0.0, 2.0, 0.0, 1.0, 1.5),
                                           (-2.0, 0.5, 40.0, 3.0, 3.001), (7.0, 0.0, 9.0, 0.0, 2.0)])
def test_g_integral_matches_quadrature(g, g1, om, ta, tb):
    from scipy.integrate import quad
    want, _ = quad(lambda t: g + g1 * np.cos(om * t), ta, tb, epsabs=1e-14, epsrel=1e-13)
    assert abs(oracle.g_integral(g, g1, om, ta, tb) - want) <= 1e-12 * max(1.0, abs(want))


@pytest.mark.parametrize("shape", [(12, 10, 9), (14, 11, 1)])
def test_strang_is_time_reversible_and_lie_is_not(shape):
    h, dt = (0.5, 0.6, 0.7), 0.05
    psi0 = rand_state(shape, 5)
    fwd, back = params(shape, h, dt, 8.0, 1), params(shape, h, -dt, 8.0, 1)
    s = oracle.step_ext(fwd, psi0.copy(), 1, strang=True)
    s = oracle.step_ext(back, s, 1, strang=True)
    assert np.linalg.norm(s - psi0) <= 1e-13 * np.linalg.norm(psi0)
    l_ = oracle.step_ext(fwd, psi0.copy(), 1, strang=False)
    l_ = oracle.step_ext(back, l_, 1, strang=False)
    assert np.linalg.norm(l_ - psi0) >= 1e-5 * np.linalg.norm(psi0)


def _order(strang, mode):
    shape, h, T = (20, 18, 16), (0.5, 0.55, 0.6), 0.4
    g, g1, om = 5.0, 3.0, 15.0

    def run(dt):
        p = params(shape, h, dt, g, mode)
        psi = oracle.seed(p)
        return oracle.step_ext(p, psi, int(round(T / dt)), 0, strang, g1, om)

    pr = params(shape, h, 0.02 / 32, g, mode)
    ref = oracle.step_ext(pr, oracle.seed(pr), int(round(T / (0.02 / 32))), 0, True, g1, om)
    errs = [np.linalg.norm(run(dt) - ref) for dt in (0.02, 0.01, 0.005)]
    return errs[0] / errs[1], errs[1] / errs[2]


def test_real_time_global_order_strang_two_lie_one():
    r1, r2 = _order(True, 1)
    assert 3.4 <= r1 <= 4.6 and 3.4 <= r2 <= 4.6, (r1, r2)
    l1, l2 = _order(False, 1)
    assert 1.6 <= l1 <= 2.4 and 1.6 <= l2 <= 2.4, (l1, l2)


@pytest.mark.parametrize("strang", [False, True])
def test_steps_split_at_any_step_index_give_the_same_state(strang):
    shape, h, dt = (10, 9, 8), (0.6, 0.6, 0.6), 0.01
    p = params(shape, h, dt, 4.0, 1)
    a = oracle.step_ext(p, rand_state(shape, 2), 10, 0, strang, 2.0, 30.0)
    b = oracle.step_ext(p, rand_state(shape, 2), 4, 0, strang, 2.0, 30.0)
    b = oracle.step_ext(p, b, 6, 4, strang, 2.0, 30.0)
    assert np.array_equal(a, b)
    c = oracle.step_ext(p, rand_state(shape, 2), 10, 3, strang, 2.0, 30.0)
    assert not np.array_equal(a, c)                 # the modulation phase matters


def test_real_time_norm_conserved_with_strang_and_modulation():
    shape, h, dt = (16, 14, 12), (0.5, 0.5, 0.5), 0.01
    p = params(shape, h, dt, 10.0, 1)
    psi = rand_state(shape, 9)
    n0 = oracle.norm(p, psi)
    oracle.step_ext(p, psi, 200, 0, True, 6.0, 12.0)
    assert abs(oracle.norm(p, psi) / n0 - 1) <= 200 * 1e-15


def test_imaginary_time_fixed_points_first_order_strang_ten_times_closer():
    shape, h, g = (16, 16, 16), (0.5, 0.5, 0.5), 10.0

    def mu(dt, strang):
        p = params(shape, h, dt, g, 0)
        psi = oracle.seed(p)
        oracle.step_ext(p, psi, int(round(25.0 / dt)), 0, strang)
        return oracle.observables(p, psi)["mu"]

    ref = mu(0.0025, True)
    es = [abs(mu(dt, True) - ref) for dt in (0.04, 0.02)]
    el = [abs(mu(dt, False) - ref) for dt in (0.04, 0.02)]
    assert 1.6 <= es[0] / es[1] <= 2.6, es
    assert 1.6 <= el[0] / el[1] <= 2.6, el
    assert es[0] < el[0] / 5 and es[1] < el[1] / 5, (es, el)
