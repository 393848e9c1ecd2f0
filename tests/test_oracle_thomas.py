"""Pins for the oracle's tridiagonal (Thomas) solve, the core of every
Crank-Nicolson sweep (calclux / calcluy / calcluz in the paper's "Summary of
revisions").  The oracle's recurrence is checked against LAPACK's dense solve
and against the LU factorisation its tables must represent."""
import numpy as np
import pytest

import oracle


def lap(m):
    return (np.diag(-2.0 * np.ones(m)) + np.diag(np.ones(m - 1), 1)
            + np.diag(np.ones(m - 1), -1))


KAPPAS = [0.0125, 0.05, 3.7, 0.0125j, 0.5j, 40.0j]


@pytest.mark.parametrize("m", [1, 2, 3, 7, 63, 255])
@pytest.mark.parametrize("kappa", KAPPAS)
def test_thomas_matches_dense_lu(m, kappa):
    rng = np.random.default_rng(1000 + m)
    b = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    a = np.eye(m) - complex(kappa) * lap(m)
    want = np.linalg.solve(a, b)
    got = oracle.thomas_solve(complex(kappa), b)
    assert np.linalg.norm(got - want) <= 1e-13 * np.linalg.norm(want)


@pytest.mark.parametrize("m", [1, 2, 5, 64])
@pytest.mark.parametrize("kappa", KAPPAS)
def test_tables_are_the_lu_factors(m, kappa):
    """(I - kappa L) = Lo @ Up with Up = bidiag(1/mult_i, -kappa) and
    Lo = unit lower bidiag with subdiagonal -kappa mult_{i-1}."""
    k = complex(kappa)
    cp, mult = oracle.thomas_tables(m, k)
    up = np.diag(1.0 / mult) + np.diag(-k * np.ones(m - 1), 1)
    lo = np.eye(m, dtype=complex) + np.diag(-k * mult[:-1], -1)
    a = np.eye(m) - k * lap(m)
    assert np.abs(lo @ up - a).max() <= 1e-14 * max(1.0, abs(k))
    # c'_i = -kappa mult_i
    assert np.allclose(cp, -k * mult, rtol=0, atol=1e-16)


def test_cprime_decays_for_small_kappa():
    """For |kappa| << 1 the elimination multipliers settle at |c'| ~ |kappa|;
    the GPU's windowed back substitution relies on this decay."""
    for k in (0.0125, 0.0125j):
        cp, _ = oracle.thomas_tables(255, k)
        assert np.all(np.abs(cp) < 1.1 * abs(k))
