"""FP64 CPU oracle for the split-step Crank-Nicolson GP solver.

TEST INFRASTRUCTURE ONLY: the checker that the CUDA path is compared against.
Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg import this package.  It shares no code with the CUDA library;
the C source (``sscn_ref.c``) states the discretisation of every step.

Arrays are numpy complex128, C-contiguous, shape (nz, ny, nx) (x fastest).
"""
import ctypes
import os

import numpy as np

from . import build as _build

__all__ = ["Params", "lib", "coord", "seed", "step", "step_ext", "nonlinear",
           "nonlinear_part", "g_integral", "sweep",
           "norm", "observables", "energy_parts", "sums", "thomas_tables",
           "thomas_solve", "set_threads", "get_threads", "AxialParams", "axial_seed",
           "axial_step", "axial_sweep", "axial_nonlinear_part", "axial_norm",
           "axial_observables", "axial_rho", "axial_weights", "tridiag_solve"]


class Params(ctypes.Structure):
    """Mirror of ``ref_params`` in sscn_ref.c."""
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("nz", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("hx", ctypes.c_double), ("hy", ctypes.c_double),
                ("hz", ctypes.c_double), ("dt", ctypes.c_double),
                ("gamma", ctypes.c_double), ("nu", ctypes.c_double),
                ("lambda_", ctypes.c_double), ("g", ctypes.c_double)]

    @classmethod
    def make(cls, shape, h, dt, gamma, nu, lam, g, mode):
        """shape = (nx, ny, nz); h = (hx, hy, hz); mode 0 imaginary, 1 real."""
        nx, ny, nz = shape
        hx, hy, hz = h
        return cls(nx, ny, nz, mode, hx, hy, hz, dt, gamma, nu, lam, g)

    @property
    def shape3(self):
        return (self.nz, self.ny, self.nx)


class AxialParams(ctypes.Structure):
    """Mirror of ``ref_axial`` in sscn_ref.c (axially symmetric psi(rho, z))."""
    _fields_ = [("nr", ctypes.c_int32), ("nz", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("hr", ctypes.c_double), ("hz", ctypes.c_double),
                ("dt", ctypes.c_double), ("gamma", ctypes.c_double),
                ("lambda_", ctypes.c_double), ("g", ctypes.c_double)]

    @classmethod
    def make(cls, nr, nz, hr, hz, dt, gamma, lam, g, mode):
        return cls(nr, nz, mode, 0, hr, hz, dt, gamma, lam, g)

    @property
    def shape2(self):
        return (self.nz, self.nr)


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER(Params)
        A = ctypes.POINTER(AxialParams)
        vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        sig = {
            "ref_set_threads": (None, [ctypes.c_int]),
            "ref_get_threads": (ctypes.c_int, []),
            "ref_coord": (dbl, [i32, dbl, i32]),
            "ref_thomas_tables": (None, [i32, dbl, dbl, vp, vp]),
            "ref_thomas_solve": (None, [i32, dbl, dbl, vp, vp, vp]),
            "ref_nonlinear": (None, [P, vp]),
            "ref_nonlinear_part": (None, [P, vp, dbl, dbl]),
            "ref_g_integral": (dbl, [dbl, dbl, dbl, dbl, dbl]),
            "ref_step_ext": (None, [P, vp, i64, i64, i32, dbl, dbl]),
            "ref_sweep": (None, [P, i32, vp]),
            "ref_norm": (dbl, [P, vp]),
            "ref_scale": (None, [P, vp, dbl]),
            "ref_step": (None, [P, vp, i64]),
            "ref_seed": (None, [P, vp]),
            "ref_sums": (None, [P, vp, vp]),
            "ref_energy_parts": (None, [P, vp, vp]),
            "ref_observables": (None, [P, vp, vp]),
            "ref_axial_rho": (dbl, [dbl, i32]),
            "ref_axial_weights": (None, [i32, vp, vp]),
            "ref_tridiag_solve": (None, [i32, dbl, dbl, vp, vp, vp, vp, vp]),
            "ref_axial_nonlinear_part": (None, [A, vp, dbl, dbl]),
            "ref_axial_sweep": (None, [A, i32, vp]),
            "ref_axial_norm": (dbl, [A, vp]),
            "ref_axial_step_ext": (None, [A, vp, i64, i64, i32, dbl, dbl]),
            "ref_axial_seed": (None, [A, vp]),
            "ref_axial_observables": (None, [A, vp, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(p, psi):
    if psi.dtype != np.complex128 or not psi.flags.c_contiguous:
        raise TypeError("psi must be C-contiguous complex128")
    if psi.shape != p.shape3:
        raise ValueError("psi shape %s != (nz, ny, nx) %s" % (psi.shape, p.shape3))


def set_threads(n):
    lib().ref_set_threads(int(n))


def get_threads():
    return lib().ref_get_threads()


def coord(n, h, i):
    return lib().ref_coord(n, h, i)


def seed(p):
    psi = np.zeros(p.shape3, np.complex128)
    lib().ref_seed(ctypes.byref(p), _ptr(psi))
    return psi


def step(p, psi, n):
    """n SSCN steps in place."""
    _check(p, psi)
    lib().ref_step(ctypes.byref(p), _ptr(psi), int(n))
    return psi


def step_ext(p, psi, n, step0=0, strang=False, g1=0.0, omega=0.0):
    """n steps in place from step index step0 with g(t) = p.g + g1 cos(omega t)
    and the Lie (strang=False) or Strang splitting."""
    _check(p, psi)
    lib().ref_step_ext(ctypes.byref(p), _ptr(psi), int(n), int(step0), int(bool(strang)),
                       float(g1), float(omega))
    return psi


def g_integral(g, g1, omega, ta, tb):
    """Integral of g + g1 cos(omega t) over [ta, tb]."""
    return lib().ref_g_integral(float(g), float(g1), float(omega), float(ta), float(tb))


def nonlinear_part(p, psi, frac, G):
    """Pointwise step theta = frac dt V + G |psi|^2."""
    _check(p, psi)
    lib().ref_nonlinear_part(ctypes.byref(p), _ptr(psi), float(frac), float(G))
    return psi


def nonlinear(p, psi):
    _check(p, psi)
    lib().ref_nonlinear(ctypes.byref(p), _ptr(psi))
    return psi


def sweep(p, axis, psi):
    _check(p, psi)
    lib().ref_sweep(ctypes.byref(p), int(axis), _ptr(psi))
    return psi


def norm(p, psi):
    _check(p, psi)
    return lib().ref_norm(ctypes.byref(p), _ptr(psi))


def sums(p, psi):
    _check(p, psi)
    out = np.zeros(9)
    lib().ref_sums(ctypes.byref(p), _ptr(psi), _ptr(out))
    return out


def energy_parts(p, psi):
    """(E_kin, E_pot, E_int) per particle."""
    _check(p, psi)
    out = np.zeros(3)
    lib().ref_energy_parts(ctypes.byref(p), _ptr(psi), _ptr(out))
    return out


OBS_NAMES = ("norm", "mu", "energy", "rms_x", "rms_y", "rms_z", "rms_r")


def observables(p, psi):
    """dict with norm, mu, energy, rms_x, rms_y, rms_z, rms_r."""
    _check(p, psi)
    out = np.zeros(7)
    lib().ref_observables(ctypes.byref(p), _ptr(psi), _ptr(out))
    return dict(zip(OBS_NAMES, out.tolist()))


def thomas_tables(m, kappa):
    cp = np.zeros(m, np.complex128)
    mu = np.zeros(m, np.complex128)
    lib().ref_thomas_tables(m, kappa.real, kappa.imag, _ptr(cp), _ptr(mu))
    return cp, mu


def thomas_solve(kappa, b):
    """Solve (I - kappa L) u = b, L = tridiag(1, -2, 1), zero ends."""
    b = np.ascontiguousarray(b, np.complex128)
    m = b.shape[0]
    u = np.zeros(m, np.complex128)
    work = np.zeros(2 * m, np.complex128)
    lib().ref_thomas_solve(m, kappa.real, kappa.imag, _ptr(b), _ptr(u), _ptr(work))
    return u


# ------------------------------------------------------- axially symmetric

def _check_axial(p, psi):
    if psi.dtype != np.complex128 or not psi.flags.c_contiguous:
        raise TypeError("psi must be C-contiguous complex128")
    if psi.shape != p.shape2:
        raise ValueError("psi shape %s != (nz, nr) %s" % (psi.shape, p.shape2))


def axial_rho(hr, i):
    return lib().ref_axial_rho(float(hr), int(i))


def axial_weights(n):
    """(a, c): sub- and super-diagonal weights of the radial operator."""
    a, c = np.zeros(n), np.zeros(n)
    lib().ref_axial_weights(int(n), _ptr(a), _ptr(c))
    return a, c


def tridiag_solve(kappa, a, c, b):
    """Solve (I - kappa tridiag(a, -2, c)) u = b, zero beyond both ends."""
    a = np.ascontiguousarray(a, np.float64)
    c = np.ascontiguousarray(c, np.float64)
    b = np.ascontiguousarray(b, np.complex128)
    m = b.shape[0]
    u = np.zeros(m, np.complex128)
    work = np.zeros(2 * m, np.complex128)
    lib().ref_tridiag_solve(m, kappa.real, kappa.imag, _ptr(a), _ptr(c), _ptr(b), _ptr(u),
                            _ptr(work))
    return u


def axial_seed(p):
    psi = np.zeros(p.shape2, np.complex128)
    lib().ref_axial_seed(ctypes.byref(p), _ptr(psi))
    return psi


def axial_step(p, psi, n, step0=0, strang=False, g1=0.0, omega=0.0):
    _check_axial(p, psi)
    lib().ref_axial_step_ext(ctypes.byref(p), _ptr(psi), int(n), int(step0), int(bool(strang)),
                             float(g1), float(omega))
    return psi


def axial_sweep(p, axis, psi):
    _check_axial(p, psi)
    lib().ref_axial_sweep(ctypes.byref(p), int(axis), _ptr(psi))
    return psi


def axial_nonlinear_part(p, psi, frac, G):
    _check_axial(p, psi)
    lib().ref_axial_nonlinear_part(ctypes.byref(p), _ptr(psi), float(frac), float(G))
    return psi


def axial_norm(p, psi):
    _check_axial(p, psi)
    return lib().ref_axial_norm(ctypes.byref(p), _ptr(psi))


def axial_observables(p, psi):
    _check_axial(p, psi)
    out = np.zeros(7)
    lib().ref_axial_observables(ctypes.byref(p), _ptr(psi), _ptr(out))
    return dict(zip(OBS_NAMES, out.tolist()))
