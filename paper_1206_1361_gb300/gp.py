"""Python binding of libgp's C ABI (include/gp.h): the same entry points,
argument marshalling only.  Every step of the computation runs in the CUDA
library; nothing here computes.

psi arguments may be a numpy array (host), a torch tensor (host or CUDA), or a
raw integer address with ``on_device`` given explicitly.  complex128 pairs
with GP_C128 and GP_CFF (the float-float form keeps float-float pairs on the
device and exchanges complex128) and complex64 with GP_C64.  Failures raise ``GPError`` carrying
the library's code and message.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgp.so")

GP_IMAG, GP_REAL = 0, 1
GP_C128, GP_C64, GP_CFF = 0, 1, 2
GP_OK, GP_EINVAL, GP_ENOMEM, GP_ECUDA, GP_ENONFINITE, GP_ETIMEOUT, GP_EINTERNAL, GP_EFULL = (
    0, -1, -2, -3, -4, -5, -6, -7)
GP_MAX_EDGE = 8192
GP_OPT_SWEEP_PATH, GP_OPT_TILE_SHAPE, GP_OPT_SPLITTING, GP_OPT_POTENTIAL_TABLE = 1, 2, 3, 4
GP_PATH_AUTO, GP_PATH_EXACT, GP_PATH_TMA, GP_PATH_WINDOW, GP_PATH_SLAB = 0, 1, 2, 3, 4
GP_SPLIT_LIE, GP_SPLIT_STRANG = 0, 1
GP_PEAK_FP64_FMA, GP_PEAK_FP32_FMA, GP_PEAK_FP32X2_FMA = 0, 1, 2

ERROR_NAMES = {GP_EINVAL: "GP_EINVAL", GP_ENOMEM: "GP_ENOMEM", GP_ECUDA: "GP_ECUDA",
               GP_ENONFINITE: "GP_ENONFINITE", GP_ETIMEOUT: "GP_ETIMEOUT",
               GP_EINTERNAL: "GP_EINTERNAL", GP_EFULL: "GP_EFULL"}


class GPError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERROR_NAMES.get(code, "?"), code, msg))
        self.code = code


class gp_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32)]


class gp_obs(ctypes.Structure):
    _fields_ = [("norm", ctypes.c_double), ("mu", ctypes.c_double),
                ("energy", ctypes.c_double), ("rms_x", ctypes.c_double),
                ("rms_y", ctypes.c_double), ("rms_z", ctypes.c_double),
                ("rms_r", ctypes.c_double), ("step", ctypes.c_int64),
                ("t", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# Every entry point include/gp.h declares: name -> (restype, argtypes).
_vp, _i32, _i64, _dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
_int = ctypes.c_int
SIGNATURES = {
    "gp_create": (_int, [ctypes.POINTER(gp_grid), ctypes.POINTER(ctypes.c_double), _dbl,
                         _dbl, _dbl, _dbl, _dbl, _int, _int, _vp, ctypes.POINTER(_vp)]),
    "gp_load": (_int, [_vp, _vp, _i64, _int]),
    "gp_store": (_int, [_vp, _vp, _i64, _int]),
    "gp_set_params": (_int, [_vp, _dbl, _int]),
    "gp_step": (_int, [_vp, _i64]),
    "gp_observables": (_int, [_vp, ctypes.POINTER(gp_obs)]),
    "gp_sync": (_int, [_vp]),
    "gp_set_option": (_int, [_vp, _int, _int]),
    "gp_set_modulation": (_int, [_vp, _dbl, _dbl]),
    "gp_apply_pending_scale": (_int, [_vp]),
    "gp_create_axial": (_int, [_int, _int, _dbl, _dbl, _dbl, _dbl, _dbl, _dbl, _int, _int, _vp,
                               ctypes.POINTER(_vp)]),
    "gp_footprint_axial": (_int, [_int, _int, _int, ctypes.POINTER(ctypes.c_size_t)]),
    "gp_sweep_paths": (_int, [_vp, ctypes.POINTER(_int)]),
    "gp_get_option": (_int, [_vp, _int, ctypes.POINTER(_int)]),
    "gp_autotune": (_int, [_vp, _int, ctypes.POINTER(_int), ctypes.POINTER(_int),
                           ctypes.POINTER(ctypes.c_double)]),
    "gp_tile_shapes": (_int, [_int, ctypes.POINTER(_int)]),
    "gp_time_kernels": (_int, [_vp, _i64, ctypes.POINTER(ctypes.c_double), _int]),
    "gp_launches_per_step": (_int, [_vp, ctypes.POINTER(_int), ctypes.POINTER(_int)]),
    "gp_device_psi": (_int, [_vp, ctypes.POINTER(_vp)]),
    "gp_footprint": (_int, [ctypes.POINTER(gp_grid), _int, ctypes.POINTER(ctypes.c_size_t)]),
    "gp_sweep_noalloc": (_int, [_vp, ctypes.POINTER(gp_grid), _int, _dbl, _dbl, _int, _int,
                                _vp]),
    "gp_measure_peak": (_int, [_int, _i64, ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_double)]),
    "gp_create_slab": (_int, [ctypes.POINTER(gp_grid), ctypes.POINTER(ctypes.c_double), _dbl,
                              _dbl, _dbl, _dbl, _dbl, _int, ctypes.POINTER(_int), _int, _vp,
                              ctypes.POINTER(_vp)]),
    "gp_slab_exchange_count": (_int, [_vp, ctypes.POINTER(_i64)]),
    "gp_slab_seed": (_int, [_vp]),
    "gp_slab_scale": (_int, [_vp, _dbl]),
    "gp_slab_step_begin": (_int, [_vp, _vp]),
    "gp_slab_step_end": (_int, [_vp, _vp]),
    "gp_slab_first_plane": (_int, [_vp, _vp]),
    "gp_slab_local_sums": (_int, [_vp, _vp, ctypes.POINTER(ctypes.c_double)]),
    "gp_slab_observables": (_int, [_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(gp_obs)]),
    "gp_last_error": (ctypes.c_char_p, [_vp]),
    "gp_destroy": (None, [_vp]),
    "gp_batch_create": (_int, [_int, ctypes.c_size_t, _vp, ctypes.POINTER(_vp)]),
    "gp_batch_footprint": (_int, [ctypes.POINTER(gp_grid), _int, ctypes.POINTER(ctypes.c_size_t)]),
    "gp_batch_add": (_int, [_vp, ctypes.POINTER(gp_grid), ctypes.POINTER(ctypes.c_double), _dbl,
                            _dbl, _dbl, _dbl, _dbl, _int, ctypes.POINTER(_int)]),
    "gp_batch_load": (_int, [_vp, _int, _vp, _i64, _int]),
    "gp_batch_store": (_int, [_vp, _int, _vp, _i64, _int]),
    "gp_batch_set_params": (_int, [_vp, _int, _dbl, _int]),
    "gp_batch_step": (_int, [_vp, _i64]),
    "gp_batch_set_wait_ns": (_int, [_vp, _i64]),
    "gp_batch_observables": (_int, [_vp, ctypes.POINTER(gp_obs), _int]),
    "gp_batch_observables_of": (_int, [_vp, ctypes.POINTER(_int), _int, ctypes.POINTER(gp_obs)]),
    "gp_batch_remove": (_int, [_vp, _int]),
    "gp_batch_info": (_int, [_vp, ctypes.POINTER(_int), ctypes.POINTER(_int),
                             ctypes.POINTER(ctypes.c_size_t)]),
    "gp_batch_sync": (_int, [_vp]),
    "gp_batch_last_error": (ctypes.c_char_p, [_vp]),
    "gp_batch_destroy": (None, [_vp]),
}

_lib = None


def load_library(path=None):
    """Load libgp.so (built in-tree by ``__graft_entry__.build()``).  Raises
    if it is missing: there is no fallback implementation."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError("libgp.so not built at %s: run __graft_entry__.build()" % p)
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if path is None:
        _lib = lib
    return lib


def _err(ctx, rc):
    if rc != GP_OK:
        msg = load_library().gp_last_error(ctx)
        raise GPError(rc, msg.decode() if msg else "")


def _buffer(psi):
    """(address, element count, on_device, keepalive) for a psi argument."""
    if psi is None:
        return None, 0, 0, None
    if isinstance(psi, np.ndarray):
        if not psi.flags.c_contiguous:
            raise ValueError("psi must be C-contiguous")
        return psi.ctypes.data, psi.size, 0, psi
    mod = type(psi).__module__
    if mod.startswith("torch"):
        if not psi.is_contiguous():
            raise ValueError("psi must be contiguous")
        return psi.data_ptr(), psi.numel(), 1 if psi.is_cuda else 0, psi
    raise TypeError("psi must be a numpy array, a torch tensor or None")


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream          # torch.cuda.Stream


# ----------------------------------------------------------- entry points

def gp_create(grid, dx, dt, gamma, nu, lam, g, mode=GP_IMAG, precision=GP_C128,
              cuda_stream=None):
    """grid = (nx, ny, nz); dx = (hx, hy, hz).  Returns the context handle."""
    L = load_library()
    gr = gp_grid(*[int(v) for v in grid])
    h = (ctypes.c_double * 3)(*[float(v) for v in dx])
    out = _vp()
    rc = L.gp_create(ctypes.byref(gr), h, float(dt), float(gamma), float(nu), float(lam),
                     float(g), int(mode), int(precision), _stream_handle(cuda_stream),
                     ctypes.byref(out))
    if rc != GP_OK:
        msg = L.gp_last_error(None)
        raise GPError(rc, msg.decode() if msg else "")
    return out.value


def gp_create_axial(nr, nz, hr, hz, dt, gamma, lam, g, mode=GP_IMAG, precision=GP_C128,
                    cuda_stream=None):
    """Axially symmetric psi(rho, z) on n_r radial x n_z axial points."""
    L = load_library()
    out = _vp()
    rc = L.gp_create_axial(int(nr), int(nz), float(hr), float(hz), float(dt), float(gamma),
                           float(lam), float(g), int(mode), int(precision),
                           _stream_handle(cuda_stream), ctypes.byref(out))
    if rc != GP_OK:
        msg = L.gp_last_error(None)
        raise GPError(rc, msg.decode() if msg else "")
    return out.value


def gp_footprint_axial(nr, nz, precision=GP_C128):
    b = ctypes.c_size_t()
    rc = load_library().gp_footprint_axial(int(nr), int(nz), int(precision), ctypes.byref(b))
    if rc != GP_OK:
        raise GPError(rc, load_library().gp_last_error(None).decode())
    return b.value


def gp_load(ctx, psi=None, count=None, on_device=None):
    """psi None loads the normalised Gaussian seed."""
    addr, n, dev, _keep = _buffer(psi) if not isinstance(psi, int) else (psi, count, on_device, None)
    if count is not None:
        n = count
    if on_device is not None:
        dev = on_device
    _err(ctx, load_library().gp_load(ctx, addr, int(n or 0), int(dev or 0)))


def gp_store(ctx, out, count=None, on_device=None):
    addr, n, dev, _keep = _buffer(out) if not isinstance(out, int) else (out, count, on_device, None)
    if count is not None:
        n = count
    if on_device is not None:
        dev = on_device
    _err(ctx, load_library().gp_store(ctx, addr, int(n), int(dev)))
    return out


def gp_set_params(ctx, g, mode):
    _err(ctx, load_library().gp_set_params(ctx, float(g), int(mode)))


def gp_step(ctx, n):
    _err(ctx, load_library().gp_step(ctx, int(n)))


def gp_observables(ctx):
    o = gp_obs()
    _err(ctx, load_library().gp_observables(ctx, ctypes.byref(o)))
    return o.as_dict()


KERNEL_SLOTS = ("sweep_x", "sweep_y", "sweep_z", "norm_finish", "observables")


def gp_time_kernels(ctx, steps):
    """Mean ms per launch of each kernel slot (dict keyed by KERNEL_SLOTS)."""
    out = (ctypes.c_double * 8)()
    _err(ctx, load_library().gp_time_kernels(ctx, int(steps), out, 8))
    return dict(zip(KERNEL_SLOTS, list(out)[:5]))


def gp_launches_per_step(ctx):
    """(kernel launches per SSCN step, kernel launches per gp_observables)."""
    k, o = ctypes.c_int(), ctypes.c_int()
    _err(ctx, load_library().gp_launches_per_step(ctx, ctypes.byref(k), ctypes.byref(o)))
    return k.value, o.value


def gp_apply_pending_scale(ctx):
    """Apply any pending imaginary-time renormalisation to the device psi."""
    _err(ctx, load_library().gp_apply_pending_scale(ctx))


class _DeviceArray:
    """__cuda_array_interface__ of a device buffer the context owns."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3,
                                         "strides": None}


def gp_set_modulation(ctx, g1, omega):
    """g(t) = g + g1 cos(omega t) from the next step on (g1 = 0: off)."""
    _err(ctx, load_library().gp_set_modulation(ctx, float(g1), float(omega)))


def gp_set_option(ctx, option, value):
    _err(ctx, load_library().gp_set_option(ctx, int(option), int(value)))


def gp_get_option(ctx, option):
    v = ctypes.c_int()
    _err(ctx, load_library().gp_get_option(ctx, int(option), ctypes.byref(v)))
    return v.value


def gp_autotune(ctx, steps=5):
    """(sweep path, tile shape, ms per step) of the fastest candidate, now set."""
    p, sh, ms = _int(), _int(), ctypes.c_double()
    _err(ctx, load_library().gp_autotune(ctx, int(steps), ctypes.byref(p), ctypes.byref(sh),
                                         ctypes.byref(ms)))
    return p.value, sh.value, ms.value


def gp_tile_shapes(precision):
    n = ctypes.c_int()
    rc = load_library().gp_tile_shapes(int(precision), ctypes.byref(n))
    if rc != GP_OK:
        raise GPError(rc, gp_last_error(None))
    return n.value


def gp_sweep_paths(ctx):
    """Sweep path per axis now in use: GP_PATH_EXACT, GP_PATH_TMA, GP_PATH_WINDOW or
    GP_PATH_SLAB (0 if none)."""
    p = (ctypes.c_int * 3)()
    _err(ctx, load_library().gp_sweep_paths(ctx, p))
    return tuple(p)


def gp_sync(ctx):
    _err(ctx, load_library().gp_sync(ctx))


def gp_device_psi(ctx):
    p = _vp()
    _err(ctx, load_library().gp_device_psi(ctx, ctypes.byref(p)))
    return p.value


def gp_footprint(grid, precision=GP_C128):
    gr = gp_grid(*[int(v) for v in grid])
    b = ctypes.c_size_t()
    rc = load_library().gp_footprint(ctypes.byref(gr), int(precision), ctypes.byref(b))
    if rc != GP_OK:
        raise GPError(rc, load_library().gp_last_error(None).decode())
    return b.value


def gp_sweep_noalloc(psi_device, grid, axis, h, dt, mode, precision, cuda_stream=None):
    """One Crank-Nicolson sweep in place on a caller-owned device buffer (a
    CUDA torch tensor or a device address), with no device allocation."""
    if isinstance(psi_device, int):
        addr = psi_device
    else:
        addr, _n, dev, _keep = _buffer(psi_device)
        if not dev:
            raise ValueError("gp_sweep_noalloc needs a device buffer")
    gr = gp_grid(*[int(v) for v in grid])
    rc = load_library().gp_sweep_noalloc(addr, ctypes.byref(gr), int(axis), float(h), float(dt),
                                         int(mode), int(precision), _stream_handle(cuda_stream))
    if rc != GP_OK:
        raise GPError(rc, gp_last_error(None))


def gp_measure_peak(kind, iters=20000):
    """Measured TFLOP/s of one arithmetic pipe of the current device (and the
    milliseconds of the best launch)."""
    tf, ms = ctypes.c_double(), ctypes.c_double()
    rc = load_library().gp_measure_peak(int(kind), int(iters), ctypes.byref(tf), ctypes.byref(ms))
    if rc != GP_OK:
        raise GPError(rc, gp_last_error(None))
    return tf.value, ms.value


def gp_create_slab(grid, dx, dt, gamma, nu, lam, g, bounds, rank, cuda_stream=None):
    """One rank's context of a grid split along z (see zslab.py)."""
    gr = gp_grid(*[int(v) for v in grid])
    h = (ctypes.c_double * 3)(*[float(v) for v in dx])
    b = (_int * len(bounds))(*[int(v) for v in bounds])
    out = _vp()
    rc = load_library().gp_create_slab(ctypes.byref(gr), h, float(dt), float(gamma), float(nu),
                                       float(lam), float(g), len(bounds) - 1, b, int(rank),
                                       _stream_handle(cuda_stream), ctypes.byref(out))
    if rc != GP_OK:
        raise GPError(rc, gp_last_error(None))
    return out.value


def gp_slab_exchange_count(ctx):
    n = _i64()
    _err(ctx, load_library().gp_slab_exchange_count(ctx, ctypes.byref(n)))
    return n.value


def gp_slab_seed(ctx):
    _err(ctx, load_library().gp_slab_seed(ctx))


def gp_slab_scale(ctx, factor):
    _err(ctx, load_library().gp_slab_scale(ctx, float(factor)))


def gp_slab_step_begin(ctx, bnd_device):
    _err(ctx, load_library().gp_slab_step_begin(ctx, bnd_device))


def gp_slab_step_end(ctx, bnd_all_device):
    _err(ctx, load_library().gp_slab_step_end(ctx, bnd_all_device))


def gp_slab_first_plane(ctx, out_device):
    _err(ctx, load_library().gp_slab_first_plane(ctx, out_device))


def gp_slab_local_sums(ctx, next_first_device=None):
    s = (ctypes.c_double * 9)()
    _err(ctx, load_library().gp_slab_local_sums(ctx, next_first_device, s))
    return np.array(s[:], dtype=np.float64)


def gp_slab_observables(ctx, global_sums):
    s = (ctypes.c_double * 9)(*[float(v) for v in global_sums])
    o = gp_obs()
    _err(ctx, load_library().gp_slab_observables(ctx, s, ctypes.byref(o)))
    return o.as_dict()


def gp_last_error(ctx=None):
    msg = load_library().gp_last_error(ctx)
    return msg.decode() if msg else ""


def gp_destroy(ctx):
    load_library().gp_destroy(ctx)


# ------------------------------------------------------------ convenience

class Solver:
    """Owns one context.  ``shape`` is (nx, ny, nz); arrays are (nz, ny, nx)."""

    def __init__(self, shape, dx, dt, gamma, nu, lam, g, mode=GP_IMAG,
                 precision=GP_C128, stream=None, _ctx=None):
        self.shape = tuple(int(v) for v in shape)
        self.precision = precision
        self.ctx = _ctx if _ctx is not None else gp_create(self.shape, dx, dt, gamma, nu, lam, g,
                                                           mode, precision, stream)

    @classmethod
    def axial(cls, nr, nz, hr, hz, dt, gamma, lam, g, mode=GP_IMAG, stream=None):
        """Axially symmetric psi(rho, z); arrays are (nz, nr)."""
        ctx = gp_create_axial(nr, nz, hr, hz, dt, gamma, lam, g, mode, GP_C128, stream)
        s = cls((nr, nz, 1), None, dt, gamma, lam, 0.0, g, mode, GP_C128, stream, _ctx=ctx)
        s.is_axial = True
        return s

    is_axial = False

    @property
    def array_shape(self):
        nx, ny, nz = self.shape
        return (ny, nx) if self.is_axial else (nz, ny, nx)

    @property
    def dtype(self):
        """Host dtype of gp_load / gp_store (GP_CFF exchanges complex128)."""
        return np.complex64 if self.precision == GP_C64 else np.complex128

    def load(self, psi=None):
        gp_load(self.ctx, psi)
        return self

    def step(self, n):
        gp_step(self.ctx, n)
        return self

    def set_params(self, g, mode):
        gp_set_params(self.ctx, g, mode)
        return self

    def observables(self):
        return gp_observables(self.ctx)

    def psi(self):
        out = np.empty(self.array_shape, self.dtype)
        gp_store(self.ctx, out)
        return out

    def sync(self):
        gp_sync(self.ctx)

    def device_view(self):
        """A torch CUDA tensor that borrows the context's psi buffer (no copy;
        valid until close), normalised: any pending imaginary-time scale is
        applied first.  Steps taken later update it in place."""
        import torch
        gp_apply_pending_scale(self.ctx)
        gp_sync(self.ctx)
        if self.precision == GP_CFF:
            # float-float pairs: (..., 4) float32 = (re_hi, im_hi, re_lo, im_lo)
            return torch.as_tensor(_DeviceArray(gp_device_psi(self.ctx), self.array_shape + (4,),
                                                "<f4"), device="cuda")
        typestr = "<c16" if self.precision == GP_C128 else "<c8"
        return torch.as_tensor(_DeviceArray(gp_device_psi(self.ctx), self.array_shape, typestr),
                               device="cuda")

    def set_path(self, path):
        gp_set_option(self.ctx, GP_OPT_SWEEP_PATH, path)
        return self

    def set_splitting(self, split):
        gp_set_option(self.ctx, GP_OPT_SPLITTING, split)
        return self

    def set_modulation(self, g1, omega):
        gp_set_modulation(self.ctx, g1, omega)
        return self

    def paths(self):
        return gp_sweep_paths(self.ctx)

    def close(self):
        if self.ctx:
            gp_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- batches

def _berr(b, rc):
    if rc != GP_OK:
        msg = load_library().gp_batch_last_error(b)
        raise GPError(rc, msg.decode() if msg else "")


def gp_batch_create(precision=GP_C64, cap_bytes=1 << 34, cuda_stream=None):
    out = _vp()
    rc = load_library().gp_batch_create(int(precision), int(cap_bytes),
                                        _stream_handle(cuda_stream), ctypes.byref(out))
    if rc != GP_OK:
        raise GPError(rc, gp_last_error(None))
    return out.value


def gp_batch_footprint(grid, precision=GP_C64):
    gr = gp_grid(*[int(v) for v in grid])
    b = ctypes.c_size_t()
    rc = load_library().gp_batch_footprint(ctypes.byref(gr), int(precision), ctypes.byref(b))
    if rc != GP_OK:
        raise GPError(rc, gp_last_error(None))
    return b.value


def gp_batch_add(b, grid, dx, dt, gamma, nu, lam, g, mode=GP_IMAG):
    gr = gp_grid(*[int(v) for v in grid])
    h = (ctypes.c_double * 3)(*[float(v) for v in dx])
    slot = _int()
    _berr(b, load_library().gp_batch_add(b, ctypes.byref(gr), h, float(dt), float(gamma), float(nu),
                                         float(lam), float(g), int(mode), ctypes.byref(slot)))
    return slot.value


def gp_batch_load(b, slot, psi=None, count=None, on_device=None):
    addr, n, dev, _keep = _buffer(psi) if not isinstance(psi, int) else (psi, count, on_device, None)
    if count is not None:
        n = count
    if on_device is not None:
        dev = on_device
    _berr(b, load_library().gp_batch_load(b, int(slot), addr, int(n or 0), int(dev or 0)))


def gp_batch_store(b, slot, out, count=None, on_device=None):
    addr, n, dev, _keep = _buffer(out) if not isinstance(out, int) else (out, count, on_device, None)
    if count is not None:
        n = count
    if on_device is not None:
        dev = on_device
    _berr(b, load_library().gp_batch_store(b, int(slot), addr, int(n), int(dev)))
    return out


def gp_batch_set_params(b, slot, g, mode):
    _berr(b, load_library().gp_batch_set_params(b, int(slot), float(g), int(mode)))


def gp_batch_step(b, n):
    _berr(b, load_library().gp_batch_step(b, int(n)))


def gp_batch_set_wait_ns(b, ns):
    """Budget of each dependency wait of the batch's persistent kernel (ns)."""
    _berr(b, load_library().gp_batch_set_wait_ns(b, int(ns)))


def gp_batch_observables(b, capacity, slots=None):
    """List of capacity dicts, one per slot id (step == -1: unused slot); with
    `slots`, a dict of those slots' entries only (no conversion of the rest)."""
    arr = (gp_obs * max(1, capacity))()
    _berr(b, load_library().gp_batch_observables(b, arr, int(capacity)))
    if slots is not None:
        return {s: arr[s].as_dict() for s in slots}
    return [arr[i].as_dict() for i in range(capacity)]


def gp_batch_observables_of(b, slots):
    """Dict slot -> observables of the given slots only."""
    slots = [int(v) for v in slots]
    ids = (_int * max(1, len(slots)))(*slots)
    arr = (gp_obs * max(1, len(slots)))()
    _berr(b, load_library().gp_batch_observables_of(b, ids, len(slots), arr))
    return {s: arr[i].as_dict() for i, s in enumerate(slots)}


def gp_batch_remove(b, slot):
    _berr(b, load_library().gp_batch_remove(b, int(slot)))


def gp_batch_info(b):
    """(active instances, slot table size, bytes charged against the cap)."""
    a, s, u = _int(), _int(), ctypes.c_size_t()
    _berr(b, load_library().gp_batch_info(b, ctypes.byref(a), ctypes.byref(s), ctypes.byref(u)))
    return a.value, s.value, u.value


def gp_batch_sync(b):
    _berr(b, load_library().gp_batch_sync(b))


def gp_batch_last_error(b=None):
    msg = load_library().gp_batch_last_error(b)
    return msg.decode() if msg else ""


def gp_batch_destroy(b):
    load_library().gp_batch_destroy(b)


class Batch:
    """Owns one batch; instances are addressed by slot id."""

    def __init__(self, precision=GP_C64, cap_bytes=1 << 34, stream=None):
        self.precision = precision
        self.b = gp_batch_create(precision, cap_bytes, stream)
        self.shapes = {}

    def add(self, shape, dx, dt, gamma, nu, lam, g, mode=GP_IMAG, psi=None):
        slot = gp_batch_add(self.b, shape, dx, dt, gamma, nu, lam, g, mode)
        self.shapes[slot] = tuple(int(v) for v in shape)
        gp_batch_load(self.b, slot, psi)
        return slot

    def step(self, n):
        gp_batch_step(self.b, n)
        return self

    def set_wait_ns(self, ns):
        gp_batch_set_wait_ns(self.b, ns)
        return self

    def observables(self, slots=None):
        """Dict slot -> observables: of every instance, or of `slots` only."""
        if slots is not None:
            return gp_batch_observables_of(self.b, slots)
        cap = max(self.shapes) + 1 if self.shapes else 0
        return gp_batch_observables(self.b, cap, list(self.shapes))

    def psi(self, slot):
        nx, ny, nz = self.shapes[slot]
        dt = np.complex128 if self.precision == GP_C128 else np.complex64
        out = np.empty((nz, ny, nx), dt)
        gp_batch_store(self.b, slot, out)
        return out

    def set_params(self, slot, g, mode):
        gp_batch_set_params(self.b, slot, g, mode)

    def remove(self, slot):
        gp_batch_remove(self.b, slot)
        self.shapes.pop(slot, None)

    def info(self):
        return gp_batch_info(self.b)

    def close(self):
        if self.b:
            gp_batch_destroy(self.b)
            self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
