"""On-disk cache of sweep-kernel choices (gp_autotune) per problem class.

The key is what decides the best kernel: grid shape, precision, mode and
the Crank-Nicolson kappa per axis (dt / 4 h^2, which sets the look-back
window of the TMA path), rounded to two significant digits.  The cache is a
JSON file at $GP_AUTOTUNE_CACHE, else ~/.cache/gp_sscn/autotune.json; a
missing or unreadable file only means tuning runs again.
"""
import json
import os

from . import gp


def cache_path():
    return os.environ.get("GP_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "gp_sscn",
                                       "autotune.json"))


# Revision of the libraries' tile-shape tables: a cached shape index names an
# entry of the table it was measured on.
SHAPE_TABLE = 2


def problem_key(shape, h, dt, precision, mode):
    kap = ["%.2g" % (dt / (4.0 * hk * hk)) for hk in h[:3 if shape[2] > 1 else 2]]
    return "%dx%dx%d/p%d/m%d/k%s/t%d" % (shape[0], shape[1], shape[2], precision, mode,
                                        ",".join(kap), SHAPE_TABLE)


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path, table):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(solver, h, dt, mode, steps=5, path=None):
    """Apply the cached choice for solver's problem class, or autotune and
    cache it.  Returns the dict {path, shape, ms, cached}."""
    path = path or cache_path()
    key = problem_key(solver.shape, h, dt, solver.precision, mode)
    table = _load(path)
    hit = table.get(key)
    if hit is not None:
        try:
            gp.gp_set_option(solver.ctx, gp.GP_OPT_TILE_SHAPE, hit["shape"])
            gp.gp_set_option(solver.ctx, gp.GP_OPT_SWEEP_PATH, hit["path"])
            return dict(hit, cached=True)
        except gp.GPError:
            pass                      # stale entry: tune again
    p, sh, ms = gp.gp_autotune(solver.ctx, steps)
    table[key] = {"path": p, "shape": sh, "ms": ms}
    try:
        _store(path, table)
    except OSError:
        pass
    return {"path": p, "shape": sh, "ms": ms, "cached": False}
