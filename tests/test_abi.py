"""The C-ABI library builds, loads and exports every entry point that
include/gp.h declares; argument validation that needs no GPU."""
import os
import re

import pytest

import paper_1206_1361_gb300 as P
from paper_1206_1361_gb300 import gp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(gp_\w+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for must in ("gp_create", "gp_load", "gp_step", "gp_observables", "gp_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol():
    lib = P.load_library()
    missing = [n for n in declared_entry_points() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert set(declared_entry_points()) <= set(gp.SIGNATURES)
    for n in declared_entry_points():
        assert callable(getattr(gp, n))


def test_footprint_and_invalid_shapes():
    b = gp.gp_footprint((256, 256, 256), gp.GP_C128)
    assert b >= 2 * 256 ** 3 * 16
    assert gp.gp_footprint((256, 256, 256), gp.GP_C64) < b
    for bad in ((2, 8, 8), (8, 8, 2), (8, 8, 0), (9000, 8, 8)):
        with pytest.raises(gp.GPError) as e:
            gp.gp_footprint(bad)
        assert e.value.code == gp.GP_EINVAL


@pytest.mark.parametrize("kw", [dict(dx=(0.0, 0.1, 0.1)), dict(dt=-1.0), dict(mode=7),
                                dict(precision=9), dict(grid=(8, 8, 2))])
def test_create_rejects_bad_arguments_before_touching_the_device(kw):
    args = dict(grid=(8, 8, 8), dx=(0.1, 0.1, 0.1), dt=0.01, gamma=1.0, nu=1.0, lam=1.0,
                g=0.0, mode=gp.GP_IMAG, precision=gp.GP_C128)
    args.update(kw)
    with pytest.raises(gp.GPError) as e:
        gp.gp_create(**args)
    assert e.value.code == gp.GP_EINVAL
    assert gp.gp_last_error(None)
