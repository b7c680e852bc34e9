"""The C ABI library: it builds, loads and exports every symbol that
include/*.h declares (no compute call: this runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(lrs\w*)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_2311_03824_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ["lrs_create", "lrs_set_measurements", "lrs_init", "lrs_iterate", "lrs_solve",
                 "lrs_get", "lrs_destroy", "lrs_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_loads_and_reports_argument_errors(libpath):
    import paper_2311_03824_gb300.lrs as L
    L.lib()
    with pytest.raises(L.LrsError) as e:
        L.lrs_create(0, 10, 10, 2, 1)
    assert e.value.status == L.LRS_ERR_ARG
    with pytest.raises(L.LrsError) as e:
        L.lrs_create(100, 10, 10, 20, 1)       # r > 16
    assert e.value.status == L.LRS_ERR_ARG
    with pytest.raises(L.LrsError) as e:
        L.lrs_create(100, 10, 10, 2, 101)      # rho > n
    assert e.value.status == L.LRS_ERR_ARG
    with pytest.raises(L.LrsError) as e:
        L.lrs_create(5120, 10, 10, 2, 1, L.LRS_OP_DFT2D_MASK, L.make_options(nx=80, ny=64))
    assert e.value.status == L.LRS_ERR_ARG      # nx not a power of two, frame above 4096
    assert "power" in L.lrs_last_error()
