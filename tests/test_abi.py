"""The C-ABI library builds, loads and exports every entry point include/lmbd.h declares.

No compute call is made here, so this runs without a GPU.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:int|const char\*)\s+(lmbd_\w+)\s*\(", src, re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    from paper_2407_06409_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = _declared()
    for n in ("lmbd_create", "lmbd_energy_forces", "lmbd_energy_forces_weighted", "lmbd_destroy",
              "lmbd_status_string"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    lib.lmbd_status_string.restype = ctypes.c_char_p
    assert lib.lmbd_status_string(0) == b"ok"
    assert lib.lmbd_status_string(3) == b"screening matrix singular (zero pivot in the LU fallback)"


def test_binding_loads_and_rejects_bad_arguments(libpath):
    from paper_2407_06409_gb300 import lmbd
    p = lmbd.default_params()
    assert p.r_scs == 5.0 and p.r_sphere == 7.0 and p.beta == 0.83 and p.d == 6.0
    # invalid parameters are rejected on the host, before any device work
    with pytest.raises(lmbd.LmbdError) as e:
        lmbd.LMBD([[6.0, 20.0, 3.2]], lmbd.default_params(r_scs=9.0), 12, 6)   # r_scs > sphere
    assert e.value.status == lmbd.LMBD_EINVAL
    with pytest.raises(lmbd.LmbdError) as e:
        lmbd.LMBD([[6.0, 20.0, 3.2]], p, 12, 1)
    assert e.value.status == lmbd.LMBD_EUNSUPPORTED
    with pytest.raises(lmbd.LmbdError):
        lmbd.LMBD([[-1.0, 20.0, 3.2]], p, 12, 6)
