"""The C ABI: libmbgb300.so builds for sm_103a, loads, and exports every
function include/mb.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(headers=("mb.h",)):
    names = set()
    for hname in headers:
        src = open(os.path.join(ROOT, "include", hname)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names.update(re.findall(r"\b(mb_[A-Za-z_0-9]+)\s*\(", src))
    return sorted(names)


def _all_headers():
    return tuple(sorted(f for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("mb_setup", "mb_apply_H", "mb_apply_S", "mb_apply_Sinv", "mb_eigsolve", "mb_destroy",
              "mb_sizes", "mb_strerror"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_1406_4960_gb300 import build
    try:
        path = build.build()
    except RuntimeError as e:     # no CUDA toolkit on this machine
        pytest.skip(str(e))
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared(_all_headers()) if not hasattr(lib, n)]
    assert not missing, missing
    lib.mb_strerror.restype = ctypes.c_char_p
    assert lib.mb_strerror(0) == b"ok"          # pure host function, no device touched


def test_binding_lists_the_same_symbols():
    from paper_1406_4960_gb300 import mb
    assert sorted(mb.EXPORTS) == _declared()


def test_oracle_checker_builds():
    from oracle import eigen
    assert os.path.exists(eigen.build_jacobi())
