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


def _c_structs():
    """{typedef name: [(field, C type, array length)]} of include/mb.h's
    plain structs (comments stripped)."""
    src = open(os.path.join(ROOT, "include", "mb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    type_words = {"const", "double", "int", "long", "unsigned", "char", "float", "void", "short"}
    out = {}
    for body, name in re.findall(r"typedef struct\s*\{(.*?)\}\s*(mb_\w+)\s*;", src, flags=re.S):
        fields = []
        for decl in body.split(";"):
            toks = re.findall(r"\w+|\*|\[\d+\]|,", decl)
            if not toks:
                continue
            i = 0
            while i < len(toks) and (toks[i] in type_words or toks[i].startswith("mb_")):
                i += 1
            ctype = " ".join(t for t in toks[:i] if t != "const")
            stars, n = 0, 1
            for t in toks[i:] + [","]:
                if t == "*":
                    stars += 1
                elif t.startswith("["):
                    n = int(t[1:-1])
                elif t == ",":
                    fields.append((fname, ctype + "*" * stars, n))
                    stars, n = 0, 1
                else:
                    fname = t
        out[name] = fields
    return out


_CTYPE = {"double": ctypes.c_double, "int": ctypes.c_int, "long long": ctypes.c_longlong}


@pytest.mark.parametrize("cname,pyname", [("mb_cell", "_Cell"), ("mb_atom", "_Atom"), ("mb_opts", "_Opts"),
                                           ("mb_request", "_Request"), ("mb_solve_opts", "SolveOpts"),
                                           ("mb_solve_info", "SolveInfo"), ("mb_scf_opts", "ScfOpts"),
                                           ("mb_scf_info", "ScfInfo")])
def test_binding_structs_match_the_header(cname, pyname):
    """The ctypes structures of the binding have the header's fields, in its
    order, with its scalar types and array lengths (pointer fields: pointers)."""
    from paper_1406_4960_gb300 import mb
    cfields = _c_structs()[cname]
    pyfields = getattr(mb, pyname)._fields_
    assert [f for f, _, _ in cfields] == [f for f, _ in pyfields], (cname, pyname)
    for (f, ct, n), (_, pt) in zip(cfields, pyfields):
        if ct.endswith("*"):
            assert issubclass(pt, (ctypes._Pointer, ctypes.c_void_p)) or pt is ctypes.c_void_p, (cname, f)
            continue
        if ct in _CTYPE:
            want = _CTYPE[ct] * n if n > 1 else _CTYPE[ct]
            if n > 1:
                assert pt._length_ == n and pt._type_ is _CTYPE[ct], (cname, f)
            else:
                assert pt is want, (cname, f, pt)


def test_raw_abi_test_structs_match_the_header():
    """The hand-written ctypes structures of the raw C-ABI GPU test follow the
    header too (field names in order)."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("raw_cabi", os.path.join(ROOT, "tests", "test_gpu_cabi.py"))
    mod = importlib.util.module_from_spec(spec)
    try:
        spec.loader.exec_module(mod)
    except pytest.skip.Exception:
        pytest.skip("torch not importable")
    cs = _c_structs()
    for cname, pyname in (("mb_cell", "Cell"), ("mb_atom", "Atom"), ("mb_opts", "Opts")):
        if hasattr(mod, pyname):
            assert [f for f, _, _ in cs[cname]] == [f for f, _ in getattr(mod, pyname)._fields_], cname
