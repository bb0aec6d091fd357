"""CPU checks of the C-ABI boundary: the library builds, loads without a GPU,
exports every function include/*.h declares, and rejects bad arguments on the
host before touching a device."""
import ctypes as C
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1411_4622_gb300 import _lib, build

    build.build()
    return _lib.load()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+char\s*\*|int)\s+(\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported(lib):
    from paper_1411_4622_gb300 import _lib

    names = declared_functions()
    assert len(names) >= 10
    assert names == set(_lib.EXPORTS)
    for n in names:
        assert hasattr(lib, n), n
    assert lib.satpila_version() >= 10000


def test_host_side_argument_checks(lib):
    from paper_1411_4622_gb300 import _lib

    out = C.c_void_p()
    g = _lib.PilaGeom(0, 10, 11, None, None)
    assert lib.pila_build(C.byref(g), 0, None, C.byref(out)) == _lib.ERR_INVALID_ARG
    assert b"n_angles" in lib.satpila_last_error() or b">= 1" in lib.satpila_last_error()
    g = _lib.PilaGeom(8, 10, 11, None, None)
    assert lib.pila_build(C.byref(g), 7, None, C.byref(out)) == _lib.ERR_INVALID_ARG
    g = _lib.PilaGeom(8, 10, 40000, None, None)
    assert lib.pila_build(C.byref(g), _lib.PILA_F16, None, C.byref(out)) == _lib.ERR_INVALID_ARG
    prm = _lib.SatParams()
    assert lib.sat_run(None, 1, None, None, C.byref(prm), None, None) == _lib.ERR_INVALID_ARG
    assert lib.sat_run_ptrs(None, 1, None, None, C.byref(prm), None, None) == _lib.ERR_INVALID_ARG
    sp = _lib.SirtParams(1, 5, 1.0, 0)
    assert lib.sirt_run(None, 1, None, None, C.byref(sp), None, None) == _lib.ERR_INVALID_ARG
    assert lib.pila_free(None) == 0
    g = C.c_double()
    assert lib.satpila_probe_read(None, 1 << 20, 0, 0, 1, C.byref(g), None) == _lib.ERR_INVALID_ARG
    assert lib.satpila_probe_smem(5, 1, C.byref(g), None) == _lib.ERR_INVALID_ARG


def test_struct_layouts_match_header():
    from paper_1411_4622_gb300 import _lib

    # sizes the C compiler gives these structs on LP64
    assert C.sizeof(_lib.SatTraceRec) == 32
    assert C.sizeof(_lib.PilaInfo) == 48
    assert C.sizeof(_lib.SatParams) == 96
    assert C.sizeof(_lib.PilaGeom) == 32
    assert C.sizeof(_lib.SatStats) == 88
    assert C.sizeof(_lib.SatServerCfg) == 32


def header_constants():
    """Every integer #define of include/satpila.h, evaluated."""
    text = open(os.path.join(ROOT, "include", "satpila.h")).read()
    out = {}
    for m in re.finditer(r"^#define\s+(\w+)\s+(.+?)\s*(?:/\*.*)?$", text, flags=re.M):
        expr = re.sub(r"(\d+)u\b", r"\1", m.group(2).strip())
        if re.fullmatch(r"[\d\s()<>+\-*]+", expr):
            out[m.group(1)] = eval(expr)
    return out


def test_binding_constants_match_header():
    """The Python binding's constants are the header's values (a stale copy
    would pass wrong flags or misread plans and status codes)."""
    from paper_1411_4622_gb300 import _lib

    h = header_constants()
    assert len(h) >= 30
    for name, value in h.items():
        if name == "SATPILA_NOALLOC_SCRATCH_BYTES":
            assert _lib.NOALLOC_SCRATCH_BYTES == value
            continue
        py = name[len("SATPILA_"):] if name.startswith("SATPILA_") else name
        assert hasattr(_lib, py), name
        assert getattr(_lib, py) == value, name
