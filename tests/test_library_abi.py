"""The C-ABI library builds for sm_103a, loads, and exports every symbol include/iim.h declares.

No compute call is made here (no GPU on the CPU runner)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w\s\*]*?\b(iim_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2503_22455_gb300 import build as b
    if not os.path.exists(b.LIB):
        b.build()
    return b.LIB


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("iim_problem_create", "iim_set_data", "iim_apply", "iim_precondition", "iim_solve",
                     "iim_solve_host", "iim_batch_solve", "iim_problem_destroy", "iim_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header(lib_path):
    import paper_2503_22455_gb300 as iim
    lib = iim.load(lib_path)
    for n in _declared():
        assert n in iim.SIGNATURES or n in ("iim_default_options",), n
    # calls that need no device
    o = iim.default_options()
    assert o.restart == 10 and abs(o.tol - 1e-10) < 1e-25
    assert lib.iim_status_string(2).decode().startswith("curvature")


def test_invalid_descriptor_is_rejected_without_touching_the_device(lib_path):
    import paper_2503_22455_gb300 as iim
    lib = iim.load(lib_path)
    d = iim.make_desc(3, 64, iim.GEOM["sphere"], (0, 0, 0, 0.5), True, iim.BC["dirichlet"], 0, order=6)
    h = ctypes.c_void_p()
    st = lib.iim_problem_create(ctypes.byref(d), ctypes.byref(iim.default_options()), None, ctypes.byref(h))
    assert st == 1 and not h.value
    d = iim.make_desc(2, 64, iim.GEOM["star"], (0, 0, 0.5, 0.1, 5, 0), False, iim.BC["interface"], 0, order=6)
    st = lib.iim_problem_create(ctypes.byref(d), ctypes.byref(iim.default_options()), None, ctypes.byref(h))
    assert st == 1 and "box" in lib.iim_last_error().decode()
