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


def _header_enums():
    src = open(os.path.join(ROOT, "include", "iim.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    vals = {}
    for body in re.findall(r"enum\s*\{(.*?)\}", src, flags=re.S):
        for name, val in re.findall(r"(IIM_\w+)\s*=\s*(\d+)", body):
            vals[name] = int(val)
    return vals


def test_binding_constants_match_the_header():
    """The binding's geometry, condition, precision, cycle and Krylov codes are the header's."""
    import paper_2503_22455_gb300 as iim
    import workloads as W
    e = _header_enums()
    for key, name in (("circle", "CIRCLE"), ("ellipse", "ELLIPSE"), ("star", "STAR"), ("sphere", "SPHERE"),
                      ("ellipsoid", "ELLIPSOID"), ("perturbed_sphere", "PERTURBED_SPHERE"), ("fourier", "FOURIER"),
                      ("levelset_grid", "LEVELSET_GRID")):
        assert iim.GEOM[key] == e["IIM_GEOM_" + name] == getattr(W, name), key
    for key in ("dirichlet", "neumann", "interface"):
        assert iim.BC[key] == e["IIM_BC_" + key.upper()] == getattr(W, key.upper())
    assert (W.BOX_NONE, W.BOX_DIRICHLET) == (e["IIM_BOX_NONE"], e["IIM_BOX_DIRICHLET"])
    assert (iim.MG_FP32, iim.MG_FP64, iim.MG_FP32_BF16R) == (e["IIM_MG_FP32"], e["IIM_MG_FP64"], e["IIM_MG_FP32_BF16R"])
    assert (iim.CYCLE_V, iim.CYCLE_W) == (e["IIM_CYCLE_V"], e["IIM_CYCLE_W"])
    assert iim.MAX_FOURIER_MODES == e["IIM_MAX_FOURIER_MODES"]
    assert (iim.KRYLOV_FGMRES, iim.KRYLOV_GMRES_LEFT) == (e["IIM_KRYLOV_FGMRES"], e["IIM_KRYLOV_GMRES_LEFT"])
    status = {k: v for k, v in e.items() if k.startswith("IIM_ERR_") or k == "IIM_OK"}
    assert len(status) == len(iim.STATUS_NAMES)
    for name, val in status.items():
        assert getattr(iim, name) == val, name


def test_options_struct_matches_the_header(lib_path):
    """iim_default_options fills every field the binding's struct declares (no layout drift):
    the defaults the header documents come back through ctypes."""
    import paper_2503_22455_gb300 as iim
    iim.load(lib_path)
    o = iim.default_options()
    assert (o.restart, o.max_iter, o.nu1, o.nu2, o.mg_precision, o.use_graph, o.reorth, o.cycle, o.krylov) == \
        (10, 500, 2, 2, iim.MG_FP32, 1, 1, iim.CYCLE_V, iim.KRYLOV_FGMRES)


@pytest.mark.parametrize("field,value", [("cycle", 0), ("cycle", 3), ("krylov", 2), ("krylov", -1),
                                         ("restart", 17), ("mg_precision", 3)])
def test_invalid_options_are_rejected_without_touching_the_device(lib_path, field, value):
    import paper_2503_22455_gb300 as iim
    lib = iim.load(lib_path)
    d = iim.make_desc(2, 64, iim.GEOM["circle"], (0.0, 0.0, 0.5), True, iim.BC["dirichlet"], 0, order=4)
    o = iim.default_options()
    setattr(o, field, value)
    h = ctypes.c_void_p()
    st = lib.iim_problem_create(ctypes.byref(d), ctypes.byref(o), None, ctypes.byref(h))
    assert st == 1 and not h.value, (field, value, st)


def test_struct_layouts_match_the_header(tmp_path):
    """sizeof and every field offset of the descriptor, options and solve-info structs, as the
    C compiler lays them out from include/iim.h, equal the binding's ctypes structs."""
    import shutil
    import subprocess
    import paper_2503_22455_gb300 as iim
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"iim_problem_desc": iim.Desc, "iim_options": iim.Options, "iim_solve_info": iim.SolveInfo}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "iim.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, cls in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)


@pytest.mark.parametrize("case", ["even_count", "too_many_modes", "no_coef", "negative_radius", "grid_no_phi",
                                  "fourier_3d"])
def test_invalid_geometry_input_is_rejected_without_touching_the_device(lib_path, case):
    import paper_2503_22455_gb300 as iim
    lib = iim.load(lib_path)
    kind, dim, coef = iim.GEOM["fourier"], 2, [0.5, 0.01, 0.02]
    if case == "even_count":
        coef = [0.5, 0.01]
    elif case == "too_many_modes":
        coef = [0.5] + [0.001] * (2 * iim.MAX_FOURIER_MODES + 2)
    elif case == "no_coef":
        coef = None
    elif case == "negative_radius":
        coef = [0.1, 0.2, 0.0]
    elif case == "grid_no_phi":
        kind, coef = iim.GEOM["levelset_grid"], None
    elif case == "fourier_3d":
        dim = 3
    d = iim.make_desc(dim, 64, kind, (0.0, 0.0), False, iim.BC["dirichlet"], 0, order=4, coef=coef)
    h = ctypes.c_void_p()
    st = lib.iim_problem_create(ctypes.byref(d), ctypes.byref(iim.default_options()), None, ctypes.byref(h))
    assert st == iim.IIM_ERR_INVALID_ARG and not h.value, (case, st)
