"""The C-ABI library loads and exports every entry point that include/hfe.h declares, the
host-only entry points fill the documented defaults, the binding's structs match the
header's layouts and its marshalling is consistent (CPU only, no compute call)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2606_17390_b300 import hfe

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "hfe.h")


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:hfe_status|void|const char\*)\s+(hfe_\w+)\s*\(", txt, re.M)))


def test_header_declares_entry_points():
    names = _declared()
    for n in ("hfe_create", "hfe_destroy", "hfe_gp_sweep", "hfe_forward", "hfe_adjoint", "hfe_solve",
              "hfe_spmv", "hfe_get_bsr", "hfe_set_state", "hfe_get_state", "hfe_set_material"):
        assert n in names


def test_library_exports_every_declared_symbol():
    if not os.path.exists(hfe.LIB_PATH):
        from paper_2606_17390_b300 import build
        build.build()
    L = ctypes.CDLL(hfe.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_default_options(precision):
    L = hfe.lib()
    o = hfe.Options()
    L.hfe_default_options(ctypes.byref(o), hfe.PRECISION[precision])
    assert o.precision == hfe.PRECISION[precision]
    assert o.newton_rtol == (1e-10 if precision == "fp64" else 1e-7)
    assert o.local_maxit > 0 and o.pcg_maxit > 0 and o.pcg_check_every > 0
    assert o.predictor == 2     # linear extrapolation (Sec. 2.2, automatic time stepping)


def test_null_arguments_rejected_without_device_work():
    L = hfe.lib()
    assert L.hfe_create(None, None, None, None, None, None) == -1
    assert L.hfe_get_info(None, None) == -1
    assert L.hfe_last_error(None) == b"null handle"
    L.hfe_set_warm_start.argtypes = [ctypes.c_void_p, ctypes.c_int]
    assert L.hfe_set_warm_start(None, 0) == -1


def test_ctypes_mirrors_match_the_header_layout(tmp_path):
    """Every struct of include/hfe.h that the binding mirrors has the same size and field
    offsets in ctypes as in C (the header compiled by the host compiler)."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    mirrors = {"hfe_mesh": hfe._Mesh, "hfe_bc": hfe._BC, "hfe_material": hfe._Material,
               "hfe_options": hfe.Options, "hfe_stats": hfe.Stats, "hfe_info": hfe.Info,
               "hfe_barlat_material": hfe.BarlatMaterialC, "hfe_cpp_options": hfe.CppOptions}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "hfe.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            a, b, c = line.split()
            got[(a, b)] = int(c)
    for cname, py in mirrors.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_binding_marshalling_without_device_work():
    """Host-side argument marshalling of the binding: parameter arrays (uniform or per element,
    material frames dropped when they are the identity, one frame repeated for per-element
    parameters), the Barlat material record, and the local-projection options, whose Python
    defaults equal the library's hfe_default_cpp_options."""
    th = np.arange(11.0)
    a, T = hfe.material_arrays(th)
    assert a.shape == (1, 11) and T is None
    a, T = hfe.material_arrays(np.tile(th, (3, 1)), np.eye(3))
    assert a.shape == (3, 11) and T is None
    R = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    a, T = hfe.material_arrays(np.tile(th, (3, 1)), R)
    assert T.shape == (3, 9) and np.array_equal(T[2], R.ravel())
    from paper_2606_17390_b300 import inputs
    m = inputs.barlat_verification_material()
    s = hfe.barlat_material(m)
    assert list(s.c1) == list(m.c1) and list(s.c2) == list(m.c2) and s.m == m.m
    assert s.orthotropic == 0 and list(s.Theta) == list(np.eye(3).ravel())
    L = hfe.lib()
    o = hfe.CppOptions()
    L.hfe_default_cpp_options.argtypes = [ctypes.POINTER(hfe.CppOptions)]
    L.hfe_default_cpp_options.restype = None
    L.hfe_default_cpp_options(ctypes.byref(o))
    p = hfe.cpp_options()
    assert [getattr(o, f) for f, _ in o._fields_] == [getattr(p, f) for f, _ in p._fields_]
