"""The C-ABI library loads and exports every entry point that include/hfe.h declares, and the
host-only entry point fills the documented defaults (CPU only, no compute call)."""
import ctypes
import os
import re

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


def test_null_arguments_rejected_without_device_work():
    L = hfe.lib()
    assert L.hfe_create(None, None, None, None, None, None) == -1
    assert L.hfe_get_info(None, None) == -1
    assert L.hfe_last_error(None) == b"null handle"
