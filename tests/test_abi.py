"""The C ABI library loads and exports every entry point include/oq.h
declares (no compute call: this runs without a GPU)."""
import os
import re
import ctypes

from paper_2202_07388_gb300 import oq, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?[a-z_]+\*?\s+\*?(oq_[a-z0-9_]+)\s*\(", src, flags=re.M))
    return names


def test_library_exports_every_declared_symbol():
    build.build()
    lib = oq.lib()
    names = declared()
    assert "oq_dw_hat_apply" in names and "oq_cgne_solve" in names
    for n in sorted(names):
        assert hasattr(lib, n), n
    assert set(oq.exported_symbols()) >= names


def test_error_strings_and_argument_checks():
    lib = oq.lib()
    assert lib.oq_error_string(0) == b"ok"
    assert lib.oq_error_string(-1) == b"invalid argument"
    h = ctypes.c_void_p()
    bad = (oq.OqLattice * 1)()
    bad[0].L[0], bad[0].L[1], bad[0].L[2], bad[0].L[3], bad[0].bc_t = 3, 4, 4, 4, -1   # odd extent
    assert lib.oq_create(ctypes.byref(h), bad, 1) == oq.ERR_ARG
    assert lib.oq_dw_apply(None, 0, 1, None, None, 1, 0, None) == oq.ERR_ARG
