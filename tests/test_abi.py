"""Host-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every function include/tmg.h declares.  No compute calls (no GPU)."""
import ctypes
import os
import re

from paper_1409_5254_gb300 import build_ext, tmg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(tmg_[a-z_0-9]+)\s*\(", text))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    path = build_ext.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert {"tmg_setup", "tmg_solve", "tmg_destroy"} <= names
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing
    assert set(tmg.EXPORTS) <= names


def test_strerror_and_defaults_without_gpu():
    lib = tmg._lib()
    assert lib.tmg_strerror(0) == b"ok"
    assert b"unsupported" in lib.tmg_strerror(7)
    o = tmg._Opts()
    lib.tmg_opts_default(ctypes.byref(o))
    assert o.tol == 1e-10 and o.nu1 == 1 and o.nu2 == 1 and o.gamma == 1 and o.precision == tmg.MIXED


def test_setup_rejects_bad_arguments_before_touching_the_gpu():
    lib = tmg._lib()
    h = ctypes.c_void_p()
    bad = [(21, 0.1, 1.0, 16), (1, 0.0, 1.0, 16), (1, 0.1, -1.0, 16), (1, 0.1, 1.0, 0),
           (1, float("nan"), 1.0, 16), (-1, 0.1, 1.0, 16)]
    for p, tau, lam, N in bad:
        st = lib.tmg_setup(ctypes.byref(h), p, tau, lam, N, 0, 0.0, None, None)
        assert st == tmg.TMG_EINVAL, (p, tau, lam, N, st)
    # degrees up to 20 that are not built
    for p in (6, 9, 11, 20):
        st = lib.tmg_setup(ctypes.byref(h), p, 0.1, 1.0, 16, 0, 0.0, None, None)
        assert st == tmg.TMG_EUNSUPPORTED, (p, st)
    st = lib.tmg_setup(ctypes.byref(h), 1, 0.1, 1.0, 16, 0, 2.5, None, None)
    assert st == tmg.TMG_EINVAL
