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
    for p in (6, 9, 11, 19):
        st = lib.tmg_setup(ctypes.byref(h), p, 0.1, 1.0, 16, 0, 0.0, None, None)
        assert st == tmg.TMG_EUNSUPPORTED, (p, st)
    st = lib.tmg_setup(ctypes.byref(h), 1, 0.1, 1.0, 16, 0, 2.5, None, None)
    assert st == tmg.TMG_EINVAL


def test_batched_setup_rejects_bad_arguments_before_touching_the_gpu():
    """tmg_setup_batched validates every instance and the options on the host:
    degrees 0..5, 10 and 20 (other degrees up to 20 are unsupported), tau > 0,
    lambda >= 0 (finite), N >= 1, V- or W-cycles, a known schedule, omega < 2."""
    import numpy as np
    lib = tmg._lib()
    h = ctypes.c_void_p()

    def call(p, tau, lam, N, omega=0.0, **opt):
        n = len(p)
        pa = np.asarray(p, dtype=np.int32)
        ta = np.asarray(tau, dtype=np.float64)
        la = np.asarray(lam, dtype=np.float64)
        Na = np.asarray(N, dtype=np.int64)
        o = tmg._Opts()
        lib.tmg_opts_default(ctypes.byref(o))
        for k, v in opt.items():
            setattr(o, k, v)
        ip, dp, lp = (ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                      ctypes.POINTER(ctypes.c_int64))
        return lib.tmg_setup_batched(ctypes.byref(h), n, pa.ctypes.data_as(ip), ta.ctypes.data_as(dp),
                                     la.ctypes.data_as(dp), Na.ctypes.data_as(lp), omega, ctypes.byref(o), None)

    ok = ([1, 2], [0.1, 0.1], [1.0, 2.0], [64, 128])
    bad_instances = [
        ([1, 21], [0.1, 0.1], [1.0, 2.0], [64, 128]),      # p_t = 21 (degrees go to 20)
        ([1, -1], [0.1, 0.1], [1.0, 2.0], [64, 128]),
        ([1, 2], [0.1, 0.0], [1.0, 2.0], [64, 128]),       # tau = 0
        ([1, 2], [0.1, 0.1], [1.0, -2.0], [64, 128]),      # lambda < 0
        ([1, 2], [0.1, 0.1], [1.0, float("inf")], [64, 128]),
        ([1, 2], [0.1, 0.1], [1.0, 2.0], [64, 0]),         # N = 0
    ]
    for args in bad_instances:
        assert call(*args) == tmg.TMG_EINVAL, args
    for p in (6, 9, 19):                                      # degrees up to 20 that are not built
        assert call([1, p], [0.1, 0.1], [1.0, 2.0], [64, 128]) == tmg.TMG_EUNSUPPORTED, p
    assert call(*ok, omega=2.5) == tmg.TMG_EINVAL
    assert call(*ok, gamma=3) == tmg.TMG_EINVAL              # V- or W-cycles only
    assert call(*ok, schedule=3) == tmg.TMG_EINVAL
    assert call(*ok, nu1=0, nu2=0) == tmg.TMG_EINVAL
    assert call([], [], [], []) == tmg.TMG_EINVAL             # no instances


def test_heat_setup_rejects_bad_arguments_before_any_device_call():
    """tmg_heat_setup validates sizes and options on the host and returns
    TMG_EINVAL before it touches the device (runs without a GPU)."""
    import ctypes
    from paper_1409_5254_gb300 import tmg
    L = tmg._lib()
    o = tmg._opts(precision="mixed")
    h = ctypes.c_void_p()
    bad = [(1, 1e-3, 6, 16, 2),      # n + 1 not a power of two
           (1, 1e-3, 7, 12, 2),      # N not a power of two
           (6, 1e-3, 7, 16, 2),      # degree above 5
           (1, 0.0, 7, 16, 2),       # tau <= 0
           (1, 1e-3, 1 << 14, 16, 2),  # n too large for 32-bit offsets
           (1, 1e-3, 7, 16, 0)]      # nu_c < 1
    for p, tau, n, N, nuc in bad:
        st = L.tmg_heat_setup(ctypes.byref(h), p, tau, n, N, ctypes.byref(o), nuc, None)
        assert st == tmg.TMG_EINVAL, (p, tau, n, N, nuc, st)
    o.gamma = 2
    assert L.tmg_heat_setup(ctypes.byref(h), 1, 1e-3, 7, 16, ctypes.byref(o), 2, None) == tmg.TMG_EINVAL


def test_debug_bounds_query_without_the_debug_build():
    """The normal library has no bounds records: tmg_debug_bounds answers
    TMG_EUNSUPPORTED (no device access)."""
    import ctypes
    from paper_1409_5254_gb300 import tmg
    c, f = ctypes.c_uint(1), ctypes.c_ulonglong(1)
    assert tmg._lib().tmg_debug_bounds(ctypes.byref(c), ctypes.byref(f)) == tmg.TMG_EUNSUPPORTED
    assert c.value == 0 and f.value == 0
