"""The C ABI on a machine without a GPU: the library builds, loads, exports every function that
include/*.h declares, and its host-side logic (argument validation, footprint sizing for
admission, error reporting) works before any device call."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b((?:ipeps|ctmrg)_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1910_11359_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


@pytest.mark.parametrize("header", ["ipeps.h", "ipeps_kernels.h"])
def test_every_declared_function_is_exported(lib, header):
    names = _declared(header)
    assert len(names) >= 8
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def _params(**kw):
    import paper_1910_11359_gb300._lib as L
    p = dict(J=[1.0, 1.0], V=[1.0, 0.0], h=[5.0, 2.0], D=3, chi=18, order=2, dt=0.05, precision=0,
             seed=0, d_A=2)
    p.update(kw)
    return L._params(p["J"], p["V"], p["h"], p["D"], p["chi"], p["order"], p["dt"], p["precision"],
                     p["seed"], d_A=p["d_A"])


def test_footprint_sizing_without_device():
    import paper_1910_11359_gb300 as pkg
    one = pkg.footprint_bytes([1.0], [1.0], [5.0], D=3, chi=18)
    three = pkg.footprint_bytes([1.0] * 3, [1.0] * 3, [1.0, 5.0, 10.0], D=3, chi=18)
    big = pkg.footprint_bytes([1.0], [1.0], [5.0], D=4, chi=32)
    split = pkg.footprint_bytes([1.0], [1.0], [5.0], D=4, chi=32, precision=pkg.SPLIT_BF16X3)
    assert 0 < one < three < 3.5 * one          # per-instance arrays plus shared tables
    assert big > 2 * one
    assert split > big                           # the tensor-core operand workspace
    levels3 = pkg.footprint_bytes([1.0], [1.0], [5.0], D=3, chi=18, d_A=3)
    assert levels3 > one                         # d = 6: larger site tensors, gates and readout


@pytest.mark.parametrize("kw,status", [
    (dict(chi=4), 1),                 # chi < D^2
    (dict(order=3), 1),               # Trotter order
    (dict(D=0), 1),
    (dict(precision=7), 1),
    (dict(chi=4096), 8),              # beyond the supported chi
    (dict(d_A=6), 1),                 # more disorder levels than the library takes
    (dict(d_A=1), 1),
    (dict(d_A=3, D=2, chi=8), 8),     # the reduced simple update needs D^2 >= d = 6
])
def test_invalid_parameters_are_rejected_before_any_device_call(lib, kw, status):
    import paper_1910_11359_gb300._lib as L
    p, keep = _params(**kw)
    h = ctypes.c_void_p(None)
    rc = L.lib().ipeps_init(ctypes.byref(p), None, ctypes.byref(h))
    assert rc == status
    assert not h.value
    msg = L.lib().ipeps_last_error(None)
    assert msg and len(msg) > 5


def test_null_handles_and_bad_sizes_fail_cleanly(lib):
    """Every entry point refuses a NULL handle or an impossible size with IPEPS_EINVAL (1) and a
    message, without touching the device; destroying NULL is a no-op."""
    vp = ctypes.c_void_p
    lib.ipeps_last_error.restype = ctypes.c_char_p
    calls = [
        lambda: lib.ipeps_set_tensors(vp(None), vp(None), vp(None), vp(None)),
        lambda: lib.ipeps_trotter_step(vp(None), 1, vp(None)),
        lambda: lib.ctmrg_reset(vp(None)),
        lambda: lib.ctmrg_converge(vp(None), ctypes.c_double(1e-10), 10, vp(None), vp(None)),
        lambda: lib.ipeps_measure(vp(None), vp(None)),
        lambda: lib.ipeps_corner_spectrum(vp(None), 0, 0, 0, vp(None)),
        lambda: lib.ipeps_get_lambda(vp(None), vp(None)),
        lambda: lib.ipeps_get_tensors(vp(None), vp(None), vp(None)),
        lambda: lib.ipeps_get_env(vp(None), 0, vp(None), vp(None)),
        lambda: lib.ipeps_set_env(vp(None), 0, vp(None), vp(None)),
        lambda: lib.ipeps_set_graphs(vp(None), 1),
        lambda: lib.ipeps_ed_bytes(vp(None), vp(None)),
        # m < n, and a batch beyond the allocation-free entry point's fixed scratch
        lambda: lib.ipeps_kernel_svd(3, 5, 1, vp(1), vp(None), vp(1), vp(None), ctypes.c_double(1e-14),
                                     10, vp(None), vp(None)),
        lambda: lib.ipeps_kernel_svd_noalloc(8, 8, 5000, vp(1), vp(None), vp(1), vp(None),
                                             ctypes.c_double(1e-14), 10, vp(None), vp(None)),
    ]
    for call in calls:
        assert call() == 1
        assert len(lib.ipeps_last_error(vp(None)) or b"") > 5
    assert lib.ipeps_destroy(vp(None)) == 0


def test_noalloc_svd_rejects_blocks_beyond_shared_memory(lib):
    """The allocation-free SVD keeps the columns in shared memory only: a block too tall for the
    cluster's shared memory, which ipeps_kernel_svd still serves from a global-memory column buffer,
    is refused with IPEPS_EUNSUPPORTED (8) before any device call."""
    vp = ctypes.c_void_p
    lib.ipeps_last_error.restype = ctypes.c_char_p
    rc = lib.ipeps_kernel_svd_noalloc(2592, 80, 1, vp(1), vp(None), vp(1), vp(None),
                                      ctypes.c_double(1e-14), 10, vp(None), vp(None))
    assert rc == 8
    assert b"shared memory" in lib.ipeps_last_error(vp(None))


def test_ed_rejects_before_any_device_work():
    """The ED entry point validates on the host: a 40 x 40 lattice is beyond the device eigensolver
    (EUNSUPPORTED), bad sizes are EINVAL, non-finite fields ENAN; ed_bytes sizes a 20 x 20 run."""
    import ctypes
    import numpy as np
    import paper_1910_11359_gb300 as pkg
    from paper_1910_11359_gb300._lib import EdParams
    assert 400 <= pkg.ed_max_sites() < 1600
    out = np.zeros(4)
    sw = np.zeros(2, dtype=np.int32)
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    ip = sw.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    f = np.zeros(1600)
    t = np.zeros(1)
    p = EdParams(Lx=40, Ly=40, R=1, J=1.0, T=1, bin_width=0.05)
    assert pkg.lib().ipeps_ed_run(ctypes.byref(p), dp(f), dp(t), dp(out), dp(out), dp(out), None, None, ip,
                                  None) == 8
    p = EdParams(Lx=4, Ly=4, R=0, J=1.0, T=1, bin_width=0.05)
    assert pkg.lib().ipeps_ed_run(ctypes.byref(p), dp(f), dp(t), dp(out), dp(out), dp(out), None, None, ip,
                                  None) == 1
    f[3] = np.nan
    p = EdParams(Lx=4, Ly=4, R=1, J=1.0, T=1, bin_width=0.05)
    assert pkg.lib().ipeps_ed_run(ctypes.byref(p), dp(f), dp(t), dp(out), dp(out), dp(out), None, None, ip,
                                  None) == 4
    b = ctypes.c_size_t()
    p = EdParams(Lx=20, Ly=20, R=100, J=1.0, T=51, bin_width=0.05)
    assert pkg.lib().ipeps_ed_bytes(ctypes.byref(p), ctypes.byref(b)) == 0 and b.value > 10 ** 8
