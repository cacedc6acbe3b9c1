"""ctypes binding of libipeps (argument marshalling only; every computation runs in the library).

The shared library is built in-tree by ``paper_1910_11359_gb300.build``.  Loading fails loudly if
it is missing: there is no fallback path.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libipeps.so")

FP64, SPLIT_BF16X3, SPLIT_TF32X3 = 0, 1, 2
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ENOCONV", 4: "ENAN", 5: "ECUDA", 6: "ETIMEOUT",
          7: "EBUSY", 8: "EUNSUPPORTED"}
ENOCONV = 3


class IpepsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class EdParams(ctypes.Structure):
    _fields_ = [("Lx", ctypes.c_int), ("Ly", ctypes.c_int), ("R", ctypes.c_int), ("J", ctypes.c_double),
                ("T", ctypes.c_int), ("bin_width", ctypes.c_double)]


class Params(ctypes.Structure):
    _fields_ = [("batch", ctypes.c_int), ("d_A", ctypes.c_int), ("D", ctypes.c_int),
                ("chi", ctypes.c_int), ("trotter_order", ctypes.c_int), ("dt", ctypes.c_double),
                ("precision", ctypes.c_int), ("seed", ctypes.c_ulonglong),
                ("J", ctypes.POINTER(ctypes.c_double)), ("V", ctypes.POINTER(ctypes.c_double)),
                ("h", ctypes.POINTER(ctypes.c_double)), ("ctm_cut_rel", ctypes.c_double),
                ("projector_svd", ctypes.c_int)]


class Obs(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("nA", ctypes.c_double), ("nB", ctypes.c_double),
                ("imbalance", ctypes.c_double), ("tauzA", ctypes.c_double),
                ("tauzB", ctypes.c_double), ("energy", ctypes.c_double),
                ("purityA", ctypes.c_double), ("trunc_err_acc", ctypes.c_double),
                ("ctm_sweeps", ctypes.c_int), ("ctm_delta", ctypes.c_double),
                ("renyi1A", ctypes.c_double), ("renyi_halfA", ctypes.c_double),
                ("renyi2A", ctypes.c_double)]


_lib = None
EXPORTS = ["ipeps_init", "ipeps_set_tensors", "ipeps_trotter_step", "ctmrg_converge", "ctmrg_reset",
           "ipeps_measure", "ipeps_corner_spectrum", "ipeps_get_lambda", "ipeps_get_tensors",
           "ipeps_footprint_bytes", "ipeps_destroy", "ipeps_last_error", "ipeps_kernel_zgemm",
           "ipeps_kernel_permute", "ipeps_kernel_svd", "ipeps_kernel_gate", "ipeps_launch_count",
           "ipeps_profile_enable", "ipeps_profile_classes", "ipeps_profile_name", "ipeps_profile_read",
           "ipeps_kernel_fp64_peak", "ipeps_kernel_svd_noalloc", "ipeps_kernel_zgemm_split",
           "ipeps_get_env", "ipeps_set_env", "ipeps_profile_tc_executed", "ipeps_profile_counters",
           "ipeps_kernel_orth", "ipeps_kernel_zgemm_split_tf32", "ipeps_set_graphs", "ipeps_ed_max_sites",
           "ipeps_ed_bytes", "ipeps_ed_run"]


def lib():
    """Load libipeps.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libipeps.so not built: run `python -m paper_1910_11359_gb300.build`")
    L = ctypes.CDLL(LIB_PATH)
    P, vp, i, d, dp, ip = (ctypes.POINTER, ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int))
    ll = ctypes.c_longlong
    L.ipeps_init.argtypes = [P(Params), vp, P(vp)]
    L.ipeps_set_tensors.argtypes = [vp, dp, dp, dp]
    L.ipeps_trotter_step.argtypes = [vp, i, dp]
    L.ctmrg_converge.argtypes = [vp, d, i, ip, dp]
    L.ctmrg_reset.argtypes = [vp]
    L.ipeps_set_graphs.argtypes = [vp, i]
    L.ipeps_ed_max_sites.argtypes = []
    L.ipeps_ed_bytes.argtypes = [P(EdParams), P(ctypes.c_size_t)]
    L.ipeps_ed_run.argtypes = [P(EdParams), dp, dp, dp, dp, dp, dp, dp, ip, vp]
    L.ipeps_measure.argtypes = [vp, P(Obs)]
    L.ipeps_corner_spectrum.argtypes = [vp, i, i, i, dp]
    L.ipeps_get_lambda.argtypes = [vp, dp]
    L.ipeps_get_tensors.argtypes = [vp, dp, dp]
    L.ipeps_get_env.argtypes = [vp, i, dp, dp]
    L.ipeps_set_env.argtypes = [vp, i, dp, dp]
    L.ipeps_footprint_bytes.argtypes = [P(Params), P(ctypes.c_size_t)]
    L.ipeps_destroy.argtypes = [vp]
    L.ipeps_last_error.argtypes = [vp]
    L.ipeps_last_error.restype = ctypes.c_char_p
    L.ipeps_kernel_zgemm.argtypes = [i, i, i, i, i, i, vp, ll, ll, vp, ll, ll, vp, ll, ll, vp]
    L.ipeps_kernel_permute.argtypes = [vp, vp, i, ip, ip, i, ll, ll, vp]
    L.ipeps_kernel_svd.argtypes = [i, i, i, vp, vp, vp, vp, d, i, vp, vp]
    L.ipeps_kernel_gate.argtypes = [d, d, d, d, dp]
    L.ipeps_launch_count.argtypes = []
    L.ipeps_launch_count.restype = ctypes.c_ulonglong
    L.ipeps_profile_enable.argtypes = [i]
    L.ipeps_profile_classes.argtypes = []
    L.ipeps_profile_name.argtypes = [i]
    L.ipeps_profile_name.restype = ctypes.c_char_p
    L.ipeps_profile_read.argtypes = [dp, dp, P(ctypes.c_ulonglong)]
    L.ipeps_profile_tc_executed.argtypes = [dp]
    L.ipeps_profile_counters.argtypes = [P(ctypes.c_ulonglong), i]
    L.ipeps_kernel_orth.argtypes = [i, i, i, vp, vp, i, vp, vp]
    L.ipeps_kernel_fp64_peak.argtypes = [dp]
    L.ipeps_kernel_svd_noalloc.argtypes = [i, i, i, vp, vp, vp, vp, d, i, vp, vp]
    L.ipeps_kernel_zgemm_split.argtypes = [i, i, i, i, i, i, vp, ll, ll, vp, ll, ll, vp, ll, ll, vp]
    L.ipeps_kernel_zgemm_split_tf32.argtypes = [i, i, i, i, i, i, vp, ll, ll, vp, ll, ll, vp, ll, ll, vp]
    for name in EXPORTS:
        if name not in ("ipeps_last_error", "ipeps_launch_count", "ipeps_profile_name"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(rc, handle=None, allow=()):
    if rc != 0 and rc not in allow:
        msg = lib().ipeps_last_error(handle)
        raise IpepsError(rc, msg.decode() if msg else "")
    return rc


def _params(J, V, h, D, chi, order, dt, precision, seed, cut_rel=0.0, projector_svd=0, d_A=2):
    J = np.ascontiguousarray(np.atleast_1d(J), dtype=np.float64)
    V = np.ascontiguousarray(np.broadcast_to(np.atleast_1d(V), J.shape), dtype=np.float64)
    h = np.ascontiguousarray(np.broadcast_to(np.atleast_1d(h), J.shape), dtype=np.float64)
    p = Params(batch=len(J), d_A=d_A, D=D, chi=chi, trotter_order=order, dt=dt, precision=precision,
               seed=seed, J=_dptr(J), V=_dptr(V), h=_dptr(h), ctm_cut_rel=cut_rel,
               projector_svd=projector_svd)
    return p, (J, V, h)


def footprint_bytes(J, V, h, D, chi, order=2, dt=0.05, precision=FP64, seed=0, d_A=2):
    p, keep = _params(J, V, h, D, chi, order, dt, precision, seed, d_A=d_A)
    out = ctypes.c_size_t(0)
    _check(lib().ipeps_footprint_bytes(ctypes.byref(p), ctypes.byref(out)))
    return out.value


class IPEPS:
    """One library handle: ``batch`` = len(J) instances with shared D, chi, Trotter order and dt."""

    def __init__(self, J, V, h, D, chi, order=1, dt=0.02, precision=FP64, seed=0, stream=None,
                 cut_rel=0.0, projector_svd=0, d_A=2):
        p, self._keep = _params(J, V, h, D, chi, order, dt, precision, seed, cut_rel, projector_svd, d_A)
        self.batch, self.D, self.chi, self.d = p.batch, D, chi, 2 * d_A
        self._h = ctypes.c_void_p(None)
        st = ctypes.c_void_p(stream) if stream else None
        _check(lib().ipeps_init(ctypes.byref(p), st, ctypes.byref(self._h)))

    def close(self):
        if self._h:
            lib().ipeps_destroy(self._h)
            self._h = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tensors(self, GA, GB, lam=None):
        shape = (self.batch, self.d) + (self.D,) * 4
        GA = np.ascontiguousarray(np.broadcast_to(GA, shape), dtype=np.complex128)
        GB = np.ascontiguousarray(np.broadcast_to(GB, shape), dtype=np.complex128)
        lp = None
        if lam is not None:
            lam = np.ascontiguousarray(np.broadcast_to(lam, (self.batch, 4, self.D)), dtype=np.float64)
            lp = _dptr(lam)
        _check(lib().ipeps_set_tensors(self._h, _dptr(GA.view(np.float64)),
                                       _dptr(GB.view(np.float64)), lp), self._h)

    def trotter_step(self, n=1, sync=True):
        eps = np.zeros(self.batch)
        _check(lib().ipeps_trotter_step(self._h, n, _dptr(eps) if sync else None), self._h)
        return eps

    def ctmrg_converge(self, tol=1e-10, max_sweeps=500, allow_noconv=False):
        sw = np.zeros(self.batch, dtype=np.int32)
        dl = np.zeros(self.batch)
        rc = lib().ctmrg_converge(self._h, tol, max_sweeps,
                                  sw.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dptr(dl))
        _check(rc, self._h, allow=(ENOCONV,) if allow_noconv else ())
        return sw, dl, rc

    def ctmrg_reset(self):
        _check(lib().ctmrg_reset(self._h), self._h)

    def set_graphs(self, enable=True):
        """Converge through one CUDA graph (default) or from the host loop."""
        _check(lib().ipeps_set_graphs(self._h, 1 if enable else 0), self._h)

    def measure(self):
        arr = (Obs * self.batch)()
        _check(lib().ipeps_measure(self._h, arr), self._h)
        return [{k: getattr(o, k) for k, _ in Obs._fields_} for o in arr]

    def corner_spectrum(self, inst, pos, corner):
        out = np.zeros(self.chi)
        _check(lib().ipeps_corner_spectrum(self._h, inst, pos, corner, _dptr(out)), self._h)
        return out

    def get_lambda(self):
        out = np.zeros((self.batch, 4, self.D))
        _check(lib().ipeps_get_lambda(self._h, _dptr(out)), self._h)
        return out

    def get_env(self, inst=0):
        """(C, T) of instance ``inst``: C[i][pos] (chi x chi), T[i][pos] (chi x D^2 x chi),
        i = 0..3 for C1..C4 / T1..T4, pos = x + 2 y."""
        C = np.zeros((4, 4, self.chi, self.chi), dtype=np.complex128)
        T = np.zeros((4, 4, self.chi, self.D * self.D, self.chi), dtype=np.complex128)
        _check(lib().ipeps_get_env(self._h, inst, _dptr(C.view(np.float64)),
                                   _dptr(T.view(np.float64))), self._h)
        return C, T

    def set_env(self, C, T, inst=0):
        C = np.ascontiguousarray(C, dtype=np.complex128)
        T = np.ascontiguousarray(T, dtype=np.complex128)
        assert C.shape == (4, 4, self.chi, self.chi) and T.shape == (4, 4, self.chi, self.D ** 2, self.chi)
        _check(lib().ipeps_set_env(self._h, inst, _dptr(C.view(np.float64)),
                                   _dptr(T.view(np.float64))), self._h)

    def get_tensors(self):
        shape = (self.batch, self.d) + (self.D,) * 4
        GA = np.zeros(shape, dtype=np.complex128)
        GB = np.zeros(shape, dtype=np.complex128)
        _check(lib().ipeps_get_tensors(self._h, _dptr(GA.view(np.float64)),
                                       _dptr(GB.view(np.float64))), self._h)
        return GA, GB


def launch_count():
    """Kernels launched by the library since it was loaded."""
    return int(lib().ipeps_launch_count())


def profile_enable(on=True):
    _check(lib().ipeps_profile_enable(1 if on else 0))


def profile_read():
    """Per kernel class: {name: (ms, flops, launches)} accumulated since profile_enable(True)."""
    L = lib()
    n = L.ipeps_profile_classes()
    ms, fl = np.zeros(n), np.zeros(n)
    cnt = np.zeros(n, dtype=np.uint64)
    _check(L.ipeps_profile_read(_dptr(ms), _dptr(fl), cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_ulonglong))))
    return {L.ipeps_profile_name(k).decode(): (float(ms[k]), float(fl[k]), int(cnt[k])) for k in range(n)}


def profile_tc_executed():
    """Executed tensor-pipe flops of the tcgen05 GEMM launches since profile_enable(True)."""
    out = ctypes.c_double(0.0)
    _check(lib().ipeps_profile_tc_executed(ctypes.byref(out)))
    return out.value


COUNTERS = ("jacobi_problems", "jacobi_rounds", "jacobi_sweeps", "subspace_rounds",
            "subspace_accepted", "subspace_unconverged", "orth_fallback")


def profile_counters():
    """Device-side work counters since profile_enable(True), as a dict (see COUNTERS)."""
    out = np.zeros(len(COUNTERS), dtype=np.uint64)
    _check(lib().ipeps_profile_counters(out.ctypes.data_as(ctypes.POINTER(ctypes.c_ulonglong)), len(COUNTERS)))
    return {k: int(v) for k, v in zip(COUNTERS, out)}


def fp64_peak_tflops():
    out = ctypes.c_double(0.0)
    _check(lib().ipeps_kernel_fp64_peak(ctypes.byref(out)))
    return out.value


def ed_max_sites():
    """Largest lattice (Lx * Ly sites) the free-fermion ED workload accepts."""
    return lib().ipeps_ed_max_sites()


def ed_run(Lx, Ly, J, fields, times, bin_width=0.05, stream=None):
    """Free-fermion ED of R realisations (fields [R][Lx*Ly]) on the device: realisation-averaged
    even / odd occupations at `times`, averaged cumulative IPR, spectra and IPRs per realisation,
    Jacobi sweeps per realisation (include/ipeps_ed.h)."""
    f = np.ascontiguousarray(np.atleast_2d(fields), dtype=np.float64)
    t = np.ascontiguousarray(times, dtype=np.float64)
    R, N = f.shape
    if N != Lx * Ly:
        raise ValueError("fields must have Lx * Ly columns")
    p = EdParams(Lx=Lx, Ly=Ly, R=R, J=J, T=len(t), bin_width=bin_width)
    nb = int(np.ceil(1.0 / bin_width - 1e-9))
    ev, od, cum = np.zeros(len(t)), np.zeros(len(t)), np.zeros(nb)
    spec, ipr = np.zeros((R, N)), np.zeros((R, N))
    sw = np.zeros(R, dtype=np.int32)
    rc = lib().ipeps_ed_run(ctypes.byref(p), _dptr(f), _dptr(t), _dptr(ev), _dptr(od), _dptr(cum),
                            _dptr(spec), _dptr(ipr), sw.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                            stream)
    _check(rc)
    return dict(n_even=ev, n_odd=od, cum_ipr=cum, spectra=spec, ipr=ipr, sweeps=sw)
