"""ctypes front end of the C oracle in ``cwm_oracle.c``.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU-baseline
leg use it; the CUDA path never imports it.  The C file states every reading of the
paper it takes; this module only marshals numpy arrays.

Matrices are CSR triples (row_ptr int32[n+1], col int32[nnz], val float64[nnz]) with
ascending columns per row.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cwm_oracle.c")
_LIBDIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIBDIR, "libcwm_oracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_NOT_SPD, ERR_OOM, ERR_BREAKDOWN, ERR_NOT_CONVERGED = 0, 1, 2, 4, 6, 7
PREC_AMG, PREC_IDENTITY, PREC_L1JACOBI = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction).  Returns the library path."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        vp, i, l, d = C.c_void_p, C.c_int, C.c_long, C.c_double
        sig = {
            "or_check_csr": (i, [i, _i32p, _i32p]),
            "or_paper_coarse_max": (i, [i]),
            "or_check_symmetric": (i, [i, _i32p, _i32p, _f64p]),
            "or_edge_weights": (i, [i, _i32p, _i32p, _f64p, _f64p, _f64p]),
            "or_greedy_match": (i, [i, _i32p, _i32p, _f64p, _i32p]),
            "or_suitor_match": (i, [i, _i32p, _i32p, _f64p, _i32p]),
            "or_aggregate": (i, [i, _i32p, _i32p, C.POINTER(i), C.POINTER(i)]),
            "or_prolongator": (i, [i, i, _i32p, _f64p, _f64p, _f64p]),
            "or_galerkin_nnz": (l, [i, _i32p, _i32p, _f64p, i, _i32p, _f64p]),
            "or_galerkin": (i, [i, _i32p, _i32p, _f64p, i, _i32p, _f64p, i, _i32p, _i32p, _f64p]),
            "or_setup": (vp, [i, _i32p, _i32p, _f64p, _f64p, i, i, i, d, i, C.POINTER(i)]),
            "or_set_cycle": (None, [vp, i, i, i]),
            "or_set_gamma": (None, [vp, i]),
            "or_num_levels": (i, [vp]),
            "or_level_n": (i, [vp, i]),
            "or_level_nnz": (l, [vp, i]),
            "or_level_sweeps": (i, [vp, i]),
            "or_sweep_n": (i, [vp, i, i]),
            "or_level_export": (None, [vp, i, vp, vp, vp, vp, vp, vp, vp]),
            "or_sweep_mate": (None, [vp, i, i, _i32p]),
            "or_l1_jacobi": (None, [vp, i, _f64p, _f64p, i]),
            "or_vcycle": (None, [vp, _f64p, _f64p]),
            "or_pcg": (i, [vp, _f64p, _f64p, d, i, i, C.POINTER(i), C.POINTER(d), C.POINTER(d)]),
            "or_stats": (None, [vp, C.POINTER(d), C.POINTER(d)]),
            "or_free": (None, [vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _csr(rp, ci, val):
    rp = np.ascontiguousarray(rp, dtype=np.int32)
    ci = np.ascontiguousarray(ci, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    return rp, ci, val


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def check_csr(rp, ci) -> bool:
    rp, ci, _ = _csr(rp, ci, np.zeros(0))
    return _load().or_check_csr(len(rp) - 1, rp, ci) == OK


def check_symmetric(rp, ci, val) -> bool:
    rp, ci, val = _csr(rp, ci, val)
    return _load().or_check_symmetric(len(rp) - 1, rp, ci, val) == OK


def edge_weights(rp, ci, val, v):
    """Per-slot weights c_ij (0 on the diagonal and on ineligible entries)."""
    rp, ci, val = _csr(rp, ci, val)
    v = np.ascontiguousarray(v, dtype=np.float64)
    w = np.zeros(len(ci), np.float64)
    st = _load().or_edge_weights(len(rp) - 1, rp, ci, val, v, w)
    if st != OK:
        raise ValueError(f"oracle edge_weights status {st}")
    return w


def greedy_match(rp, ci, w):
    rp, ci, w = _csr(rp, ci, w)
    mate = np.empty(len(rp) - 1, np.int32)
    if _load().or_greedy_match(len(rp) - 1, rp, ci, w, mate) != OK:
        raise MemoryError
    return mate


def suitor_match(rp, ci, w):
    rp, ci, w = _csr(rp, ci, w)
    mate = np.empty(len(rp) - 1, np.int32)
    if _load().or_suitor_match(len(rp) - 1, rp, ci, w, mate) != OK:
        raise MemoryError
    return mate


def aggregate(mate):
    """Returns (agg, n_c, n_pairs, n_singletons)."""
    mate = np.ascontiguousarray(mate, dtype=np.int32)
    agg = np.empty(len(mate), np.int32)
    npairs, nsing = C.c_int(0), C.c_int(0)
    nc = _load().or_aggregate(len(mate), mate, agg, C.byref(npairs), C.byref(nsing))
    return agg, nc, npairs.value, nsing.value


def prolongator(agg, nc, v):
    """Returns (p, v_c): p[i] is the one nonzero of row i of P, v_c = P^T v."""
    agg = np.ascontiguousarray(agg, dtype=np.int32)
    v = np.ascontiguousarray(v, dtype=np.float64)
    p = np.empty(len(agg), np.float64)
    vc = np.empty(nc, np.float64)
    _load().or_prolongator(len(agg), nc, agg, v, p, vc)
    return p, vc


def galerkin(rp, ci, val, agg, nc, p, fp32=False):
    """A_c = P^T A P as a CSR triple, in the canonical summation order (fp32: terms and
    sums in binary32, stored as doubles)."""
    rp, ci, val = _csr(rp, ci, val)
    agg = np.ascontiguousarray(agg, dtype=np.int32)
    p = np.ascontiguousarray(p, dtype=np.float64)
    lib = _load()
    n = len(rp) - 1
    z = lib.or_galerkin_nnz(n, rp, ci, val, nc, agg, p)
    if z < 0:
        raise MemoryError
    rpc = np.empty(nc + 1, np.int32)
    cic = np.empty(z, np.int32)
    valc = np.empty(z, np.float64)
    if lib.or_galerkin(n, rp, ci, val, nc, agg, p, 1 if fp32 else 0, rpc, cic, valc) != OK:
        raise MemoryError
    return rpc, cic, valc


def paper_coarse_max(n: int) -> int:
    """The paper's coarse size for an input of n rows (Sec. 5): floor(40 n^(1/3));
    Hierarchy(coarse_max=-1) uses it."""
    return int(_load().or_paper_coarse_max(int(n)))


class Hierarchy:
    """An oracle hierarchy (levels of A^k, composed P^k, smooth vectors)."""

    def __init__(self, rp, ci, val, v, sweeps=2, coarse_max=40, max_levels=40,
                 pre=1, post=1, coarse_sweeps=20, stall_ratio=0.0, gamma=1, galerkin_fp32_from=0):
        rp, ci, val = _csr(rp, ci, val)
        v = np.ascontiguousarray(v, dtype=np.float64)
        self._lib = _load()
        st = C.c_int(0)
        self._h = self._lib.or_setup(len(rp) - 1, rp, ci, val, v, sweeps, coarse_max,
                                     max_levels, float(stall_ratio), int(galerkin_fp32_from), C.byref(st))
        if not self._h:
            raise ValueError(f"oracle setup failed with status {st.value}")
        self._lib.or_set_cycle(self._h, pre, post, coarse_sweeps)
        self._lib.or_set_gamma(self._h, gamma)

    def close(self):
        if self._h:
            self._lib.or_free(self._h)
            self._h = None

    __del__ = close

    @property
    def nl(self) -> int:
        return self._lib.or_num_levels(self._h)

    def level_n(self, k):
        return self._lib.or_level_n(self._h, k)

    def level_nnz(self, k):
        return self._lib.or_level_nnz(self._h, k)

    def level(self, k):
        """dict with A (rp, ci, val), v, dl1 and, below the coarsest, agg and p."""
        n, z = self.level_n(k), self.level_nnz(k)
        rp = np.empty(n + 1, np.int32)
        ci = np.empty(z, np.int32)
        val = np.empty(z, np.float64)
        v = np.empty(n, np.float64)
        dl1 = np.empty(n, np.float64)
        last = k == self.nl - 1
        agg = None if last else np.empty(n, np.int32)
        p = None if last else np.empty(n, np.float64)
        self._lib.or_level_export(self._h, k, _ptr(rp), _ptr(ci), _ptr(val), _ptr(v),
                                  _ptr(dl1), _ptr(agg), _ptr(p))
        return dict(rp=rp, ci=ci, val=val, v=v, dl1=dl1, agg=agg, p=p, n=n, nnz=z)

    def sweeps(self, k):
        return self._lib.or_level_sweeps(self._h, k)

    def sweep_mate(self, k, s):
        m = np.empty(self._lib.or_sweep_n(self._h, k, s), np.int32)
        self._lib.or_sweep_mate(self._h, k, s, m)
        return m

    def l1_jacobi(self, k, b, x, sweeps):
        x = np.array(x, dtype=np.float64, copy=True)
        self._lib.or_l1_jacobi(self._h, k, np.ascontiguousarray(b, np.float64), x, sweeps)
        return x

    def vcycle(self, r):
        r = np.ascontiguousarray(r, np.float64)
        w = np.empty_like(r)
        self._lib.or_vcycle(self._h, r, w)
        return w

    def pcg(self, b, x0=None, rtol=1e-8, itmax=5000, prec=PREC_AMG):
        """Returns (x, status, iters, relres_recursive, relres_true)."""
        b = np.ascontiguousarray(b, np.float64)
        x = np.zeros_like(b) if x0 is None else np.array(x0, np.float64, copy=True)
        it, rr, rt = C.c_int(0), C.c_double(0), C.c_double(0)
        st = self._lib.or_pcg(self._h, b, x, rtol, itmax, prec, C.byref(it), C.byref(rr),
                              C.byref(rt))
        return x, st, it.value, rr.value, rt.value

    def stats(self):
        """(Vcmplx, cratio) as the paper defines them in Sec. 5.2."""
        a, b = C.c_double(0), C.c_double(0)
        self._lib.or_stats(self._h, C.byref(a), C.byref(b))
        return a.value, b.value
