"""Python binding of the C ABI in ``include/cwm_amg.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls and passes torch CUDA
tensors' ``data_ptr()`` and the current CUDA stream.  All computation happens in the
CUDA library ``lib/libcwmamg.so``; if that library is missing this module raises -- there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libcwmamg.so")

AMG_OK, AMG_ERR_INVALID_ARG, AMG_ERR_NOT_SPD, AMG_ERR_CUDA, AMG_ERR_OOM = 0, 1, 2, 3, 4
AMG_ERR_TIMEOUT, AMG_ERR_BREAKDOWN, AMG_ERR_NOT_CONVERGED, AMG_ERR_UNSUPPORTED = 5, 6, 7, 8

# Every symbol include/cwm_amg.h declares.
EXPORTS = (
    "amg_default_params", "amg_setup", "amg_vcycle", "amg_pcg_solve", "amg_free", "amg_stats",
    "amg_num_levels", "amg_level_info", "amg_level_export", "amg_sweep_mate", "cwm_edge_weights",
    "cwm_suitor_match", "cwm_aggregate", "cwm_galerkin", "amg_status_string", "amg_last_error",
    "amg_trace_enable", "amg_trace_reset", "amg_trace_count", "amg_trace_get", "amg_launch_count",
    "cwm_suitor_match_noalloc", "cwm_pattern_outer", "cwm_fp64_rates", "cwm_div_check", "cwm_copy",
)


class AmgParams(C.Structure):
    _fields_ = [
        ("sweeps_per_level", C.c_int),
        ("coarse_max", C.c_int),
        ("max_levels", C.c_int),
        ("pre_sweeps", C.c_int),
        ("post_sweeps", C.c_int),
        ("coarse_sweeps", C.c_int),
        ("vcycle_fp32", C.c_int),
        ("check_input", C.c_int),
        ("keep_sweeps", C.c_int),
        ("loop_cap", C.c_int64),
        ("trace", C.c_int),
        ("trace_filter", C.c_char * 32),
        ("tail_rows", C.c_int),
        ("stall_ratio", C.c_double),
        ("gamma", C.c_int),
        ("galerkin_fp32_from", C.c_int),
        ("coupled_post", C.c_int),
        ("block3", C.c_int),
        ("sliced", C.c_int),
    ]


class AmgInfo(C.Structure):
    _fields_ = [
        ("iters", C.c_int),
        ("rel_res", C.c_double),
        ("rel_res_true", C.c_double),
        ("nl", C.c_int),
        ("vcmplx", C.c_double),
        ("cratio", C.c_double),
        ("t_setup_ms", C.c_double),
        ("t_solve_ms", C.c_double),
    ]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class AmgTraceEntry(C.Structure):
    _fields_ = [("name", C.c_char * 48), ("launches", C.c_int64), ("total_ms", C.c_double), ("bytes", C.c_double)]


class AmgError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {status_name(status)}: {message}")
        self.status = status


_lib = None
_lock = threading.Lock()


def load(path: str | None = None):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"{p} is missing: build it with paper_1810_04221_gb300.build.build()")
        lib = C.CDLL(p)
        vp, i, i64, d = C.c_void_p, C.c_int, C.c_int64, C.c_double
        ip = C.POINTER(C.c_int)
        sig = {
            "amg_default_params": (None, [C.POINTER(AmgParams)]),
            "amg_setup": (i, [i, i64, vp, vp, vp, vp, C.POINTER(AmgParams), vp, C.POINTER(vp)]),
            "amg_vcycle": (i, [vp, vp, vp, vp]),
            "amg_pcg_solve": (i, [vp, vp, vp, d, i, vp, C.POINTER(AmgInfo)]),
            "amg_free": (None, [vp]),
            "amg_stats": (i, [vp, C.POINTER(AmgInfo)]),
            "amg_num_levels": (i, [vp]),
            "amg_level_info": (i, [vp, i, ip, C.POINTER(i64), ip]),
            "amg_level_export": (i, [vp, i, vp, vp, vp, vp, vp, vp, vp, vp]),
            "amg_sweep_mate": (i, [vp, i, i, vp, ip, vp]),
            "cwm_edge_weights": (i, [i, i64, vp, vp, vp, vp, vp, vp]),
            "cwm_suitor_match": (i, [i, i64, vp, vp, vp, vp, vp]),
            "cwm_suitor_match_noalloc": (i, [i, i64, vp, vp, vp, vp, vp]),
            "cwm_pattern_outer": (i, [i, i64, vp, vp, vp, vp, d, vp, vp]),
            "cwm_aggregate": (i, [i, vp, vp, vp, vp, vp, ip, ip, vp]),
            "cwm_galerkin": (i, [i, vp, vp, vp, i, vp, vp, vp, vp, vp, i64, C.POINTER(i64), i, vp]),
            "amg_trace_enable": (i, [vp, i, C.c_char_p]),
            "amg_trace_reset": (i, [vp]),
            "amg_trace_count": (i, [vp]),
            "amg_trace_get": (i, [vp, i, C.POINTER(AmgTraceEntry)]),
            "amg_launch_count": (i64, []),
            "cwm_fp64_rates": (i, [C.POINTER(d), C.POINTER(d), vp]),
            "cwm_div_check": (i, [C.c_longlong, C.c_ulonglong, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong), vp]),
            "cwm_copy": (i, [vp, vp, i64, vp]),
            "amg_status_string": (C.c_char_p, [i]),
            "amg_last_error": (C.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def status_name(status: int) -> str:
    try:
        return load().amg_status_string(status).decode()
    except Exception:  # noqa: BLE001 - only for messages
        return str(status)


def _check(status: int, where: str, allow=(AMG_OK,)):
    if status not in allow:
        raise AmgError(status, where, load().amg_last_error().decode())
    return status


def _stream(stream):
    if stream is None:
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def _dev(t: torch.Tensor | None, dtype: torch.dtype, name: str, numel: int | None = None):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {dtype} tensor (got {t.dtype})")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{name} needs at least {numel} elements (got {t.numel()})")
    return C.c_void_p(t.data_ptr())


def _buf(t: torch.Tensor | None, dtype: torch.dtype, name: str, numel: int | None = None):
    """A device or host (pinned or pageable) tensor for the calls that accept either."""
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {dtype} tensor (got {t.dtype})")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{name} needs at least {numel} elements (got {t.numel()})")
    return C.c_void_p(t.data_ptr())


def amg_default_params(**overrides) -> AmgParams:
    p = AmgParams()
    load().amg_default_params(C.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v.encode() if isinstance(v, str) else v)
    return p


class AmgHandle:
    """Owns an amg_handle; freed by amg_free (or when garbage-collected)."""

    def __init__(self, ptr: int, n: int, nnz: int):
        self.ptr = ptr
        self.n = n
        self.nnz = nnz

    def free(self):
        if self.ptr:
            load().amg_free(C.c_void_p(self.ptr))
            self.ptr = None

    __del__ = free


def amg_setup(row_ptr, col, val, v, params: AmgParams | None = None, stream=None) -> AmgHandle:
    n = row_ptr.numel() - 1
    nnz = col.numel()
    out = C.c_void_p()
    st = load().amg_setup(n, nnz, _buf(row_ptr, torch.int32, "row_ptr"), _buf(col, torch.int32, "col"),
                          _buf(val, torch.float64, "val", nnz), _buf(v, torch.float64, "v", n),
                          C.byref(params) if params is not None else None, _stream(stream), C.byref(out))
    _check(st, "amg_setup")
    return AmgHandle(out.value, n, nnz)


def amg_free(h: AmgHandle):
    h.free()


def amg_vcycle(h: AmgHandle, r, w, stream=None):
    _check(load().amg_vcycle(C.c_void_p(h.ptr), _dev(r, torch.float64, "r", h.n), _dev(w, torch.float64, "w", h.n),
                             _stream(stream)), "amg_vcycle")
    return w


def amg_pcg_solve(h: AmgHandle, b, x, rtol: float = 1e-8, itmax: int = 5000, stream=None):
    """Returns (status, info dict); NOT_CONVERGED is returned, other errors raise."""
    info = AmgInfo()
    st = load().amg_pcg_solve(C.c_void_p(h.ptr), _buf(b, torch.float64, "b", h.n), _buf(x, torch.float64, "x", h.n),
                              float(rtol), int(itmax), _stream(stream), C.byref(info))
    _check(st, "amg_pcg_solve", allow=(AMG_OK, AMG_ERR_NOT_CONVERGED))
    return st, info.as_dict()


def amg_stats(h: AmgHandle) -> dict:
    info = AmgInfo()
    _check(load().amg_stats(C.c_void_p(h.ptr), C.byref(info)), "amg_stats")
    return info.as_dict()


def amg_num_levels(h: AmgHandle) -> int:
    return load().amg_num_levels(C.c_void_p(h.ptr))


def amg_level_info(h: AmgHandle, level: int):
    n, nnz, ns = C.c_int(0), C.c_int64(0), C.c_int(0)
    _check(load().amg_level_info(C.c_void_p(h.ptr), level, C.byref(n), C.byref(nnz), C.byref(ns)), "amg_level_info")
    return n.value, nnz.value, ns.value


def amg_level_export(h: AmgHandle, level: int, stream=None) -> dict:
    n, nnz, ns = amg_level_info(h, level)
    dev = torch.device("cuda")
    out = dict(rp=torch.empty(n + 1, dtype=torch.int32, device=dev), ci=torch.empty(nnz, dtype=torch.int32, device=dev),
               val=torch.empty(nnz, dtype=torch.float64, device=dev), v=torch.empty(n, dtype=torch.float64, device=dev),
               dl1=torch.empty(n, dtype=torch.float64, device=dev))
    last = level == amg_num_levels(h) - 1
    agg = None if last else torch.empty(n, dtype=torch.int32, device=dev)
    p = None if last else torch.empty(n, dtype=torch.float64, device=dev)
    _check(load().amg_level_export(C.c_void_p(h.ptr), level, _dev(out["rp"], torch.int32, "rp"),
                                   _dev(out["ci"], torch.int32, "ci"), _dev(out["val"], torch.float64, "val"),
                                   _dev(out["v"], torch.float64, "v"), _dev(out["dl1"], torch.float64, "dl1"),
                                   _dev(agg, torch.int32, "agg"), _dev(p, torch.float64, "p"), _stream(stream)),
           "amg_level_export")
    out.update(agg=agg, p=p, n=n, nnz=nnz, nsweeps=ns)
    return out


def amg_sweep_mate(h: AmgHandle, level: int, sweep: int, stream=None):
    n = C.c_int(0)
    lib = load()
    _check(lib.amg_sweep_mate(C.c_void_p(h.ptr), level, sweep, None, C.byref(n), _stream(stream)), "amg_sweep_mate")
    mate = torch.empty(n.value, dtype=torch.int32, device="cuda")
    _check(lib.amg_sweep_mate(C.c_void_p(h.ptr), level, sweep, _dev(mate, torch.int32, "mate"), C.byref(n),
                              _stream(stream)), "amg_sweep_mate")
    return mate


def cwm_edge_weights(row_ptr, col, val, v, w=None, stream=None):
    n, nnz = row_ptr.numel() - 1, col.numel()
    if w is None:
        w = torch.empty(nnz, dtype=torch.float64, device=val.device)
    _check(load().cwm_edge_weights(n, nnz, _dev(row_ptr, torch.int32, "row_ptr"), _dev(col, torch.int32, "col"),
                                   _dev(val, torch.float64, "val", nnz), _dev(v, torch.float64, "v", n),
                                   _dev(w, torch.float64, "w", nnz), _stream(stream)), "cwm_edge_weights")
    return w


def cwm_suitor_match(row_ptr, col, w, mate=None, stream=None):
    n, nnz = row_ptr.numel() - 1, col.numel()
    if mate is None:
        mate = torch.empty(n, dtype=torch.int32, device=w.device)
    _check(load().cwm_suitor_match(n, nnz, _dev(row_ptr, torch.int32, "row_ptr"), _dev(col, torch.int32, "col"),
                                   _dev(w, torch.float64, "w", nnz), _dev(mate, torch.int32, "mate", n),
                                   _stream(stream)), "cwm_suitor_match")
    return mate


def cwm_suitor_match_noalloc(row_ptr, col, w, mate, stream=None):
    """cwm_suitor_match without any device allocation: `mate` must be given (n int32)."""
    n, nnz = row_ptr.numel() - 1, col.numel()
    _check(load().cwm_suitor_match_noalloc(n, nnz, _dev(row_ptr, torch.int32, "row_ptr"), _dev(col, torch.int32, "col"),
                                           _dev(w, torch.float64, "w", nnz), _dev(mate, torch.int32, "mate", n),
                                           _stream(stream)), "cwm_suitor_match_noalloc")
    return mate


def cwm_aggregate(mate, v, stream=None):
    """Returns (agg, p, v_c, n_c, n_pairs); v_c has n_c entries."""
    n = mate.numel()
    dev = mate.device
    agg = torch.empty(n, dtype=torch.int32, device=dev)
    p = torch.empty(n, dtype=torch.float64, device=dev)
    vc = torch.empty(max(n, 1), dtype=torch.float64, device=dev)
    nc, npairs = C.c_int(0), C.c_int(0)
    _check(load().cwm_aggregate(n, _dev(mate, torch.int32, "mate"), _dev(v, torch.float64, "v", n),
                                _dev(agg, torch.int32, "agg"), _dev(p, torch.float64, "p"), _dev(vc, torch.float64, "vc"),
                                C.byref(nc), C.byref(npairs), _stream(stream)), "cwm_aggregate")
    return agg, p, vc[: nc.value], nc.value, npairs.value


def cwm_galerkin(row_ptr, col, val, nc: int, agg, p, fp32: bool = False, stream=None):
    """Returns (rpc, colc, valc) of A_c = P^T A P for a pairwise P (fp32: the binary32
    product, values stored as doubles)."""
    n, nnz = row_ptr.numel() - 1, col.numel()
    dev = val.device
    rpc = torch.empty(nc + 1, dtype=torch.int32, device=dev)
    cap = max(nnz, 1)
    colc = torch.empty(cap, dtype=torch.int32, device=dev)
    valc = torch.empty(cap, dtype=torch.float64, device=dev)
    nnzc = C.c_int64(0)
    _check(load().cwm_galerkin(n, _dev(row_ptr, torch.int32, "row_ptr"), _dev(col, torch.int32, "col"),
                               _dev(val, torch.float64, "val", nnz), nc, _dev(agg, torch.int32, "agg", n),
                               _dev(p, torch.float64, "p", n), _dev(rpc, torch.int32, "rpc"),
                               _dev(colc, torch.int32, "colc"), _dev(valc, torch.float64, "valc"), cap,
                               C.byref(nnzc), 1 if fp32 else 0, _stream(stream)), "cwm_galerkin")
    z = nnzc.value
    return rpc, colc[:z], valc[:z]


def amg_trace_enable(h: AmgHandle, on: bool = True, filter: str | None = None):
    _check(load().amg_trace_enable(C.c_void_p(h.ptr), 1 if on else 0, filter.encode() if filter else None),
           "amg_trace_enable")


def amg_trace_reset(h: AmgHandle):
    _check(load().amg_trace_reset(C.c_void_p(h.ptr)), "amg_trace_reset")


def amg_trace_count(h: AmgHandle) -> int:
    return load().amg_trace_count(C.c_void_p(h.ptr))


def amg_trace_get(h: AmgHandle, i: int) -> dict:
    e = AmgTraceEntry()
    _check(load().amg_trace_get(C.c_void_p(h.ptr), i, C.byref(e)), "amg_trace_get")
    return {"name": e.name.decode(), "launches": e.launches, "total_ms": e.total_ms, "bytes": e.bytes}


def amg_trace(h: AmgHandle) -> list[dict]:
    """Every trace entry (waits for the recorded events)."""
    return [amg_trace_get(h, i) for i in range(amg_trace_count(h))]


def amg_launch_count() -> int:
    return int(load().amg_launch_count())


def cwm_pattern_outer(row_ptr, col, lam, x, alpha: float = 1.0, out=None, stream=None):
    """out[k] = alpha * lam[i] * x[j] on the stored pattern (i, j) of A."""
    n, nnz = row_ptr.numel() - 1, col.numel()
    if out is None:
        out = torch.empty(nnz, dtype=torch.float64, device=x.device)
    _check(load().cwm_pattern_outer(n, nnz, _dev(row_ptr, torch.int32, "row_ptr"), _dev(col, torch.int32, "col"),
                                    _dev(lam, torch.float64, "lam", n), _dev(x, torch.float64, "x", n), float(alpha),
                                    _dev(out, torch.float64, "out", nnz), _stream(stream)), "cwm_pattern_outer")
    return out


def cwm_fp64_rates(stream=None) -> tuple[float, float]:
    """(fused multiply-adds per second, correctly rounded divisions per second) in FP64."""
    f, d = C.c_double(), C.c_double()
    _check(load().cwm_fp64_rates(C.byref(f), C.byref(d), _stream(stream)), "cwm_fp64_rates")
    return f.value, d.value


def cwm_copy(dst: torch.Tensor, src: torch.Tensor, stream=None):
    """dst <- src (same byte size; at least one of them on the device), as the library moves
    host arrays."""
    nb = src.numel() * src.element_size()
    if dst.numel() * dst.element_size() < nb or not (dst.is_contiguous() and src.is_contiguous()):
        raise ValueError("cwm_copy: dst must be contiguous and at least as large as src")
    _check(load().cwm_copy(C.c_void_p(dst.data_ptr()), C.c_void_p(src.data_ptr()), nb, _stream(stream)), "cwm_copy")
    return dst


def cwm_div_check(n: int, seed: int, stream=None) -> tuple[int, int]:
    """(mismatching pairs, first mismatching index or -1) of the edge weights' integer-pipe
    quotient against the hardware division over n generated operand pairs."""
    mm, first = C.c_longlong(), C.c_longlong()
    _check(load().cwm_div_check(int(n), int(seed) & (2**64 - 1), C.byref(mm), C.byref(first), _stream(stream)),
           "cwm_div_check")
    return mm.value, first.value
