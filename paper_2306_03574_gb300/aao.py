"""ctypes binding of libaao.so (include/aao.h).  Argument marshalling only.

Vectors are FP64 CUDA tensors (contiguous, time-major (nrhs, n, m)); the
stream defaults to torch's current stream.  aao_solve_host takes host
(numpy or CPU torch) arrays.  Every non-OK status raises AaoError, except that
the solvers return (status, infos) so that AAO_ENOTCONV can be inspected.
"""
from __future__ import annotations

import ctypes
import os
import re
from typing import List, Optional, Tuple

__all__ = [
    "AaoError", "AAO_OK", "AAO_EINVAL", "AAO_EUNSUPPORTED", "AAO_ENOMEM", "AAO_ECUDA",
    "AAO_ENOTCONV", "AAO_EBREAKDOWN", "AAO_ESINGULAR", "AAO_EBUSY", "AAO_EPENDING",
    "AAO_ETIMEOUT", "AAO_PREC_FP64", "AAO_PREC_FP32_IR", "AAO_PREC_F32X2", "lib", "lib_path", "header_functions",
    "aao_create", "aao_destroy", "aao_set_coefficient", "aao_autotune", "aao_workspace_bytes", "aao_build_rhs", "aao_apply_op",
    "aao_apply_prec", "aao_apply_dst", "aao_apply_time", "aao_minres_solve", "aao_solve_host",
    "aao_residual_norm", "aao_residual_norm_noalloc",
    "aao_launch_count", "aao_wait_timeouts", "aao_alu_peak", "aao_status_str", "aao_last_error", "aao_profile_enable", "aao_profile_read",
    "Solver", "aao_serve_create", "aao_serve_submit", "aao_serve_poll", "aao_serve_wait",
    "aao_serve_stats", "aao_serve_destroy",
]

(AAO_OK, AAO_EINVAL, AAO_EUNSUPPORTED, AAO_ENOMEM, AAO_ECUDA, AAO_ENOTCONV, AAO_EBREAKDOWN,
 AAO_ESINGULAR, AAO_EBUSY, AAO_EPENDING, AAO_ETIMEOUT) = range(11)
AAO_PREC_FP64, AAO_PREC_FP32_IR, AAO_PREC_F32X2 = 0, 1, 2

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
lib_path = os.path.join(_HERE, "libaao.so")
HEADER = os.path.join(_ROOT, "include", "aao.h")


class AaoError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {_status_name(status)} {detail}".strip())


class aao_grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("N", ctypes.c_int), ("c2", ctypes.c_double)]


class aao_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("nrhs_max", ctypes.c_int),
                ("variable_coefficient", ctypes.c_int), ("graph", ctypes.c_int),
                ("host_staging", ctypes.c_int), ("reserved", ctypes.c_int * 3)]


class aao_solve_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("status", ctypes.c_int),
                ("relres_true", ctypes.c_double), ("relres_est", ctypes.c_double),
                ("ir_steps", ctypes.c_int), ("reserved", ctypes.c_int)]

    def as_dict(self):
        return dict(iters=self.iters, status=self.status, relres_true=self.relres_true,
                    relres_est=self.relres_est, ir_steps=self.ir_steps)


class aao_request(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("N", ctypes.c_int), ("nt", ctypes.c_int),
                ("tau", ctypes.c_double), ("alpha", ctypes.c_double), ("c2", ctypes.c_double),
                ("rtol", ctypes.c_double), ("maxit", ctypes.c_int),
                ("f", ctypes.c_void_p), ("psi0", ctypes.c_void_p), ("psi1", ctypes.c_void_p),
                ("x", ctypes.c_void_p), ("precision", ctypes.c_int)]


class aao_serve_result(ctypes.Structure):
    _fields_ = [("info", aao_solve_info), ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double),
                ("t_done", ctypes.c_double), ("ticket", ctypes.c_uint64)]


class aao_serve_stats_t(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("submitted", "admitted", "completed", "failed",
                                               "handles_created", "evictions", "pool_bytes",
                                               "peak_pool_bytes", "budget")] + \
               [("in_flight", ctypes.c_int), ("pending", ctypes.c_int)] + \
               [(n, ctypes.c_uint64) for n in ("rounds", "round_problems", "grouped_launches")]


class aao_kernel_stat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_uint64), ("total_ms", ctypes.c_double)]


_lib = None
_P = ctypes.c_void_p


def lib() -> ctypes.CDLL:
    """Load libaao.so (built in-tree by paper_2306_03574_gb300/build.py)."""
    global _lib
    if _lib is None:
        if not os.path.exists(lib_path):
            raise RuntimeError(f"libaao.so not found at {lib_path}: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(lib_path)
        i, d, p, sz = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t
        sig = {
            "aao_create": ([ctypes.POINTER(aao_grid), i, d, d, i, ctypes.POINTER(aao_opts),
                            ctypes.POINTER(ctypes.c_void_p)], i),
            "aao_destroy": ([p], i),
            "aao_set_coefficient": ([p, p, p], i),
            "aao_workspace_bytes": ([p], sz),
            "aao_build_rhs": ([p, p, p, p, p, i, p], i),
            "aao_apply_op": ([p, p, p, i, p], i),
            "aao_apply_prec": ([p, p, p, i, p], i),
            "aao_apply_dst": ([p, p, p, i, p], i),
            "aao_apply_time": ([p, p, p, i, p], i),
            "aao_minres_solve": ([p, p, p, i, i, d, i, ctypes.POINTER(aao_solve_info), p], i),
            "aao_solve_host": ([p, p, p, p, p, i, d, i, ctypes.POINTER(aao_solve_info), p], i),
            "aao_launch_count": ([p], ctypes.c_uint64),
            "aao_wait_timeouts": ([], ctypes.c_uint),
            "aao_alu_peak": ([i, i, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)], i),
            "aao_residual_norm": ([p, p, p, p, i, p], i),
            "aao_residual_norm_noalloc": ([ctypes.POINTER(aao_grid), i, d, p, p, p, i, p], i),
            "aao_noalloc_last_error": ([], ctypes.c_char_p),
            "aao_status_str": ([i], ctypes.c_char_p),
            "aao_profile_enable": ([p, i], i),
            "aao_autotune": ([p, ctypes.c_char_p, ctypes.POINTER(ctypes.c_int)], i),
            "aao_serve_create": ([ctypes.c_size_t, i, ctypes.POINTER(ctypes.c_void_p)], i),
            "aao_serve_submit": ([p, ctypes.POINTER(aao_request), ctypes.POINTER(ctypes.c_uint64)], i),
            "aao_serve_poll": ([p, ctypes.c_uint64, ctypes.POINTER(aao_serve_result)], i),
            "aao_serve_wait": ([p, ctypes.c_uint64, d, ctypes.POINTER(aao_serve_result)], i),
            "aao_serve_stats_get": ([p, ctypes.POINTER(aao_serve_stats_t)], i),
            "aao_serve_destroy": ([p], i),
            "aao_serve_last_error": ([], ctypes.c_char_p),
            "aao_profile_read": ([p, ctypes.POINTER(aao_kernel_stat), i], i),
            "aao_last_error": ([], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def header_functions() -> List[str]:
    """Names of every function declared in include/aao.h."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(aao_[a-z0-9_]+)\s*\(", txt)))


def _status_name(st: int) -> str:
    try:
        return lib().aao_status_str(st).decode()
    except Exception:  # library not loadable: still give a name
        return f"status {st}"


def _check(st: int, where: str):
    if st != AAO_OK:
        raise AaoError(st, where, lib().aao_last_error().decode())


def _dev_ptr(t) -> int:
    if isinstance(t, int):
        return t
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch.Tensor or an int device pointer")
    if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
        raise ValueError("vectors must be contiguous float64 CUDA tensors")
    return t.data_ptr()


def _host_ptr(a):
    import numpy as np
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.is_cuda or a.dtype != torch.float64 or not a.is_contiguous():
                raise ValueError("host buffers must be contiguous float64 CPU tensors")
            return a.data_ptr()
    except ImportError:
        pass
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be C-contiguous float64")
        return a.ctypes.data
    raise TypeError("expected a numpy array or CPU torch tensor")


def _stream(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def aao_profile_enable(h, on: bool = True) -> None:
    _check(lib().aao_profile_enable(h, int(bool(on))), "aao_profile_enable")


def aao_profile_read(h) -> dict:
    """{kernel class: (launches, total_ms)} since the last aao_profile_enable."""
    buf = (aao_kernel_stat * 64)()
    n = lib().aao_profile_read(h, buf, 64)
    if n < 0:
        raise AaoError(AAO_ECUDA, "aao_profile_read", aao_last_error())
    return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms)) for i in range(min(n, 64))}


def aao_status_str(st: int) -> str:
    return lib().aao_status_str(st).decode()


def aao_last_error() -> str:
    return lib().aao_last_error().decode()


def aao_create(dim: int, N: int, nt: int, tau: float, alpha: float, c2: float = 1.0,
               precision: int = AAO_PREC_FP64, nrhs_max: int = 1, scheme: int = 0,
               raw_status: bool = False, variable_coefficient: bool = False, graph: bool = False,
               host_staging: bool = False):
    g = aao_grid(dim, N, c2)
    o = aao_opts(precision, nrhs_max, int(bool(variable_coefficient)), int(bool(graph)),
                 int(bool(host_staging)), (ctypes.c_int * 3)())
    h = ctypes.c_void_p()
    st = lib().aao_create(ctypes.byref(g), nt, tau, alpha, scheme, ctypes.byref(o), ctypes.byref(h))
    if raw_status:
        return st, h.value
    _check(st, "aao_create")
    return h.value


def aao_set_coefficient(h, a_face, stream=None) -> None:
    _check(lib().aao_set_coefficient(h, _dev_ptr(a_face), _stream(stream)), "aao_set_coefficient")


def aao_autotune(h, tune_file=None) -> dict:
    ch = (ctypes.c_int * 2)()
    _check(lib().aao_autotune(h, tune_file.encode() if tune_file else None, ch), "aao_autotune")
    return {"time_variant": ch[0], "dst_variant": ch[1]}


def aao_destroy(h) -> None:
    _check(lib().aao_destroy(h), "aao_destroy")


def aao_workspace_bytes(h) -> int:
    return int(lib().aao_workspace_bytes(h))


def aao_launch_count(h) -> int:
    return int(lib().aao_launch_count(h))


def aao_wait_timeouts() -> int:
    return int(lib().aao_wait_timeouts())


def aao_alu_peak(precision: int, iters: int = 1 << 16):
    """(TFLOP/s, ms) of the FMA-loop probe in FP64 (AAO_PREC_FP64) or FP32 (AAO_PREC_FP32_IR)."""
    tf, ms = ctypes.c_double(), ctypes.c_double()
    _check(lib().aao_alu_peak(precision, iters, ctypes.byref(tf), ctypes.byref(ms)), "aao_alu_peak")
    return tf.value, ms.value


def aao_build_rhs(h, f, psi0, psi1, b, nrhs: int = 1, stream=None) -> None:
    _check(lib().aao_build_rhs(h, _dev_ptr(f), _dev_ptr(psi0), _dev_ptr(psi1), _dev_ptr(b), nrhs,
                               _stream(stream)), "aao_build_rhs")


def aao_apply_op(h, x, y, nrhs: int = 1, stream=None) -> None:
    _check(lib().aao_apply_op(h, _dev_ptr(x), _dev_ptr(y), nrhs, _stream(stream)), "aao_apply_op")


def aao_apply_prec(h, r, z, nrhs: int = 1, stream=None) -> None:
    _check(lib().aao_apply_prec(h, _dev_ptr(r), _dev_ptr(z), nrhs, _stream(stream)), "aao_apply_prec")


def aao_apply_dst(h, x, y, nrhs: int = 1, stream=None) -> None:
    _check(lib().aao_apply_dst(h, _dev_ptr(x), _dev_ptr(y), nrhs, _stream(stream)), "aao_apply_dst")


def aao_apply_time(h, x, y, nrhs: int = 1, stream=None) -> None:
    _check(lib().aao_apply_time(h, _dev_ptr(x), _dev_ptr(y), nrhs, _stream(stream)), "aao_apply_time")


def aao_minres_solve(h, b, x, nrhs: int = 1, rtol: float = 1e-8, maxit: int = 100,
                     use_x0: bool = False, stream=None) -> Tuple[int, list]:
    infos = (aao_solve_info * nrhs)()
    st = lib().aao_minres_solve(h, _dev_ptr(b), _dev_ptr(x), int(bool(use_x0)), nrhs, rtol, maxit,
                                infos, _stream(stream))
    if st not in (AAO_OK, AAO_ENOTCONV, AAO_EBREAKDOWN):
        _check(st, "aao_minres_solve")
    return st, [i.as_dict() for i in infos]


def aao_residual_norm(h, b, x, relres, nrhs: int = 1, stream=None) -> None:
    _check(lib().aao_residual_norm(h, _dev_ptr(b), _dev_ptr(x), _dev_ptr(relres), nrhs, _stream(stream)),
           "aao_residual_norm")


def aao_residual_norm_noalloc(dim, N, nt, tau, b, x, relres, nrhs: int = 1, c2: float = 1.0,
                              stream=None, raw_status: bool = False):
    """Allocation-free residual norm (no handle); see include/aao.h."""
    g = aao_grid(dim, N, c2)
    st = lib().aao_residual_norm_noalloc(ctypes.byref(g), nt, tau, _dev_ptr(b), _dev_ptr(x),
                                         _dev_ptr(relres), nrhs, _stream(stream))
    if raw_status:
        return st
    if st != AAO_OK:
        raise AaoError(st, "aao_residual_norm_noalloc", lib().aao_noalloc_last_error().decode())
    return st


def aao_solve_host(h, f, psi0, psi1, u, nrhs: int = 1, rtol: float = 1e-8, maxit: int = 100,
                   stream=None) -> Tuple[int, list]:
    infos = (aao_solve_info * nrhs)()
    st = lib().aao_solve_host(h, _host_ptr(f), _host_ptr(psi0), _host_ptr(psi1), _host_ptr(u),
                              nrhs, rtol, maxit, infos, _stream(stream))
    if st not in (AAO_OK, AAO_ENOTCONV, AAO_EBREAKDOWN):
        _check(st, "aao_solve_host")
    return st, [i.as_dict() for i in infos]


def _serve_result(r):
    d = r.info.as_dict()
    d.update(t_submit=r.t_submit, t_start=r.t_start, t_done=r.t_done, ticket=r.ticket)
    return d


def aao_serve_create(hbm_budget_bytes: int, max_slots: int, raw_status: bool = False):
    s = ctypes.c_void_p()
    st = lib().aao_serve_create(int(hbm_budget_bytes), int(max_slots), ctypes.byref(s))
    if raw_status:
        return st, s.value
    if st != AAO_OK:
        raise AaoError(st, "aao_serve_create", lib().aao_serve_last_error().decode())
    return s.value


def aao_serve_submit(srv, dim, N, nt, tau, alpha, c2, rtol, maxit, f, psi0, psi1, x,
                     precision: int = AAO_PREC_FP64) -> int:
    r = aao_request(dim, N, nt, tau, alpha, c2, rtol, maxit, _dev_ptr(f), _dev_ptr(psi0), _dev_ptr(psi1),
                    _dev_ptr(x), precision)
    t = ctypes.c_uint64()
    st = lib().aao_serve_submit(srv, ctypes.byref(r), ctypes.byref(t))
    if st != AAO_OK:
        raise AaoError(st, "aao_serve_submit", lib().aao_serve_last_error().decode())
    return int(t.value)


def aao_serve_poll(srv, ticket: int):
    """(status, result dict or None); status AAO_EPENDING while running."""
    r = aao_serve_result()
    st = lib().aao_serve_poll(srv, ticket, ctypes.byref(r))
    if st == AAO_EPENDING:
        return st, None
    if st == AAO_EINVAL and r.ticket == 0:
        return st, None
    return st, _serve_result(r)


def aao_serve_wait(srv, ticket: int, timeout_s: float):
    r = aao_serve_result()
    st = lib().aao_serve_wait(srv, ticket, float(timeout_s), ctypes.byref(r))
    if st in (AAO_ETIMEOUT, AAO_EPENDING) or (st == AAO_EINVAL and r.ticket == 0):
        return st, None
    return st, _serve_result(r)


def aao_serve_stats(srv) -> dict:
    s = aao_serve_stats_t()
    _check(lib().aao_serve_stats_get(srv, ctypes.byref(s)), "aao_serve_stats_get")
    return {n: getattr(s, n) for n, _ in s._fields_}


def aao_serve_destroy(srv) -> None:
    _check(lib().aao_serve_destroy(srv), "aao_serve_destroy")


class Solver:
    """Owns one handle: `Solver(dim, N, nt, tau, alpha, ...)`; methods map 1:1 to the C calls."""

    def __init__(self, dim, N, nt, tau, alpha, c2=1.0, precision=AAO_PREC_FP64, nrhs_max=1,
                 variable_coefficient=False, graph=False, host_staging=False):
        self.dim, self.N, self.nt, self.tau, self.alpha, self.c2 = dim, N, nt, tau, alpha, c2
        self.m = N ** dim
        self.nrhs_max = nrhs_max
        self.h = aao_create(dim, N, nt, tau, alpha, c2, precision, nrhs_max,
                            variable_coefficient=variable_coefficient, graph=graph,
                            host_staging=host_staging)

    def autotune(self, tune_file=None) -> dict:
        return aao_autotune(self.h, tune_file)

    def set_coefficient(self, a_face, stream=None):
        aao_set_coefficient(self.h, a_face, stream)

    def close(self):
        if self.h:
            aao_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _nrhs(self, t):
        return t.numel() // (self.nt * self.m)

    def apply_op(self, x, y, stream=None):
        aao_apply_op(self.h, x, y, self._nrhs(x), stream)

    def apply_prec(self, r, z, stream=None):
        aao_apply_prec(self.h, r, z, self._nrhs(r), stream)

    def apply_dst(self, x, y, stream=None):
        aao_apply_dst(self.h, x, y, self._nrhs(x), stream)

    def apply_time(self, x, y, stream=None):
        aao_apply_time(self.h, x, y, self._nrhs(x), stream)

    def build_rhs(self, f, psi0, psi1, b, stream=None):
        aao_build_rhs(self.h, f, psi0, psi1, b, self._nrhs(f), stream)

    def residual_norm(self, b, x, relres, stream=None):
        aao_residual_norm(self.h, b, x, relres, self._nrhs(b), stream)

    def solve(self, b, x, rtol=1e-8, maxit=100, use_x0=False, stream=None):
        return aao_minres_solve(self.h, b, x, self._nrhs(b), rtol, maxit, use_x0, stream)

    def solve_host(self, f, psi0, psi1, u, rtol=1e-8, maxit=100, stream=None):
        nel = f.numel() if hasattr(f, "numel") else f.size
        return aao_solve_host(self.h, f, psi0, psi1, u, nel // (self.nt * self.m), rtol, maxit, stream)

    @property
    def workspace_bytes(self):
        return aao_workspace_bytes(self.h)

    @property
    def launches(self):
        return aao_launch_count(self.h)
