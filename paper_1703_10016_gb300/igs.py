"""Thin Python binding of the C ABI in include/igs.h (ctypes).

Each function here has the name of the C entry point it calls and does only
argument marshalling (numpy / torch buffers to pointers, return-code to
exception).  Every step of the computation runs in libigs.so; there is no
Python or CPU fallback: if the library is missing the import fails.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libigs.so")

IGS_OK = 0
IGS_E_INVALID_ARG = -1
IGS_E_NO_MEMORY = -2
IGS_E_CUDA = -3
IGS_E_NOT_SPD = -4
IGS_E_NOT_CONVERGED = -5
IGS_E_TIMEOUT = -6
IGS_E_ADMISSION_REFUSED = -7
IGS_E_STATE = -8
IGS_E_SINGULAR = -9
IGS_FP64, IGS_MIXED = 0, 1
IGS_MEM_HOST, IGS_MEM_DEVICE = 0, 1
IGS_F64, IGS_F32 = 0, 1

EXPORTED = [
    "igs_create", "igs_destroy", "igs_last_error", "igs_create_geometry", "igs_destroy_geometry",
    "igs_create_problem", "igs_destroy_problem", "igs_set_geometry", "igs_problem_info", "igs_problem_timing",
    "igs_build_weighted_rules", "igs_assemble", "igs_rhs_points", "igs_build_rhs", "igs_build_rhs_noalloc",
    "igs_solve", "igs_solve_data", "igs_eval_potential", "igs_collocation",
    "igs_get_rules", "igs_get_node_geometry",
    "igs_get_matrix", "igs_batch_create", "igs_batch_destroy", "igs_batch_assemble", "igs_batch_tune", "igs_batch_set_config",
    "igs_batch_get_config",
    "igs_server_create", "igs_server_submit", "igs_server_wait", "igs_server_result", "igs_server_drain",
    "igs_server_destroy", "igs_selftest_wait", "igs_measure_peak",
]
IGS_REQ_QUEUED, IGS_REQ_RUNNING, IGS_REQ_DONE, IGS_REQ_FAILED = 0, 1, 2, 3
IGS_REUSE_NONE, IGS_REUSE_RULES, IGS_REUSE_FACTOR = 0, 1, 2
IGS_ORDER_NATURAL, IGS_ORDER_INTERLEAVED, IGS_ORDER_LARGEST_FIRST = 0, 1, 2
IGS_PEAK_FP32_FMA, IGS_PEAK_MUFU_LG2, IGS_PEAK_MUFU_RCP, IGS_PEAK_FP64_FMA = 0, 1, 2, 3


class IgsError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where} failed ({code}): {msg}")
        self.code = code


class igs_info(C.Structure):
    _fields_ = [("n", C.c_int32), ("degree", C.c_int32), ("n_elems", C.c_int32), ("n_ref", C.c_int32),
                ("n_quad", C.c_int32), ("n_exact", C.c_int32), ("n_rhs_pts", C.c_int32), ("closed", C.c_int32),
                ("precision", C.c_int32), ("rules_ready", C.c_int32), ("assembled", C.c_int32),
                ("factored", C.c_int32), ("rhs_slots", C.c_int32), ("device_bytes", C.c_int64)]


class igs_timing(C.Structure):
    _fields_ = [("rules_ms", C.c_float), ("geometry_ms", C.c_float), ("assemble_ms", C.c_float),
                ("rhs_ms", C.c_float), ("factor_ms", C.c_float), ("solve_ms", C.c_float),
                ("ir_iterations", C.c_int32), ("kernel_launches", C.c_int32)]


class igs_batch_config(C.Structure):
    _fields_ = [("tile", C.c_int32), ("order", C.c_int32), ("ctas_per_sm", C.c_int32), ("ms", C.c_float)]


DATA_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.POINTER(C.c_double), C.c_int64, C.c_int, C.POINTER(C.c_double))


class igs_request(C.Structure):
    _fields_ = [("geom_degree", C.c_int32), ("n_knots", C.c_int32), ("knots", C.c_void_p), ("n_ctrl", C.c_int32),
                ("ctrl_xy", C.c_void_p), ("weights", C.c_void_p), ("closed", C.c_int32), ("degree", C.c_int32),
                ("n_elems", C.c_int32), ("n_ref", C.c_int32), ("precision", C.c_int32), ("nrhs", C.c_int32),
                ("data", DATA_FN), ("user", C.c_void_p)]


class igs_server_opts(C.Structure):
    _fields_ = [("slots", C.c_int32), ("mem_budget", C.c_int64), ("cache_budget", C.c_int64)]


class igs_request_stats(C.Structure):
    _fields_ = [("status", C.c_int32), ("error", C.c_int32), ("n", C.c_int32), ("nrhs", C.c_int32),
                ("ir_iterations", C.c_int32), ("slot", C.c_int32), ("device_bytes", C.c_int64),
                ("queue_ms", C.c_double), ("run_ms", C.c_double), ("latency_ms", C.c_double),
                ("reuse", C.c_int32), ("reserved", C.c_int32)]


def _load() -> C.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_1703_10016_gb300.build.build_library()")
    lib = C.CDLL(LIB_PATH)
    vp, i32, i64, dp = C.c_void_p, C.c_int, C.c_int64, C.POINTER(C.c_double)
    lib.igs_last_error.restype = C.c_char_p
    sigs = {
        "igs_create": [C.POINTER(vp), i32, vp],
        "igs_destroy": [vp],
        "igs_create_geometry": [vp, C.POINTER(vp), i32, vp, i32, vp, vp, i32, i32],
        "igs_destroy_geometry": [vp],
        "igs_create_problem": [vp, C.POINTER(vp), i32, i32, i32, i32],
        "igs_destroy_problem": [vp],
        "igs_set_geometry": [vp, vp],
        "igs_problem_info": [vp, C.POINTER(igs_info)],
        "igs_problem_timing": [vp, C.POINTER(igs_timing)],
        "igs_build_weighted_rules": [vp],
        "igs_assemble": [vp, vp, i64, i32, i32],
        "igs_rhs_points": [vp, vp, i64, C.POINTER(i64)],
        "igs_build_rhs": [vp, vp, i32, vp, i32],
        "igs_build_rhs_noalloc": [vp, vp, i32, vp],
        "igs_solve": [vp, vp, i32, vp, vp, i32],
        "igs_solve_data": [vp, vp, i32, vp, vp, i32],
        "igs_eval_potential": [vp, vp, vp, i32, vp, i64, vp, i32],
        "igs_collocation": [vp, vp, i32, vp, vp, vp, i32],
        "igs_get_rules": [vp, vp, vp, vp, vp],
        "igs_get_node_geometry": [vp, vp, vp],
        "igs_get_matrix": [vp, vp, i64, i32, i32],
        "igs_batch_create": [vp, C.POINTER(vp), C.POINTER(vp), i32],
        "igs_batch_destroy": [vp],
        "igs_batch_assemble": [vp, C.POINTER(C.c_float)],
        "igs_batch_tune": [vp, C.POINTER(igs_batch_config), i32],
        "igs_batch_set_config": [vp, C.POINTER(igs_batch_config)],
        "igs_batch_get_config": [vp, C.POINTER(igs_batch_config)],
        "igs_server_create": [i32, C.POINTER(igs_server_opts), C.POINTER(vp)],
        "igs_server_submit": [vp, C.POINTER(igs_request), C.POINTER(i64)],
        "igs_server_wait": [vp, i64, i32, C.POINTER(igs_request_stats)],
        "igs_server_result": [vp, i64, vp, vp, C.POINTER(igs_request_stats)],
        "igs_server_drain": [vp, i32],
        "igs_server_destroy": [vp],
        "igs_selftest_wait": [vp, C.c_double, C.POINTER(i32)],
        "igs_measure_peak": [vp, i32, C.POINTER(C.c_double), C.POINTER(C.c_double)],
    }
    for name, args in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = C.c_int
    return lib


_lib = _load()


def _check(rc: int, where: str) -> None:
    if rc != IGS_OK:
        raise IgsError(rc, where, _lib.igs_last_error().decode())


def _ptr(a) -> C.c_void_p | None:
    """Raw pointer of a numpy array (host) or torch tensor (host or device)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return C.c_void_p(a.ctypes.data)
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(a.data_ptr())
    raise TypeError(f"unsupported buffer type {type(a)}")


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------- entry points
def igs_create(device: int = 0, stream: int | None = None) -> C.c_void_p:
    h = C.c_void_p()
    _check(_lib.igs_create(C.byref(h), device, C.c_void_p(stream) if stream else None), "igs_create")
    return h


def igs_destroy(ctx) -> None:
    _check(_lib.igs_destroy(ctx), "igs_destroy")


def igs_last_error() -> str:
    return _lib.igs_last_error().decode()


def igs_create_geometry(ctx, degree: int, knots, ctrl_xy, weights, closed: bool) -> C.c_void_p:
    knots, ctrl = _f64(knots), _f64(ctrl_xy).reshape(-1, 2)
    w = None if weights is None else _f64(weights)
    h = C.c_void_p()
    _check(_lib.igs_create_geometry(ctx, C.byref(h), int(degree), _ptr(knots), len(knots), _ptr(ctrl),
                                    _ptr(w), len(ctrl), int(bool(closed))), "igs_create_geometry")
    return h


def igs_destroy_geometry(geom) -> None:
    _check(_lib.igs_destroy_geometry(geom), "igs_destroy_geometry")


def igs_create_problem(geom, degree: int, n_elems: int, n_ref: int, precision: int) -> C.c_void_p:
    h = C.c_void_p()
    _check(_lib.igs_create_problem(geom, C.byref(h), int(degree), int(n_elems), int(n_ref), int(precision)),
           "igs_create_problem")
    return h


def igs_destroy_problem(prob) -> None:
    _check(_lib.igs_destroy_problem(prob), "igs_destroy_problem")


def igs_set_geometry(prob, geom) -> None:
    _check(_lib.igs_set_geometry(prob, geom), "igs_set_geometry")


def igs_problem_info(prob) -> igs_info:
    out = igs_info()
    _check(_lib.igs_problem_info(prob, C.byref(out)), "igs_problem_info")
    return out


def igs_problem_timing(prob) -> igs_timing:
    out = igs_timing()
    _check(_lib.igs_problem_timing(prob, C.byref(out)), "igs_problem_timing")
    return out


def igs_build_weighted_rules(prob) -> None:
    _check(_lib.igs_build_weighted_rules(prob), "igs_build_weighted_rules")


def igs_assemble(prob, A_out=None, ld: int | None = None, mem: int | None = None, dtype: int | None = None) -> None:
    """A_out: None, a host numpy array or a torch tensor (host or CUDA), n x ld."""
    if A_out is None:
        _check(_lib.igs_assemble(prob, None, 0, 0, 0), "igs_assemble")
        return
    if ld is None:
        ld = A_out.shape[1]
    if mem is None:
        mem = IGS_MEM_DEVICE if (hasattr(A_out, "is_cuda") and A_out.is_cuda) else IGS_MEM_HOST
    if dtype is None:
        dtype = IGS_F32 if str(A_out.dtype).endswith("float32") else IGS_F64
    _check(_lib.igs_assemble(prob, _ptr(A_out), int(ld), int(mem), int(dtype)), "igs_assemble")


def igs_get_matrix(prob, A_out, ld: int | None = None, mem: int | None = None, dtype: int | None = None) -> None:
    """Copy the assembled A into A_out (host numpy array or torch tensor), n x ld."""
    if ld is None:
        ld = A_out.shape[1]
    if mem is None:
        mem = IGS_MEM_DEVICE if (hasattr(A_out, "is_cuda") and A_out.is_cuda) else IGS_MEM_HOST
    if dtype is None:
        dtype = IGS_F32 if str(A_out.dtype).endswith("float32") else IGS_F64
    _check(_lib.igs_get_matrix(prob, _ptr(A_out), int(ld), int(mem), int(dtype)), "igs_get_matrix")


def igs_rhs_points(prob) -> np.ndarray:
    cnt = C.c_int64()
    _check(_lib.igs_rhs_points(prob, None, 0, C.byref(cnt)), "igs_rhs_points")
    xy = np.empty((cnt.value, 2), dtype=np.float64)
    _check(_lib.igs_rhs_points(prob, _ptr(xy), cnt.value, C.byref(cnt)), "igs_rhs_points")
    return xy


def _require_dev_f64(t, shape, where: str, what: str) -> None:
    """The C ABI carries no sizes for device buffers: refuse, before the call,
    a tensor the kernels would read or write out of bounds."""
    ok = (hasattr(t, "is_cuda") and t.is_cuda and str(t.dtype) == "torch.float64"
          and t.is_contiguous() and tuple(t.shape) == tuple(shape))
    if not ok:
        got = (f"{tuple(t.shape)} {t.dtype} {'cuda' if t.is_cuda else 'cpu'} "
               f"{'contiguous' if t.is_contiguous() else 'strided'}") if hasattr(t, "is_cuda") else type(t).__name__
        raise IgsError(IGS_E_INVALID_ARG, where,
                       f"{what} must be a contiguous float64 CUDA tensor of shape {tuple(shape)}, got {got}")


def igs_build_rhs(prob, uD, return_beta: bool = True):
    """uD: (nrhs, n_rhs_pts) values at igs_rhs_points: a host array, or a CUDA
    tensor (device memory; beta is then returned as a CUDA tensor)."""
    if hasattr(uD, "is_cuda") and uD.is_cuda:
        u = uD if uD.dim() == 2 else uD[None, :]
        _require_dev_f64(u, (u.shape[0], igs_problem_info(prob).n_rhs_pts), "igs_build_rhs", "uD")
        beta = None
        if return_beta:
            import torch
            beta = torch.empty((u.shape[0], igs_problem_info(prob).n), dtype=torch.float64, device=u.device)
        _check(_lib.igs_build_rhs(prob, _ptr(u), u.shape[0], _ptr(beta), IGS_MEM_DEVICE), "igs_build_rhs")
        return beta
    u = _f64(uD)
    if u.ndim == 1:
        u = u[None, :]
    nrhs = u.shape[0]
    beta = np.empty((nrhs, igs_problem_info(prob).n), dtype=np.float64) if return_beta else None
    _check(_lib.igs_build_rhs(prob, _ptr(u), nrhs, _ptr(beta), IGS_MEM_HOST), "igs_build_rhs")
    return beta


def igs_build_rhs_noalloc(prob, uD, beta_out) -> None:
    """Right-hand side into caller-owned device memory without any device
    allocation (uD: CUDA tensor nrhs x n_rhs_pts; beta_out: CUDA tensor nrhs x n)."""
    info = igs_problem_info(prob)
    u = uD if (hasattr(uD, "dim") and uD.dim() == 2) else (uD[None, :] if hasattr(uD, "dim") else uD)
    _require_dev_f64(u, (u.shape[0], info.n_rhs_pts), "igs_build_rhs_noalloc", "uD")
    _require_dev_f64(beta_out, (u.shape[0], info.n), "igs_build_rhs_noalloc", "beta_out")
    if beta_out.device != u.device:
        raise IgsError(IGS_E_INVALID_ARG, "igs_build_rhs_noalloc", "uD and beta_out must be on the same device")
    _check(_lib.igs_build_rhs_noalloc(prob, _ptr(u), int(u.shape[0]), _ptr(beta_out)), "igs_build_rhs_noalloc")


def igs_solve(prob, beta=None, nrhs: int = 1, alpha_out=None, mem: int = IGS_MEM_HOST):
    """Returns (alpha, residuals).  beta: None (use the built rhs) or (nrhs, n)."""
    n = igs_problem_info(prob).n
    if beta is not None and mem == IGS_MEM_HOST:
        beta = _f64(beta).reshape(-1, n)
        nrhs = beta.shape[0]
    if alpha_out is None:
        alpha_out = np.empty((nrhs, n), dtype=np.float64)
    res = np.empty(nrhs, dtype=np.float64)
    _check(_lib.igs_solve(prob, _ptr(beta), int(nrhs), _ptr(alpha_out), _ptr(res), int(mem)), "igs_solve")
    return alpha_out, res


def igs_solve_data(prob, uD, alpha_out=None):
    """Right-hand side from u_D (nrhs, n_rhs_pts) and solve, overlapped on the
    GPU; returns (alpha, residuals).  Host arrays, or CUDA tensors (device
    memory; alpha_out, if given, a CUDA tensor nrhs x n)."""
    n = igs_problem_info(prob).n
    if hasattr(uD, "is_cuda") and uD.is_cuda:
        u = uD if uD.dim() == 2 else uD[None, :]
        nrhs = int(u.shape[0])
        _require_dev_f64(u, (nrhs, igs_problem_info(prob).n_rhs_pts), "igs_solve_data", "uD")
        if alpha_out is None:
            import torch
            alpha_out = torch.empty((nrhs, n), dtype=torch.float64, device=u.device)
        _require_dev_f64(alpha_out, (nrhs, n), "igs_solve_data", "alpha_out")
        res = np.empty(nrhs, dtype=np.float64)
        _check(_lib.igs_solve_data(prob, _ptr(u), nrhs, _ptr(alpha_out), _ptr(res), IGS_MEM_DEVICE), "igs_solve_data")
        return alpha_out, res
    u = _f64(uD)
    if u.ndim == 1:
        u = u[None, :]
    nrhs = u.shape[0]
    alpha = np.empty((nrhs, n), dtype=np.float64)
    res = np.empty(nrhs, dtype=np.float64)
    _check(_lib.igs_solve_data(prob, _ptr(u), nrhs, _ptr(alpha), _ptr(res), IGS_MEM_HOST), "igs_solve_data")
    return alpha, res


def igs_eval_potential(prob, alpha, uD, xy, u_out=None):
    """u at the points xy (count x 2) by the representation formula.
    alpha: (nrhs, n); uD: (nrhs, n_rhs_pts) values at igs_rhs_points (None for
    an open arc).  Host arrays, or CUDA tensors (device memory; u_out, if
    given, a CUDA tensor nrhs x count).  Returns u (nrhs, count)."""
    if hasattr(alpha, "is_cuda") and alpha.is_cuda:
        import torch
        a = alpha if alpha.dim() == 2 else alpha[None, :]
        nrhs, count = int(a.shape[0]), int(xy.shape[0])
        if u_out is None:
            u_out = torch.empty((nrhs, count), dtype=torch.float64, device=a.device)
        _check(_lib.igs_eval_potential(prob, _ptr(a), _ptr(uD), nrhs, _ptr(xy), count, _ptr(u_out), IGS_MEM_DEVICE),
               "igs_eval_potential")
        return u_out
    a = _f64(alpha)
    if a.ndim == 1:
        a = a[None, :]
    nrhs = a.shape[0]
    u = None if uD is None else _f64(uD).reshape(nrhs, -1)
    x = _f64(xy).reshape(-1, 2)
    out = np.empty((nrhs, x.shape[0]), dtype=np.float64)
    _check(_lib.igs_eval_potential(prob, _ptr(a), _ptr(u), nrhs, _ptr(x), x.shape[0], _ptr(out), IGS_MEM_HOST),
           "igs_eval_potential")
    return out


def igs_collocation(prob, uD, return_matrix: bool = False):
    """Collocation solution alpha (nrhs, n) from u_D (nrhs, n_rhs_pts) at
    igs_rhs_points (host arrays).  Returns alpha, or (alpha, Ac, nodes) with
    the n x n collocation matrix and the collocation node indices."""
    u = _f64(uD)
    if u.ndim == 1:
        u = u[None, :]
    nrhs = u.shape[0]
    n = igs_problem_info(prob).n
    alpha = np.empty((nrhs, n), dtype=np.float64)
    Ac = np.empty((n, n), dtype=np.float64) if return_matrix else None
    nodes = np.empty(n, dtype=np.int32) if return_matrix else None
    _check(_lib.igs_collocation(prob, _ptr(u), nrhs, _ptr(alpha), _ptr(Ac), _ptr(nodes), IGS_MEM_HOST),
           "igs_collocation")
    return (alpha, Ac, nodes) if return_matrix else alpha


def igs_get_rules(prob, with_ws: bool = False):
    info = igs_problem_info(prob)
    nq, d1 = info.n_quad, info.degree + 1
    eta = np.empty(nq)
    wb = np.empty((nq, d1))
    first = np.empty(nq, dtype=np.int32)
    ws = np.empty((nq, nq)) if with_ws else None
    _check(_lib.igs_get_rules(prob, _ptr(eta), _ptr(wb), _ptr(first), _ptr(ws)), "igs_get_rules")
    return eta, wb, first, ws


def igs_get_node_geometry(prob):
    nq = igs_problem_info(prob).n_quad
    xy = np.empty((nq, 2))
    J = np.empty(nq)
    _check(_lib.igs_get_node_geometry(prob, _ptr(xy), _ptr(J)), "igs_get_node_geometry")
    return xy, J


def igs_selftest_wait(ctx, budget_s=0.01):
    """Run the bounded-wait self-test; returns 1 when the wait gave up by its budget."""
    out = C.c_int(0)
    _check(_lib.igs_selftest_wait(ctx, float(budget_s), C.byref(out)), "igs_selftest_wait")
    return out.value


def igs_measure_peak(ctx, kind: int) -> tuple[float, float]:
    """(rate, ms) of one arithmetic pipe: flop/s for the FMA kinds,
    instructions/s for the MUFU kinds."""
    rate, ms = C.c_double(0.0), C.c_double(0.0)
    _check(_lib.igs_measure_peak(ctx, int(kind), C.byref(rate), C.byref(ms)), "igs_measure_peak")
    return rate.value, ms.value


# ------------------------------------------------------------------ batched form
def _cfg_dict(c: igs_batch_config) -> dict:
    return {"tile": c.tile, "order": c.order, "ctas_per_sm": c.ctas_per_sm, "ms": c.ms}


def igs_batch_create(ctx, probs) -> C.c_void_p:
    arr = (C.c_void_p * len(probs))(*[p.value if isinstance(p, C.c_void_p) else p for p in probs])
    h = C.c_void_p()
    _check(_lib.igs_batch_create(ctx, C.byref(h), arr, len(probs)), "igs_batch_create")
    return h


def igs_batch_destroy(batch) -> None:
    _check(_lib.igs_batch_destroy(batch), "igs_batch_destroy")


def igs_batch_assemble(batch) -> float:
    ms = C.c_float()
    _check(_lib.igs_batch_assemble(batch, C.byref(ms)), "igs_batch_assemble")
    return ms.value


def igs_batch_tune(batch, reps: int = 2) -> dict:
    c = igs_batch_config()
    _check(_lib.igs_batch_tune(batch, C.byref(c), int(reps)), "igs_batch_tune")
    return _cfg_dict(c)


def igs_batch_set_config(batch, tile: int = 32, order: int = IGS_ORDER_NATURAL, ctas_per_sm: int = 0) -> None:
    c = igs_batch_config(int(tile), int(order), int(ctas_per_sm), 0.0)
    _check(_lib.igs_batch_set_config(batch, C.byref(c)), "igs_batch_set_config")


def igs_batch_get_config(batch) -> dict:
    c = igs_batch_config()
    _check(_lib.igs_batch_get_config(batch, C.byref(c)), "igs_batch_get_config")
    return _cfg_dict(c)


# ------------------------------------------------------------------ served form
_callbacks: dict = {}     # (server, ticket) -> (callback, request) kept alive until the result is taken


def _stats_dict(st: igs_request_stats) -> dict:
    return {k: getattr(st, k) for k, _ in igs_request_stats._fields_}


def igs_server_create(device: int = 0, slots: int = 4, mem_budget: int = 180 * 10**9,
                      cache_budget: int = 0) -> C.c_void_p:
    h = C.c_void_p()
    opts = igs_server_opts(int(slots), int(mem_budget), int(cache_budget))
    _check(_lib.igs_server_create(int(device), C.byref(opts), C.byref(h)), "igs_server_create")
    return h


def igs_server_submit(server, curve, degree: int, n_elems: int, n_ref: int, precision: int, nrhs: int, data) -> int:
    """data(xy, nrhs) -> array (nrhs, len(xy)): Dirichlet data at the request's
    right-hand-side points (called on a server thread)."""
    knots, ctrl = _f64(curve.knots), _f64(curve.ctrl)
    w = None if curve.weights is None else _f64(curve.weights)

    def cb(_user, xy_p, count, k, out_p):
        try:
            xy = np.ctypeslib.as_array(xy_p, shape=(int(count), 2))
            out = np.ctypeslib.as_array(out_p, shape=(int(k), int(count)))
            out[:, :] = np.asarray(data(xy.copy(), int(k)), dtype=np.float64).reshape(int(k), int(count))
            return 0
        except Exception:                                   # noqa: BLE001 - reported as a failed request
            return 1

    fn = DATA_FN(cb)
    req = igs_request(int(curve.degree), len(knots), knots.ctypes.data, len(ctrl), ctrl.ctypes.data,
                      None if w is None else w.ctypes.data, int(curve.closed), int(degree), int(n_elems),
                      int(n_ref), int(precision), int(nrhs), fn, None)
    t = C.c_int64()
    _check(_lib.igs_server_submit(server, C.byref(req), C.byref(t)), "igs_server_submit")
    _callbacks[(server.value, t.value)] = (fn, req, knots, ctrl, w)
    return t.value


def igs_server_wait(server, ticket: int, timeout_ms: int = -1) -> dict:
    st = igs_request_stats()
    _check(_lib.igs_server_wait(server, int(ticket), int(timeout_ms), C.byref(st)), "igs_server_wait")
    return _stats_dict(st)


def igs_server_result(server, ticket: int, n: int, nrhs: int):
    """Returns (alpha (nrhs, n), resid (nrhs,), stats)."""
    alpha = np.empty((nrhs, n), dtype=np.float64)
    resid = np.empty(nrhs, dtype=np.float64)
    st = igs_request_stats()
    try:
        _check(_lib.igs_server_result(server, int(ticket), _ptr(alpha), _ptr(resid), C.byref(st)), "igs_server_result")
    finally:
        if st.status in (IGS_REQ_DONE, IGS_REQ_FAILED):
            _callbacks.pop((server.value, int(ticket)), None)
    return alpha, resid, _stats_dict(st)


def igs_server_drain(server, timeout_ms: int = -1) -> None:
    _check(_lib.igs_server_drain(server, int(timeout_ms)), "igs_server_drain")


def igs_server_destroy(server) -> None:
    _check(_lib.igs_server_destroy(server), "igs_server_destroy")
    for key in [k for k in _callbacks if k[0] == server.value]:
        _callbacks.pop(key, None)
