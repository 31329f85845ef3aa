"""Thin ctypes binding of libsps.so (include/sps.h), same names as the C ABI.

Argument marshalling only: every step of the solve runs in the CUDA library.
Buffers may be numpy arrays (host memory, mem = SPS_MEM_HOST) or CUDA torch
tensors (device memory, mem = SPS_MEM_DEVICE); the stream defaults to
torch's current stream when torch has a CUDA device.  If the library is
missing or fails to load, importing this module raises: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

SPS_OK, SPS_EINVAL, SPS_EDOM, SPS_ENOMEM, SPS_ESTATE = 0, -1, -2, -3, -4
SPS_EBREAKDOWN, SPS_ENOCONV, SPS_ETIMEOUT, SPS_ECUDA, SPS_EEMPTY, SPS_EINTERNAL = -5, -6, -7, -8, -9, -10
SPS_F32, SPS_F64 = 0, 1
SPS_MEM_HOST, SPS_MEM_DEVICE = 0, 1
SPS_PREC_FP64, SPS_PREC_MIXED = 0, 1

ERROR_NAMES = {0: "SPS_OK", -1: "SPS_EINVAL", -2: "SPS_EDOM", -3: "SPS_ENOMEM", -4: "SPS_ESTATE",
               -5: "SPS_EBREAKDOWN", -6: "SPS_ENOCONV", -7: "SPS_ETIMEOUT", -8: "SPS_ECUDA", -9: "SPS_EEMPTY",
               -10: "SPS_EINTERNAL"}

EXPORTED = ["sps_default_options", "sps_plan_create", "sps_set_points", "sps_solve", "sps_destroy",
            "sps_last_error", "sps_coef_count", "sps_apply", "sps_penalty_apply", "sps_diag", "sps_rhs",
            "sps_prolong", "sps_restrict", "sps_coarse_solve", "sps_vcycle", "sps_get_sort", "sps_get_omega",
            "sps_set_omega", "sps_probe_fma_rate", "sps_point_apply", "sps_launch_count",
            "sps_profile_begin", "sps_profile_end", "sps_solve_batch", "sps_set_lambda",
            "sps_penalty_apply_noalloc", "sps_get_tuning", "sps_evaluate", "sps_level_matrix",
            "sps_plan_device_bytes", "sps_solve_batch_shape", "sps_tune_batch", "sps_lanczos_estimate",
            "sps_simulate_batch"]


class sps_options(C.Structure):
    _fields_ = [("precision", C.c_int), ("nu1", C.c_int), ("nu2", C.c_int), ("omega", C.c_double),
                ("power_iters", C.c_int), ("max_iter", C.c_int), ("warm_start", C.c_int), ("tile", C.c_int),
                ("replace_ratio", C.c_double), ("hybrid", C.c_int),
                ("graphs", C.c_int), ("precondition", C.c_int), ("autotune", C.c_int),
                ("lanes_r", C.c_int), ("coarse_cg", C.c_int), ("coarse_iters", C.c_int),
                ("max_device_bytes", C.c_int64)]


class sps_result(C.Structure):
    _fields_ = [("status", C.c_int), ("iterations", C.c_int), ("rel_res", C.c_double),
                ("rel_res_true", C.c_double), ("fp64_applies", C.c_int), ("solve_ms", C.c_double)]


class sps_batch_shape(C.Structure):
    _fields_ = [("cluster", C.c_int), ("big", C.c_int), ("predicted_ms", C.c_double)]


class SpsError(RuntimeError):
    def __init__(self, code, where, msg):
        super().__init__("%s failed: %s (%s)" % (where, ERROR_NAMES.get(code, code), msg))
        self.code = code


def load(path: str | None = None) -> C.CDLL:
    path = path or _build.LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError("libsps.so not built (%s); run __graft_entry__.build()" % path)
    lib = C.CDLL(path)
    P, I, D, V = C.c_void_p, C.c_int, C.c_double, None
    sig = {
        "sps_default_options": (V, [C.POINTER(sps_options)]),
        "sps_plan_create": (I, [C.POINTER(P), I, I, C.POINTER(C.c_int), C.POINTER(D), C.POINTER(D), I, D,
                                C.POINTER(sps_options)]),
        "sps_set_points": (I, [P, C.c_int64, P, P, I, I, P]),
        "sps_solve": (I, [P, P, I, D, C.POINTER(sps_result), P]),
        "sps_destroy": (I, [P]),
        "sps_last_error": (C.c_char_p, []),
        "sps_coef_count": (I, [P, I, C.POINTER(C.c_int64)]),
        "sps_apply": (I, [P, I, I, P, P, I, P]),
        "sps_penalty_apply": (I, [P, I, I, P, P, I, P]),
        "sps_diag": (I, [P, I, P, I, P]),
        "sps_rhs": (I, [P, P, I, P]),
        "sps_prolong": (I, [P, I, I, P, P, I, P]),
        "sps_restrict": (I, [P, I, I, P, P, I, P]),
        "sps_coarse_solve": (I, [P, P, P, I, P]),
        "sps_vcycle": (I, [P, I, P, P, I, P]),
        "sps_get_sort": (I, [P, P, P, I, P]),
        "sps_get_omega": (I, [P, P]),
        "sps_get_tuning": (I, [P, I, P, P]),
        "sps_evaluate": (I, [P, P, C.c_int64, P, I, P, I, P]),
        "sps_set_omega": (I, [P, P]),
        "sps_lanczos_estimate": (I, [P, P, I, C.POINTER(D), C.POINTER(D)]),
        "sps_simulate_batch": (I, [P, P, P, I, I, I, I, C.POINTER(D)]),
        "sps_probe_fma_rate": (I, [I, C.POINTER(D), P]),
        "sps_point_apply": (I, [P, I, I, P, P, I, P]),
        "sps_launch_count": (I, [C.POINTER(C.c_uint64)]),
        "sps_profile_begin": (I, []),
        "sps_profile_end": (I, [C.POINTER(D), C.POINTER(C.c_uint64)]),
        "sps_solve_batch": (I, [C.POINTER(P), I, C.POINTER(P), I, D, C.POINTER(sps_result), P]),
        "sps_set_lambda": (I, [P, D]),
        "sps_penalty_apply_noalloc": (I, [I, C.POINTER(C.c_int), C.POINTER(D), C.POINTER(D), D, P, P, P]),
        "sps_level_matrix": (I, [P, I, P, C.POINTER(C.c_int64), I, P]),
        "sps_plan_device_bytes": (I, [P, C.POINTER(C.c_int64)]),
        "sps_solve_batch_shape": (I, [C.POINTER(P), I, C.POINTER(P), I, D, C.POINTER(sps_batch_shape),
                                      C.POINTER(sps_result), C.POINTER(sps_batch_shape), P]),
        "sps_tune_batch": (I, [C.POINTER(P), I, C.POINTER(P), I, D, C.POINTER(sps_batch_shape), P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_LIB = None


def lib() -> C.CDLL:
    global _LIB
    if _LIB is None:
        _LIB = load()
    return _LIB


def _check(code: int, where: str) -> int:
    if code != SPS_OK:
        raise SpsError(code, where, lib().sps_last_error().decode())
    return code


def _stream(stream):
    if stream is not None:
        return C.c_void_p(int(stream))
    try:
        import torch
        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return C.c_void_p(0)


def _buf(a):
    """(pointer, mem) of a numpy array or CUDA tensor."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return C.c_void_p(a.ctypes.data), SPS_MEM_HOST
    if hasattr(a, "data_ptr") and getattr(a, "is_cuda", False):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return C.c_void_p(a.data_ptr()), SPS_MEM_DEVICE
    raise TypeError("expected a numpy array or a CUDA tensor, got %r" % type(a))


# ---------------------------------------------------------------- same-name wrappers

def sps_default_options() -> sps_options:
    o = sps_options()
    lib().sps_default_options(C.byref(o))
    return o


def sps_plan_create(P, q, intervals, lo=None, hi=None, levels=1, lam=1e-3, opt=None) -> C.c_void_p:
    h = C.c_void_p()
    iv = (C.c_int * P)(*intervals)
    lo_a = (C.c_double * P)(*lo) if lo is not None else None
    hi_a = (C.c_double * P)(*hi) if hi is not None else None
    _check(lib().sps_plan_create(C.byref(h), P, q, iv, lo_a, hi_a, levels, lam,
                                 C.byref(opt) if opt is not None else None), "sps_plan_create")
    return h


def sps_set_points(plan, x, y, stream=None) -> None:
    px, mx = _buf(x)
    py, my = _buf(y)
    if mx != my:
        raise ValueError("x and y must live in the same memory")
    dt = str(x.dtype)
    dtype = SPS_F64 if dt.endswith("float64") else SPS_F32 if dt.endswith("float32") else None
    if dtype is None or str(y.dtype) != dt:
        raise TypeError("x and y must both be float32 or both float64")
    n = x.shape[0]
    _check(lib().sps_set_points(plan, n, px, py, dtype, mx, _stream(stream)), "sps_set_points")


def sps_solve(plan, coef, tol, stream=None, check=True) -> sps_result:
    pc, mc = _buf(coef)
    res = sps_result()
    code = lib().sps_solve(plan, pc, mc, tol, C.byref(res), _stream(stream))
    if check:
        _check(code, "sps_solve")
    return res


def sps_solve_batch(plans, coefs, tol, stream=None, check=True) -> list:
    """plans: list of plan handles; coefs: list of numpy arrays or CUDA tensors (one per plan)."""
    n = len(plans)
    ph = (C.c_void_p * n)(*[p.value if isinstance(p, C.c_void_p) else p for p in plans])
    bufs = [_buf(c) for c in coefs]
    mems = {m for _, m in bufs}
    if len(mems) != 1:
        raise ValueError("all coefficient buffers must live in the same memory")
    ch = (C.c_void_p * n)(*[b[0].value for b in bufs])
    res = (sps_result * n)()
    code = lib().sps_solve_batch(ph, n, ch, mems.pop(), tol, res, _stream(stream))
    if check:
        _check(code, "sps_solve_batch")
    return list(res)


def _batch_args(plans, coefs):
    n = len(plans)
    ph = (C.c_void_p * n)(*[p.value if isinstance(p, C.c_void_p) else p for p in plans])
    bufs = [_buf(c) for c in coefs]
    mems = {m for _, m in bufs}
    if len(mems) != 1:
        raise ValueError("all coefficient buffers must live in the same memory")
    ch = (C.c_void_p * n)(*[b[0].value for b in bufs])
    return n, ph, ch, mems.pop()


def sps_solve_batch_shape(plans, coefs, tol, cluster=None, big=-1, stream=None, check=True) -> tuple:
    """Batched solve with an explicit shape (cluster None: the tuned or default
    shape); returns (results, shape that ran)."""
    n, ph, ch, mem = _batch_args(plans, coefs)
    res = (sps_result * n)()
    used = sps_batch_shape()
    shp = C.byref(sps_batch_shape(cluster, big, 0.0)) if cluster is not None else None
    code = lib().sps_solve_batch_shape(ph, n, ch, mem, tol, shp, res, C.byref(used), _stream(stream))
    if check:
        _check(code, "sps_solve_batch_shape")
    return list(res), (used.cluster, used.big)


def sps_tune_batch(plans, coefs, tol, stream=None) -> tuple:
    """Autotune the batched solver for these problems: (cluster, big, predicted ms)."""
    n, ph, ch, mem = _batch_args(plans, coefs)
    best = sps_batch_shape()
    _check(lib().sps_tune_batch(ph, n, ch, mem, tol, C.byref(best), _stream(stream)), "sps_tune_batch")
    return best.cluster, best.big, best.predicted_ms


SPS_NOALLOC_MAX_COEF = 262144


def sps_penalty_apply_noalloc(P, intervals, lo, hi, scale, v, u, stream=None) -> None:
    """u = scale * Lambda v on the grid without any device allocation (v, u: CUDA tensors)."""
    pv, mv = _buf(v)
    pu, mu = _buf(u)
    if mv != SPS_MEM_DEVICE or mu != SPS_MEM_DEVICE:
        raise ValueError("v and u must be device buffers")
    iv = (C.c_int * P)(*intervals)
    lo_a = (C.c_double * P)(*lo) if lo is not None else None
    hi_a = (C.c_double * P)(*hi) if hi is not None else None
    _check(lib().sps_penalty_apply_noalloc(P, iv, lo_a, hi_a, scale, pv, pu, _stream(stream)),
           "sps_penalty_apply_noalloc")


def sps_set_lambda(plan, lam) -> None:
    _check(lib().sps_set_lambda(plan, lam), "sps_set_lambda")


def sps_destroy(plan) -> None:
    _check(lib().sps_destroy(plan), "sps_destroy")


def sps_last_error() -> str:
    return lib().sps_last_error().decode()


def sps_coef_count(plan, level) -> int:
    k = C.c_int64()
    _check(lib().sps_coef_count(plan, level, C.byref(k)), "sps_coef_count")
    return k.value


def _vec_call(name, plan, level, prec, a, b, stream):
    pa, ma = _buf(a)
    pb, mb = _buf(b)
    if ma != mb:
        raise ValueError("input and output must live in the same memory")
    _check(getattr(lib(), name)(plan, level, prec, pa, pb, ma, _stream(stream)), name)


def sps_apply(plan, level, prec, v, u, stream=None):
    _vec_call("sps_apply", plan, level, prec, v, u, stream)


def sps_point_apply(plan, level, prec, v, u, stream=None):
    _vec_call("sps_point_apply", plan, level, prec, v, u, stream)


def sps_evaluate(plan, coef, xq, out, stream=None) -> None:
    """out[j] = s(xq[j]) of the spline with coefficients coef (finest grid)."""
    pc, mc = _buf(coef)
    px, mx = _buf(xq)
    po, mo = _buf(out)
    if not (mc == mx == mo):
        raise ValueError("coef, xq and out must live in the same memory")
    dt = str(xq.dtype)
    dtype = SPS_F64 if dt.endswith("float64") else SPS_F32 if dt.endswith("float32") else None
    if dtype is None:
        raise TypeError("xq must be float32 or float64")
    _check(lib().sps_evaluate(plan, pc, xq.shape[0], px, dtype, po, mc, _stream(stream)), "sps_evaluate")


def sps_launch_count() -> int:
    c = C.c_uint64()
    _check(lib().sps_launch_count(C.byref(c)), "sps_launch_count")
    return c.value


def sps_profile_begin() -> None:
    _check(lib().sps_profile_begin(), "sps_profile_begin")


def sps_profile_end() -> tuple:
    ms = C.c_double()
    cnt = C.c_uint64()
    _check(lib().sps_profile_end(C.byref(ms), C.byref(cnt)), "sps_profile_end")
    return ms.value, cnt.value


def sps_penalty_apply(plan, level, prec, v, u, stream=None):
    _vec_call("sps_penalty_apply", plan, level, prec, v, u, stream)


def sps_prolong(plan, level, prec, c, f, stream=None):
    _vec_call("sps_prolong", plan, level, prec, c, f, stream)


def sps_restrict(plan, level, prec, f, c, stream=None):
    _vec_call("sps_restrict", plan, level, prec, f, c, stream)


def sps_diag(plan, level, d, stream=None):
    pd, md = _buf(d)
    _check(lib().sps_diag(plan, level, pd, md, _stream(stream)), "sps_diag")


def sps_rhs(plan, b, stream=None):
    pb, mb = _buf(b)
    _check(lib().sps_rhs(plan, pb, mb, _stream(stream)), "sps_rhs")


def sps_coarse_solve(plan, r, e, stream=None):
    pr, mr = _buf(r)
    pe, me = _buf(e)
    _check(lib().sps_coarse_solve(plan, pr, pe, mr, _stream(stream)), "sps_coarse_solve")


def sps_vcycle(plan, prec, r, z, stream=None):
    pr, mr = _buf(r)
    pz, mz = _buf(z)
    _check(lib().sps_vcycle(plan, prec, pr, pz, mr, _stream(stream)), "sps_vcycle")


def sps_get_sort(plan, perm=None, key=None, stream=None):
    pp, mp = _buf(perm) if perm is not None else (None, None)
    pk, mk = _buf(key) if key is not None else (None, None)
    mem = mp if mp is not None else mk
    _check(lib().sps_get_sort(plan, pp, pk, mem if mem is not None else SPS_MEM_HOST, _stream(stream)),
           "sps_get_sort")


def sps_get_omega(plan, levels) -> np.ndarray:
    out = np.zeros(levels)
    _check(lib().sps_get_omega(plan, C.c_void_p(out.ctypes.data)), "sps_get_omega")
    return out


def sps_get_tuning(plan, level) -> tuple:
    """(tile side, lanes layout) of a level's point operator."""
    ts, lr = C.c_int(0), C.c_int(0)
    _check(lib().sps_get_tuning(plan, level, C.byref(ts), C.byref(lr)), "sps_get_tuning")
    return ts.value, lr.value


def sps_set_omega(plan, omega) -> None:
    arr = np.ascontiguousarray(omega, dtype=np.float64)
    _check(lib().sps_set_omega(plan, C.c_void_p(arr.ctypes.data)), "sps_set_omega")


def sps_lanczos_estimate(alpha, beta2) -> tuple:
    """(theta, lambda_hat) from Lanczos coefficients alpha_j, beta_j^2 (host only)."""
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    b = np.ascontiguousarray(beta2, dtype=np.float64)
    if a.shape != b.shape or a.ndim != 1:
        raise ValueError("alpha and beta2 must be 1-D arrays of one length")
    th, lh = C.c_double(), C.c_double()
    _check(lib().sps_lanczos_estimate(C.c_void_p(a.ctypes.data), C.c_void_p(b.ctypes.data), a.size,
                                      C.byref(th), C.byref(lh)), "sps_lanczos_estimate")
    return th.value, lh.value


def sps_simulate_batch(order, t1, tc, cluster, big, grid) -> float:
    """Makespan (ms) of the batched solver's queues for per-problem times (host only)."""
    o = np.ascontiguousarray(order, dtype=np.int32)
    a = np.ascontiguousarray(t1, dtype=np.float64)
    b = np.ascontiguousarray(tc, dtype=np.float64)
    if not (o.ndim == a.ndim == b.ndim == 1 and o.size == a.size == b.size):
        raise ValueError("order, t1 and tc must be 1-D arrays of one length")
    out = C.c_double()
    _check(lib().sps_simulate_batch(C.c_void_p(o.ctypes.data), C.c_void_p(a.ctypes.data), C.c_void_p(b.ctypes.data),
                                    o.size, cluster, big, grid, C.byref(out)), "sps_simulate_batch")
    return out.value


def sps_plan_device_bytes(plan) -> int:
    b = C.c_int64()
    _check(lib().sps_plan_device_bytes(plan, C.byref(b)), "sps_plan_device_bytes")
    return b.value


def sps_level_matrix(plan, level, out=None, stream=None) -> int:
    """Number of entries of level `level`'s assembled matrix (0: matrix free);
    with `out` (numpy array or CUDA tensor of that many doubles) also copies them."""
    cnt = C.c_int64()
    if out is None:
        _check(lib().sps_level_matrix(plan, level, None, C.byref(cnt), SPS_MEM_HOST, _stream(stream)),
               "sps_level_matrix")
        return cnt.value
    po, mo = _buf(out)
    _check(lib().sps_level_matrix(plan, level, po, C.byref(cnt), mo, _stream(stream)), "sps_level_matrix")
    return cnt.value


def sps_probe_fma_rate(fp64: bool, stream=None) -> float:
    r = C.c_double()
    _check(lib().sps_probe_fma_rate(1 if fp64 else 0, C.byref(r), _stream(stream)), "sps_probe_fma_rate")
    return r.value


# ---------------------------------------------------------------- convenience

class Plan:
    """Owns one sps_plan: create / set_points / solve / destroy."""

    def __init__(self, P, intervals, levels, lam, lo=None, hi=None, q=3, **options):
        self.opt = sps_default_options()
        for k, v in options.items():
            setattr(self.opt, k, v)
        self.P, self.levels = P, levels
        self.h = sps_plan_create(P, q, intervals, lo, hi, levels, lam, self.opt)

    @property
    def K(self) -> int:
        return sps_coef_count(self.h, self.levels)

    def coef_count(self, level) -> int:
        return sps_coef_count(self.h, level)

    def set_points(self, x, y, stream=None):
        sps_set_points(self.h, x, y, stream)

    def solve(self, tol, coef=None, stream=None, check=True):
        if coef is None:
            coef = np.zeros(self.K)
        res = sps_solve(self.h, coef, tol, stream, check=check)
        return coef, res

    def evaluate(self, coef, xq, out=None, stream=None):
        """Values of the spline with coefficients coef at the query points xq."""
        if out is None:
            out = np.zeros(xq.shape[0])
        sps_evaluate(self.h, coef, xq, out, stream)
        return out

    def close(self):
        if self.h:
            sps_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
