"""Python binding of the GB300 level-blocked MPK library (libmpk_gb300.so).

Argument marshalling only: every step of the computation runs in the library's CUDA kernels.
PyTorch provides device memory and streams.  The functions carry the names of the C entry
points declared in include/mpk.h; they raise ``MpkError`` when a call returns an error status.
There is no CPU fallback: importing the binding without the built library raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmpk_gb300.so")

MPK_OK = 0
MPK_ERR_ARG = 1
MPK_ERR_CUDA = 2
MPK_ERR_OOM = 3
MPK_ERR_TIMEOUT = 4
MPK_ERR_BREAKDOWN = 5
MPK_ERR_NOT_CONVERGED = 6
MPK_ERR_UNIMPLEMENTED = 7
MPK_ERR_BUDGET = 8
MPK_ERR_NOT_READY = 9

MPK_F32 = 0
MPK_F64 = 1

MPK_PERMUTED_IO = 0x01
MPK_FINAL_ONLY = 0x02
MPK_HOST_IO = 0x04
MPK_UNBLOCKED = 0x08
MPK_Y0_IS_X = 0x10
MPK_RHS_INTERLEAVED = 0x20
MPK_JACOBI = 0x80
MPK_GS2 = 0x100


def MPK_GS2_GAMMA(gamma):
    """Inner-iteration count of MPK_GS2 in the flag word (0..15)."""
    return (int(gamma) & 15) << 12

MPK_DEBUG_DROP_FLAG = 0x40000000
MPK_NOALLOC_SCRATCH_BYTES = 32 << 20


class MpkError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = int(status)
        super().__init__("%s failed: %s" % (what, status_name(status)))


# ---------------------------------------------------------------------------------------------
# ctypes mirrors of the C structs
# ---------------------------------------------------------------------------------------------
class mpk_csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("row_ptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("val", ctypes.c_void_p), ("dtype", ctypes.c_int)]


class mpk_plan_opts(ctypes.Structure):
    _fields_ = [("l2_budget_bytes", ctypes.c_int64), ("p_blk", ctypes.c_int32),
                ("root_rule", ctypes.c_int32), ("n_sweeps", ctypes.c_int32),
                ("assume_symmetric", ctypes.c_int32), ("chunk_slices", ctypes.c_int32),
                ("keep_f32", ctypes.c_int32), ("keep_f64", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("wait_timeout_us", ctypes.c_uint32),
                ("schedule", ctypes.c_int32), ("slack_tasks", ctypes.c_int32),
                ("block_threads", ctypes.c_int32), ("stage", ctypes.c_int32),
                ("kernel", ctypes.c_int32), ("blocked", ctypes.c_int32),
                ("jacobi", ctypes.c_int32), ("shard_warps", ctypes.c_int32),
                ("lanes_per_row", ctypes.c_int32), ("task_units", ctypes.c_int32),
                ("task_dispatch", ctypes.c_int32), ("owner_lag", ctypes.c_int32),
                ("owner_prefetch", ctypes.c_int32), ("level_order", ctypes.c_int32)]


class mpk_plan_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("n_levels", ctypes.c_int32),
                ("n_groups", ctypes.c_int32), ("n_slices", ctypes.c_int32),
                ("n_chunks", ctypes.c_int32), ("root", ctypes.c_int32), ("p_blk", ctypes.c_int32),
                ("l2_budget_bytes", ctypes.c_int64), ("sell_nnz", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("create_ms", ctypes.c_double),
                ("bfs_sweeps", ctypes.c_int32), ("max_level_rows", ctypes.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class mpk_coeffs(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int32), ("a", ctypes.c_void_p), ("b", ctypes.c_void_p),
                ("c", ctypes.c_void_p), ("gamma", ctypes.c_void_p)]


class mpk_gmres_opts(ctypes.Structure):
    _fields_ = [("s", ctypes.c_int32), ("restart", ctypes.c_int32), ("tol", ctypes.c_double),
                ("inner_tol", ctypes.c_double), ("max_outer", ctypes.c_int32),
                ("inner_cycles", ctypes.c_int32), ("max_iters", ctypes.c_int32),
                ("basis", ctypes.c_int), ("bcgs_passes", ctypes.c_int32),
                ("shifts", ctypes.c_void_p), ("mpk_flags", ctypes.c_uint32),
                ("poly_degree", ctypes.c_int32), ("poly_f64", ctypes.c_int32),
                ("jacobi", ctypes.c_int32), ("gs2", ctypes.c_int32), ("gs2_gamma", ctypes.c_int32),
                ("trace_hist", ctypes.c_void_p), ("trace_cap", ctypes.c_int32),
                ("trace_H", ctypes.c_void_p)]


class mpk_gmres_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("outer", ctypes.c_int32), ("restarts", ctypes.c_int32),
                ("status", ctypes.c_int32), ("rel_residual", ctypes.c_double),
                ("shifts", ctypes.c_double * 64), ("ms_total", ctypes.c_double),
                ("ms_mpk", ctypes.c_double), ("ms_ortho", ctypes.c_double),
                ("ms_other", ctypes.c_double), ("poly_degree", ctypes.c_int32),
                ("poly_interval", ctypes.c_double * 2), ("trace_len", ctypes.c_int32),
                ("breakdowns", ctypes.c_int32), ("s_final", ctypes.c_int32)]


class mpk_tune_info(ctypes.Structure):
    _fields_ = [("n_trials", ctypes.c_int32), ("best_index", ctypes.c_int32),
                ("best_ms", ctypes.c_double), ("base_ms", ctypes.c_double)]


class mpk_cg_opts(ctypes.Structure):
    _fields_ = [("s", ctypes.c_int32), ("tol", ctypes.c_double), ("inner_tol", ctypes.c_double),
                ("max_outer", ctypes.c_int32), ("max_iters", ctypes.c_int32), ("basis", ctypes.c_int),
                ("shifts", ctypes.c_void_p), ("mpk_flags", ctypes.c_uint32), ("replace", ctypes.c_int32)]


class mpk_cg_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("outer", ctypes.c_int32), ("status", ctypes.c_int32),
                ("s_used", ctypes.c_int32), ("rel_residual", ctypes.c_double),
                ("shifts", ctypes.c_double * 16), ("ms_total", ctypes.c_double),
                ("ms_mpk", ctypes.c_double), ("ms_gram", ctypes.c_double),
                ("ms_other", ctypes.c_double)]


class mpk_server_opts(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("max_active", ctypes.c_int32),
                ("n_streams", ctypes.c_int32), ("gmres", mpk_gmres_opts)]


class mpk_server_result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("status", ctypes.c_int32), ("iters", ctypes.c_int32),
                ("outer", ctypes.c_int32), ("rel_residual", ctypes.c_double),
                ("t_submit_ms", ctypes.c_double), ("t_start_ms", ctypes.c_double),
                ("t_done_ms", ctypes.c_double)]


# ---------------------------------------------------------------------------------------------
# Library loading
# ---------------------------------------------------------------------------------------------
_lib = None

# (name, restype, argtypes) of every entry point declared in include/mpk.h
_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_U32 = ctypes.c_uint32
_D = ctypes.c_double
_SIGS = [
    ("mpk_plan_opts_default", ctypes.c_int, [ctypes.POINTER(mpk_plan_opts)]),
    ("mpk_plan_create", ctypes.c_int, [ctypes.POINTER(mpk_csr), _I32, ctypes.POINTER(mpk_plan_opts), _P, ctypes.POINTER(_P)]),
    ("mpk_plan_destroy", ctypes.c_int, [_P]),
    ("mpk_plan_stats", ctypes.c_int, [_P, ctypes.POINTER(mpk_plan_info)]),
    ("mpk_plan_perm", ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    ("mpk_plan_csr", ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, _P]),
    ("mpk_plan_update_values", ctypes.c_int, [_P, ctypes.POINTER(mpk_csr), _P]),
    ("mpk_apply", ctypes.c_int, [_P, ctypes.POINTER(mpk_coeffs), ctypes.c_int, _P, _I64, _P, _I64, _I32, _U32, _P]),
    ("mpk_plan_sync", ctypes.c_int, [_P, _P]),
    ("mpk_apply_final_noalloc", ctypes.c_int, [_P, ctypes.POINTER(mpk_coeffs), ctypes.c_int, _P, _P, _U32, _P]),
    ("mpk_noalloc_forget", ctypes.c_int, []),
    ("mpk_coeffs_chebyshev", ctypes.c_int, [_D, _D, _I32, _P, _P, _P]),
    ("mpk_coeffs_newton", ctypes.c_int, [_P, _I32, _P, _P, _P]),
    ("mpk_leja_order", ctypes.c_int, [_P, _I32, _I32, _P]),
    ("mpk_hessenberg_eigvals", ctypes.c_int, [_P, _I64, _I32, _P, _P]),
    ("mpk_gmres_opts_default", ctypes.c_int, [ctypes.POINTER(mpk_gmres_opts)]),
    ("sstep_gmres_solve", ctypes.c_int, [_P, _P, _P, ctypes.POINTER(mpk_gmres_opts), ctypes.POINTER(mpk_gmres_info), _P]),
    ("mpk_autotune", ctypes.c_int, [ctypes.POINTER(mpk_csr), _I32, ctypes.POINTER(mpk_coeffs), ctypes.c_int,
                                    _I32, _U32, ctypes.POINTER(mpk_plan_opts), _I32,
                                    ctypes.POINTER(mpk_plan_opts), ctypes.POINTER(mpk_tune_info), _P]),
    ("mpk_cg_opts_default", ctypes.c_int, [ctypes.POINTER(mpk_cg_opts)]),
    ("sstep_cg_solve", ctypes.c_int, [_P, _P, _P, ctypes.POINTER(mpk_cg_opts), ctypes.POINTER(mpk_cg_info), _P]),
    ("mpk_fma_peak", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_D), _P]),
    ("mpk_batch_create", ctypes.c_int, [_P, _I32, _I32, ctypes.c_int, _P, ctypes.POINTER(_P)]),
    ("mpk_batch_apply", ctypes.c_int, [_P, _P, _P, _P, _U32, _P]),
    ("mpk_batch_sync", ctypes.c_int, [_P, _P]),
    ("mpk_batch_destroy", ctypes.c_int, [_P]),
    ("mpk_gram", ctypes.c_int, [ctypes.c_int, _P, _I64, _I32, _P, _I64, _I32, _I64, _P, _P]),
    ("mpk_block_update", ctypes.c_int, [ctypes.c_int, _P, _I64, _I32, _P, _I64, _I32, _P, _P, _I64, _P, _P]),
    ("mpk_gram_pairs", ctypes.c_int, [ctypes.c_int, _P, _I64, _I32, _I64, _P, _P]),
    ("mpk_server_opts_default", ctypes.c_int, [ctypes.POINTER(mpk_server_opts)]),
    ("mpk_server_create", ctypes.c_int, [ctypes.POINTER(mpk_server_opts), ctypes.POINTER(_P)]),
    ("mpk_server_submit", ctypes.c_int, [_P, _I64, _I64, _P, _P, _P, _P, _P, ctypes.POINTER(_I64)]),
    ("mpk_server_poll", ctypes.c_int, [_P, ctypes.POINTER(mpk_server_result), _I32, ctypes.POINTER(_I32)]),
    ("mpk_server_pending", ctypes.c_int, [_P, ctypes.POINTER(_I64)]),
    ("mpk_server_destroy", ctypes.c_int, [_P]),
    ("mpk_status_str", ctypes.c_char_p, [ctypes.c_int]),
    ("mpk_version", ctypes.c_char_p, []),
]


def lib():
    """The loaded library; raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libmpk_gb300.so is not built: run __graft_entry__.build() or "
                              "python paper_2309_02228_gb300/build.py")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in _SIGS:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return [s[0] for s in _SIGS]


def status_name(st) -> str:
    try:
        return lib().mpk_status_str(int(st)).decode()
    except Exception:
        return "status %d" % int(st)


def _check(st, what):
    if st != MPK_OK:
        raise MpkError(st, what)


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _dtype_code(torch_dtype):
    import torch
    if torch_dtype == torch.float64:
        return MPK_F64
    if torch_dtype == torch.float32:
        return MPK_F32
    raise ValueError("values must be float32 or float64")


# ---------------------------------------------------------------------------------------------
# Plans
# ---------------------------------------------------------------------------------------------
def mpk_plan_opts_default(**overrides) -> mpk_plan_opts:
    o = mpk_plan_opts()
    _check(lib().mpk_plan_opts_default(ctypes.byref(o)), "mpk_plan_opts_default")
    names = {f for f, _ in o._fields_}
    for k, v in overrides.items():
        if k not in names:
            raise TypeError("mpk_plan_opts has no field %r" % k)
        setattr(o, k, v)
    return o


class Plan:
    """Owns an mpk_plan_t; destroyed with the object."""

    def __init__(self, handle, n, nnz, p_max):
        self.handle = ctypes.c_void_p(handle)
        self.n = n
        self.nnz = nnz
        self.p_max = p_max

    def __del__(self):
        try:
            if self.handle and self.handle.value:
                lib().mpk_plan_destroy(self.handle)
                self.handle = ctypes.c_void_p(0)
        except Exception:
            pass

    def stats(self):
        return mpk_plan_stats(self)


def _csr_struct(row_ptr, col, val):
    n = row_ptr.numel() - 1
    return mpk_csr(n, col.numel(), row_ptr.data_ptr(), col.data_ptr() if col.numel() else 0,
                   val.data_ptr() if val.numel() else 0, _dtype_code(val.dtype))


def mpk_plan_create(row_ptr, col, val, p_max, opts=None, stream=None) -> Plan:
    """row_ptr (int32[n+1]), col (int32[nnz]), val (float32/64[nnz]): CUDA tensors of A."""
    A = _csr_struct(row_ptr, col, val)
    h = ctypes.c_void_p(0)
    st = lib().mpk_plan_create(ctypes.byref(A), int(p_max),
                               ctypes.byref(opts) if opts is not None else None,
                               _stream_ptr(stream), ctypes.byref(h))
    _check(st, "mpk_plan_create")
    return Plan(h.value, A.n, A.nnz, p_max)


def mpk_plan_stats(plan) -> dict:
    info = mpk_plan_info()
    _check(lib().mpk_plan_stats(plan.handle, ctypes.byref(info)), "mpk_plan_stats")
    return info.as_dict()


def mpk_plan_perm(plan, stream=None):
    """Returns dict of CUDA int32 tensors: perm, iperm, level, level_ptr, group_ptr."""
    import torch
    st = mpk_plan_stats(plan)
    dev = torch.device("cuda", torch.cuda.current_device())
    out = {k: torch.empty(sz, dtype=torch.int32, device=dev) for k, sz in
           (("perm", plan.n), ("iperm", plan.n), ("level", plan.n),
            ("level_ptr", st["n_levels"] + 1), ("group_ptr", st["n_groups"] + 1))}
    _check(lib().mpk_plan_perm(plan.handle, _ptr(out["perm"]), _ptr(out["iperm"]),
                               _ptr(out["level"]), _ptr(out["level_ptr"]), _ptr(out["group_ptr"]),
                               _stream_ptr(stream)), "mpk_plan_perm")
    return out


def mpk_plan_csr(plan, dtype, stream=None):
    """The permuted matrix P A P^T: (row_ptr, col, val) CUDA tensors."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    rp = torch.empty(plan.n + 1, dtype=torch.int32, device=dev)
    ci = torch.empty(max(plan.nnz, 1), dtype=torch.int32, device=dev)
    vv = torch.empty(max(plan.nnz, 1), dtype=dtype, device=dev)
    _check(lib().mpk_plan_csr(plan.handle, _dtype_code(dtype), _ptr(rp), _ptr(ci), _ptr(vv),
                              _stream_ptr(stream)), "mpk_plan_csr")
    return rp, ci[: plan.nnz], vv[: plan.nnz]


def mpk_plan_update_values(plan, row_ptr, col, val, stream=None):
    A = _csr_struct(row_ptr, col, val)
    _check(lib().mpk_plan_update_values(plan.handle, ctypes.byref(A), _stream_ptr(stream)),
           "mpk_plan_update_values")


def mpk_plan_sync(plan, stream=None) -> int:
    """Synchronise and return the latched status (MPK_OK or MPK_ERR_TIMEOUT) without raising."""
    return int(lib().mpk_plan_sync(plan.handle, _stream_ptr(stream)))


class Coeffs:
    """Host coefficient arrays kept alive for the duration of a call."""

    def __init__(self, a, b, c, gamma=None):
        self.a = np.ascontiguousarray(a, dtype=np.float64)
        self.b = np.ascontiguousarray(b, dtype=np.float64)
        self.c = np.ascontiguousarray(c, dtype=np.float64)
        self.gamma = None if gamma is None else np.ascontiguousarray(gamma, dtype=np.float64)
        self.p = int(self.a.shape[0])
        if self.b.shape[0] != self.p or self.c.shape[0] != self.p:
            raise ValueError("a, b and c must have p entries each")
        if self.gamma is not None and self.gamma.shape[0] != self.p + 1:
            raise ValueError("gamma must have p + 1 entries")
        self.struct = mpk_coeffs(self.p, self.a.ctypes.data, self.b.ctypes.data,
                                 self.c.ctypes.data,
                                 self.gamma.ctypes.data if self.gamma is not None else 0)

    @classmethod
    def from_triples(cls, triples, gamma=None):
        t = np.asarray(triples, dtype=np.float64).reshape(-1, 3)
        return cls(t[:, 0], t[:, 1], t[:, 2], gamma)


def mpk_apply(plan, coeffs, X, Y, n_rhs=1, flags=0, ldx=None, ldy=None, dtype=None, stream=None):
    """Run the MPK.  X, Y: CUDA tensors (or host tensors with MPK_HOST_IO); see include/mpk.h
    for the layouts.  dtype defaults to Y's dtype."""
    if not isinstance(coeffs, Coeffs):
        coeffs = Coeffs.from_triples(coeffs)
    d = _dtype_code(Y.dtype if dtype is None else dtype)
    n = plan.n
    ldx = n if ldx is None else ldx
    ldy = n if ldy is None else ldy
    # the extent the call touches (a short tensor would be read or written past its end)
    inter = (flags & MPK_RHS_INTERLEAVED) != 0
    if n > 0:
        if X is not None:
            if X.dtype != Y.dtype:
                raise ValueError("X and Y must have the same dtype")
            need_x = n * n_rhs if inter else (n_rhs - 1) * ldx + n
            if X.numel() < need_x:
                raise ValueError("X holds %d elements, the call reads %d" % (X.numel(), need_x))
        nb = 1 if flags & MPK_FINAL_ONLY else coeffs.p + 1
        need_y = (nb - 1) * ldy * n_rhs + (n * n_rhs if inter else (n_rhs - 1) * ldy + n)
        if Y.numel() < need_y:
            raise ValueError("Y holds %d elements, the call writes %d" % (Y.numel(), need_y))
    st = lib().mpk_apply(plan.handle, ctypes.byref(coeffs.struct), d, _ptr(X), int(ldx), _ptr(Y),
                         int(ldy), int(n_rhs), int(flags), _stream_ptr(stream))
    _check(st, "mpk_apply")


def mpk_apply_final_noalloc(plan, coeffs, X, Y, flags=0, dtype=None, stream=None):
    """Final power (or gamma sum) of one right-hand side without any device allocation; the
    intermediate vectors live in the library's fixed per-device scratch array.  X, Y: CUDA
    vectors of n elements.  Calls that may overlap in time on one device must be ordered."""
    if not isinstance(coeffs, Coeffs):
        coeffs = Coeffs.from_triples(coeffs)
    d = _dtype_code(Y.dtype if dtype is None else dtype)
    if X.dtype != Y.dtype:
        raise ValueError("X and Y must have the same dtype")
    if X.numel() < plan.n or Y.numel() < plan.n:
        raise ValueError("X and Y must hold n = %d elements" % plan.n)
    st = lib().mpk_apply_final_noalloc(plan.handle, ctypes.byref(coeffs.struct), d, _ptr(X),
                                       _ptr(Y), int(flags), _stream_ptr(stream))
    _check(st, "mpk_apply_final_noalloc")


# ---------------------------------------------------------------------------------------------
# Host helpers
# ---------------------------------------------------------------------------------------------
def mpk_coeffs_chebyshev(alpha, beta, p) -> Coeffs:
    a, b, c = (np.zeros(p) for _ in range(3))
    _check(lib().mpk_coeffs_chebyshev(float(alpha), float(beta), int(p), a.ctypes.data,
                                      b.ctypes.data, c.ctypes.data), "mpk_coeffs_chebyshev")
    return Coeffs(a, b, c)


def mpk_coeffs_newton(theta) -> Coeffs:
    th = np.ascontiguousarray(theta, dtype=np.float64)
    p = th.shape[0]
    a, b, c = (np.zeros(p) for _ in range(3))
    _check(lib().mpk_coeffs_newton(th.ctypes.data, int(p), a.ctypes.data, b.ctypes.data,
                                   c.ctypes.data), "mpk_coeffs_newton")
    return Coeffs(a, b, c)


def mpk_leja_order(values, count) -> np.ndarray:
    v = np.ascontiguousarray(values, dtype=np.float64)
    out = np.zeros(count)
    _check(lib().mpk_leja_order(v.ctypes.data, int(v.shape[0]), int(count), out.ctypes.data),
           "mpk_leja_order")
    return out


def mpk_version() -> str:
    return lib().mpk_version().decode()


# ---------------------------------------------------------------------------------------------
# s-step GMRES
# ---------------------------------------------------------------------------------------------
def mpk_gmres_opts_default(**overrides) -> mpk_gmres_opts:
    o = mpk_gmres_opts()
    _check(lib().mpk_gmres_opts_default(ctypes.byref(o)), "mpk_gmres_opts_default")
    names = {f for f, _ in o._fields_}
    for k, v in overrides.items():
        if k not in names:
            raise TypeError("mpk_gmres_opts has no field %r" % k)
        setattr(o, k, v)
    return o


def sstep_gmres_solve(plan, b, x, opts=None, shifts=None, stream=None, check=True, trace=False):
    """Solve A x = b (b, x: CUDA float64 tensors in the original order).  Returns the info
    struct as a dict; raises on an error status unless check=False.  trace=True also returns
    the first s-step cycle's residual estimates ("trace_hist") and Arnoldi Hessenberg
    ("trace_H", (m+1) x m)."""
    o = opts if opts is not None else mpk_gmres_opts_default()
    keep = None
    if shifts is not None:
        keep = np.ascontiguousarray(shifts, dtype=np.float64)
        o.shifts = keep.ctypes.data
    th = tH = None
    if trace:
        m = int(o.restart)
        th = np.zeros(m)
        tH = np.zeros((m, m + 1))          # row c = column c of the (m+1) x m Hessenberg
        o.trace_hist = th.ctypes.data
        o.trace_cap = m
        o.trace_H = tH.ctypes.data
    info = mpk_gmres_info()
    st = lib().sstep_gmres_solve(plan.handle, _ptr(b), _ptr(x), ctypes.byref(o),
                                 ctypes.byref(info), _stream_ptr(stream))
    d = {f: getattr(info, f) for f, _ in info._fields_ if f not in ("shifts", "poly_interval")}
    d["poly_interval"] = (info.poly_interval[0], info.poly_interval[1])
    d["shifts"] = np.array(info.shifts[: o.s])
    d["status_code"] = int(st)
    if trace:
        d["trace_hist"] = th[: info.trace_len].copy()
        d["trace_H"] = tH.T.copy()
        o.trace_hist = None
        o.trace_H = None
        o.trace_cap = 0
    if check:
        _check(st, "sstep_gmres_solve")
    del keep
    return d


# ---------------------------------------------------------------------------------------------
# Autotuner
# ---------------------------------------------------------------------------------------------
def mpk_autotune(row_ptr, col, val, coeffs, n_rhs=1, flags=0, dtype=None, base=None, reps=5,
                 stream=None, check=True):
    """Time the candidate plan options for mpk_apply(coeffs, n_rhs, flags) on this matrix (see
    include/mpk.h); returns (best mpk_plan_opts, info dict)."""
    if not isinstance(coeffs, Coeffs):
        coeffs = Coeffs.from_triples(coeffs)
    A = _csr_struct(row_ptr, col, val)
    d = _dtype_code(val.dtype if dtype is None else dtype)
    best = mpk_plan_opts()
    info = mpk_tune_info()
    st = lib().mpk_autotune(ctypes.byref(A), coeffs.p, ctypes.byref(coeffs.struct), d, int(n_rhs),
                            int(flags), ctypes.byref(base) if base is not None else None, int(reps),
                            ctypes.byref(best), ctypes.byref(info), _stream_ptr(stream))
    out = {f: getattr(info, f) for f, _ in info._fields_}
    out["status_code"] = int(st)
    if check:
        _check(st, "mpk_autotune")
    return best, out


# ---------------------------------------------------------------------------------------------
# s-step CG
# ---------------------------------------------------------------------------------------------
def mpk_cg_opts_default(**overrides) -> mpk_cg_opts:
    o = mpk_cg_opts()
    _check(lib().mpk_cg_opts_default(ctypes.byref(o)), "mpk_cg_opts_default")
    names = {f for f, _ in o._fields_}
    for k, v in overrides.items():
        if k not in names:
            raise TypeError("mpk_cg_opts has no field %r" % k)
        setattr(o, k, v)
    return o


def sstep_cg_solve(plan, b, x, opts=None, shifts=None, stream=None, check=True):
    """Solve A x = b for an SPD A by s-step CG (b, x: CUDA float64 tensors in the original
    order).  Returns the info struct as a dict; raises on an error status unless check=False."""
    o = opts if opts is not None else mpk_cg_opts_default()
    keep = None
    if shifts is not None:
        keep = np.ascontiguousarray(shifts, dtype=np.float64)
        o.shifts = keep.ctypes.data
    info = mpk_cg_info()
    st = lib().sstep_cg_solve(plan.handle, _ptr(b), _ptr(x), ctypes.byref(o), ctypes.byref(info),
                              _stream_ptr(stream))
    d = {f: getattr(info, f) for f, _ in info._fields_ if f != "shifts"}
    d["shifts"] = np.array(info.shifts[: o.s])
    d["status_code"] = int(st)
    if check:
        _check(st, "sstep_cg_solve")
    del keep
    return d


# ---------------------------------------------------------------------------------------------
# Serving
# ---------------------------------------------------------------------------------------------
def mpk_server_opts_default(**overrides) -> mpk_server_opts:
    o = mpk_server_opts()
    _check(lib().mpk_server_opts_default(ctypes.byref(o)), "mpk_server_opts_default")
    names = {f for f, _ in o._fields_}
    for k, v in overrides.items():
        if k not in names:
            raise TypeError("mpk_server_opts has no field %r" % k)
        setattr(o, k, v)
    return o


class Server:
    def __init__(self, opts=None):
        o = opts if opts is not None else mpk_server_opts_default()
        h = ctypes.c_void_p(0)
        _check(lib().mpk_server_create(ctypes.byref(o), ctypes.byref(h)), "mpk_server_create")
        self.handle = h
        self._outputs = {}

    def submit(self, row_ptr, col, val, b):
        """Host numpy arrays (int32, int32, float64, float64).  Returns (id, x_out array)."""
        rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
        ci = np.ascontiguousarray(col, dtype=np.int32)
        vv = np.ascontiguousarray(val, dtype=np.float64)
        bb = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros(rp.shape[0] - 1)
        rid = ctypes.c_int64(0)
        st = lib().mpk_server_submit(self.handle, rp.shape[0] - 1, ci.shape[0], rp.ctypes.data,
                                     ci.ctypes.data, vv.ctypes.data, bb.ctypes.data, x.ctypes.data,
                                     ctypes.byref(rid))
        _check(st, "mpk_server_submit")
        self._outputs[rid.value] = x
        return rid.value, x

    def poll(self, max_results=64):
        buf = (mpk_server_result * max_results)()
        n = ctypes.c_int32(0)
        _check(lib().mpk_server_poll(self.handle, buf, max_results, ctypes.byref(n)), "mpk_server_poll")
        out = []
        for i in range(n.value):
            r = buf[i]
            out.append(dict(id=r.id, status=r.status, iters=r.iters, outer=r.outer,
                            rel_residual=r.rel_residual, t_submit_ms=r.t_submit_ms,
                            t_start_ms=r.t_start_ms, t_done_ms=r.t_done_ms,
                            x=self._outputs.pop(r.id, None)))
        return out

    def pending(self):
        n = ctypes.c_int64(0)
        _check(lib().mpk_server_pending(self.handle, ctypes.byref(n)), "mpk_server_pending")
        return n.value

    def close(self):
        if self.handle and self.handle.value:
            lib().mpk_server_destroy(self.handle)
            self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------------------------
# Orthogonalisation steps (the solvers' Gram and block-update kernels on caller blocks)
# ---------------------------------------------------------------------------------------------
def _colmajor(t, name):
    """(n, k) view of a column-major block given as a 2-D tensor of shape (k, ld) (row q is
    column q) - the layout the C ABI expects; returns (ld, k)."""
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError("%s: a contiguous (columns, ld) tensor is expected" % name)
    return t.stride(0), t.shape[0]


def mpk_gram(X, Y, n=None, stream=None):
    """G = X^T Y (FP64, K x S) for column blocks X (K, ldx) and Y (S, ldy) on the device, both
    float32 or both float64; the first n rows of each column are used (default: all)."""
    import torch
    if X.dtype != Y.dtype:
        raise ValueError("X and Y must have the same dtype")
    ldx, K = _colmajor(X, "X")
    ldy, S = _colmajor(Y, "Y")
    n = min(X.shape[1], Y.shape[1]) if n is None else int(n)
    if n > X.shape[1] or n > Y.shape[1]:
        raise ValueError("n exceeds the columns' length")
    G = torch.empty((S, K), dtype=torch.float64, device=X.device)   # row b = column b of G
    _check(lib().mpk_gram(_dtype_code(X.dtype), _ptr(X), ldx, K, _ptr(Y), ldy, S, n, _ptr(G),
                          _stream_ptr(stream)), "mpk_gram")
    return G.t()


def mpk_block_update(Q, W, C, Rinv, n=None, gram=True, stream=None):
    """W <- (W - Q C) Rinv in place (Q: (K1, ldq) or None, W: (S, ldw), C: (K1, S) FP64,
    Rinv: (S, S) FP64, upper triangle used); returns W^T W of the new W (FP64) or None."""
    import torch
    ldw, S = _colmajor(W, "W")
    K1, ldq = 0, 0
    if Q is not None:
        if Q.dtype != W.dtype:
            raise ValueError("Q and W must have the same dtype")
        ldq, K1 = _colmajor(Q, "Q")
    n = W.shape[1] if n is None else int(n)
    if n > W.shape[1] or (Q is not None and n > Q.shape[1]):
        raise ValueError("n exceeds the columns' length")
    Cd = None
    if K1:
        if tuple(C.shape) != (K1, S):
            raise ValueError("C must be K1 x S")
        Cd = C.to(W.device, torch.float64).t().contiguous()          # column-major K1 x S
    if tuple(Rinv.shape) != (S, S):
        raise ValueError("Rinv must be S x S")
    Rd = Rinv.to(W.device, torch.float64).t().contiguous()
    G = torch.empty((S, S), dtype=torch.float64, device=W.device) if gram else None
    _check(lib().mpk_block_update(_dtype_code(W.dtype), _ptr(Q), ldq, K1, _ptr(W), ldw, S, _ptr(Cd),
                                  _ptr(Rd), n, _ptr(G), _stream_ptr(stream)), "mpk_block_update")
    return G.t() if gram else None


def mpk_gram_pairs(Y, s, n, ldv, stream=None):
    """Gram of s-step CG's basis storage: Y a flat device tensor holding s + 1 pairs of 2 ldv
    values; returns the (2s + 2) x (2s + 2) FP64 matrix over the storage columns in pair order."""
    import torch
    if Y.numel() < (s + 1) * 2 * ldv:
        raise ValueError("Y holds fewer than s + 1 pairs of 2 ldv values")
    M = 2 * s + 2
    G = torch.empty((M, M), dtype=torch.float64, device=Y.device)
    _check(lib().mpk_gram_pairs(_dtype_code(Y.dtype), _ptr(Y), ldv, s, n, _ptr(G), _stream_ptr(stream)),
           "mpk_gram_pairs")
    return G.t()


def mpk_fma_peak(dtype, stream=None):
    """Measured FMA rate of the current device in TFLOP/s (MPK_F32 or MPK_F64)."""
    v = ctypes.c_double(0.0)
    _check(lib().mpk_fma_peak(int(dtype), ctypes.byref(v), _stream_ptr(stream)), "mpk_fma_peak")
    return v.value


def mpk_noalloc_forget():
    """Drop the scratch addresses mpk_apply_final_noalloc kept (after a device reset)."""
    _check(lib().mpk_noalloc_forget(), "mpk_noalloc_forget")


def mpk_hessenberg_eigvals(H, k=None):
    """Eigenvalues (complex numpy array) of the leading k x k block of the upper Hessenberg
    host matrix H (a 2-D numpy array), computed by the library's host QR iteration."""
    Hc = np.asfortranarray(np.asarray(H, dtype=np.float64))
    k = Hc.shape[1] if k is None else int(k)
    if Hc.shape[0] < k or Hc.shape[1] < k:
        raise ValueError("H is smaller than k x k")
    wr = np.zeros(k)
    wi = np.zeros(k)
    _check(lib().mpk_hessenberg_eigvals(Hc.ctypes.data, Hc.shape[0], k, wr.ctypes.data, wi.ctypes.data),
           "mpk_hessenberg_eigvals")
    return wr + 1j * wi


class Batch:
    """Batched MPK over several plans (mpk_batch_*): one persistent launch for all systems."""

    def __init__(self, plans, p, dtype, stream=None):
        import torch
        self.plans = list(plans)            # kept alive with the batch
        arr = (ctypes.c_void_p * len(self.plans))(*[pl.handle.value for pl in self.plans])
        h = ctypes.c_void_p()
        self.p = int(p)
        self.dtype = _dtype_code(dtype) if not isinstance(dtype, int) else dtype
        _check(lib().mpk_batch_create(arr, len(self.plans), self.p, self.dtype, _stream_ptr(stream),
                                      ctypes.byref(h)), "mpk_batch_create")
        self.handle = h

    def apply(self, coeffs, X, Y, flags=MPK_PERMUTED_IO, stream=None):
        """coeffs: one Coeffs (or triples) per system; X, Y: lists of CUDA tensors (X may be
        None with MPK_Y0_IS_X)."""
        cs = [c if isinstance(c, Coeffs) else Coeffs.from_triples(c) for c in coeffs]
        if len(cs) != len(self.plans) or len(Y) != len(self.plans):
            raise ValueError("one coefficient set and one output per system")
        for pl, y in zip(self.plans, Y):
            if y.numel() < (self.p + 1) * pl.n:
                raise ValueError("Y[i] must hold p + 1 blocks of n_i values")
        co = (mpk_coeffs * len(cs))(*[c.struct for c in cs])
        xs = (ctypes.c_void_p * len(cs))(*[(x.data_ptr() if x is not None else 0) for x in (X or [None] * len(cs))])
        ys = (ctypes.c_void_p * len(cs))(*[y.data_ptr() for y in Y])
        self._keep = (cs, co, xs, ys)
        _check(lib().mpk_batch_apply(self.handle, co, xs, ys, int(flags), _stream_ptr(stream)),
               "mpk_batch_apply")

    def sync(self, stream=None):
        return int(lib().mpk_batch_sync(self.handle, _stream_ptr(stream)))

    def __del__(self):
        try:
            if self.handle:
                lib().mpk_batch_destroy(self.handle)
                self.handle = None
        except Exception:
            pass
