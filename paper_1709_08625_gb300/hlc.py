"""Thin ctypes binding of the C ABI in include/hlc.h.

Argument marshalling only: every step of the computation runs in
``libhlc.so`` (CUDA, sm_103a).  Arrays may be numpy arrays (host) or CUDA
tensors (anything with ``data_ptr()``).  Importing this module loads the
library and fails loudly when it has not been built.
"""
from __future__ import annotations

import atexit
import ctypes
import os
import weakref

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhlc.so")

HLC_OK = 0
HLC_PENDING = 1
HLC_FP64 = 0
HLC_MIXED = 1
HLC_MIXED_SVD64 = 2
ERRORS = {
    -1: "HLC_ERR_ARG", -2: "HLC_ERR_OOM", -3: "HLC_ERR_NOT_SPD", -4: "HLC_ERR_TIMEOUT",
    -5: "HLC_ERR_CUDA", -6: "HLC_ERR_RANK", -7: "HLC_ERR_STATE", -8: "HLC_ERR_UNSUPPORTED",
    -9: "HLC_ERR_NUMERIC",
    -10: "HLC_ERR_SCRATCH",
}
for _code, _nm in ERRORS.items():
    globals()[_nm] = _code


class hlc_theta(ctypes.Structure):
    _fields_ = [("sigma2", ctypes.c_double), ("ell", ctypes.c_double), ("nu", ctypes.c_double),
                ("nugget", ctypes.c_double)]


class hlc_params(ctypes.Structure):
    _fields_ = [("leaf", ctypes.c_int), ("eta", ctypes.c_double), ("eps", ctypes.c_double),
                ("precision", ctypes.c_int), ("refine_tol", ctypes.c_double), ("refine_maxit", ctypes.c_int),
                ("kmax", ctypes.c_int)]


class hlc_result(ctypes.Structure):
    _fields_ = [("loglik", ctypes.c_double), ("logdet", ctypes.c_double), ("quad", ctypes.c_double),
                ("quad_factor", ctypes.c_double), ("refine_iters", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("bytes_C", ctypes.c_size_t), ("bytes_L", ctypes.c_size_t),
                ("max_rank_C", ctypes.c_int), ("max_rank_L", ctypes.c_int), ("ms_assemble", ctypes.c_double),
                ("ms_factor", ctypes.c_double), ("ms_solve", ctypes.c_double), ("ms_total", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class HlcError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__(f"{what}: {ERRORS.get(status, status)} ({_lib.hlc_strerror(status).decode()})")


_vp = ctypes.c_void_p
_i64 = ctypes.c_int64

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libhlc.so is not built ({LIB_PATH}); run __graft_entry__.build()")
_lib = ctypes.CDLL(LIB_PATH)

_SIGS = {
    "hlc_default_params": (None, [ctypes.POINTER(hlc_params)]),
    "hlc_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "hlc_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int]),
    "hlc_destroy": (None, [_vp]),
    "hlc_build_tree": (ctypes.c_int, [_vp, _vp, _i64, ctypes.POINTER(hlc_params), ctypes.POINTER(_vp)]),
    "hlc_tree_free": (None, [_vp]),
    "hlc_tree_info": (ctypes.c_int, [_vp, _vp]),
    "hlc_tree_perm": (ctypes.c_int, [_vp, _vp]),
    "hlc_tree_leaf_blocks": (ctypes.c_int, [_vp, _vp]),
    "hlc_assemble": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(hlc_theta), ctypes.POINTER(_vp)]),
    "hlc_cholesky": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(_vp)]),
    "hlc_matvec": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "hlc_matvec_noalloc": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "hlc_matvec_noalloc_capacity": (ctypes.c_int64, []),
    "hlc_selftest_barrier_timeout": (ctypes.c_int, [_vp]),
    "hlc_hmat_expand": (ctypes.c_int, [_vp, _vp, _vp]),
    "hlc_hmat_ranks": (ctypes.c_int, [_vp, _vp, _vp]),
    "hlc_hmat_free": (None, [_vp]),
    "hlc_loglik": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(hlc_theta), _vp, ctypes.POINTER(hlc_result)]),
    "hlc_ctx_stream": (ctypes.c_int, [_vp, ctypes.POINTER(_vp)]),
    "hlc_ctx_set_profiling": (ctypes.c_int, [_vp, ctypes.c_int]),
    "hlc_ctx_counters": (ctypes.c_int, [_vp, ctypes.c_int, _vp]),
    "hlc_serve_start": (ctypes.c_int, [_vp, ctypes.c_size_t, ctypes.c_int]),
    "hlc_serve_submit": (ctypes.c_int, [_vp, _vp, _vp, _i64, ctypes.POINTER(hlc_theta), ctypes.POINTER(hlc_params),
                                        ctypes.POINTER(ctypes.c_uint64)]),
    "hlc_serve_poll": (ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.POINTER(hlc_result)]),
    "hlc_serve_stop": (ctypes.c_int, [_vp]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args
    globals()[_name] = _f


def lib():
    return _lib


# Handles still alive at interpreter exit are released here, in dependency
# order, while the CUDA runtime is still loaded (object finalisers may run
# after it has been torn down).
_LIVE = {"trees": weakref.WeakSet(), "mats": weakref.WeakSet(), "ctxs": weakref.WeakSet()}


@atexit.register
def _release_all():
    for kind, meth in (("mats", "free"), ("trees", "free"), ("ctxs", "close")):
        for obj in list(_LIVE[kind]):
            try:
                getattr(obj, meth)()
            except Exception:
                pass


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return ctypes.c_void_p(a.ctypes.data)


def _check(st, what):
    if st != HLC_OK:
        raise HlcError(st, what)


def params(leaf=64, eta=2.0, eps=1e-6, precision=HLC_FP64, refine_tol=1e-12, refine_maxit=100, kmax=64):
    p = hlc_params()
    hlc_default_params(ctypes.byref(p))
    p.leaf, p.eta, p.eps, p.precision = int(leaf), float(eta), float(eps), int(precision)
    p.refine_tol, p.refine_maxit, p.kmax = float(refine_tol), int(refine_maxit), int(kmax)
    return p


def theta(sigma2, ell, nu, nugget):
    return hlc_theta(float(sigma2), float(ell), float(nu), float(nugget))


class Context:
    """hlc_create / hlc_destroy."""

    def __init__(self, device=0):
        h = _vp()
        _check(hlc_create(ctypes.byref(h), int(device)), "hlc_create")
        self.h = h
        _LIVE["ctxs"].add(self)

    def close(self):
        if getattr(self, "h", None):
            hlc_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def build_tree(self, xy, **kw):
        return Tree(self, xy, **kw)

    def stream(self):
        """The context's cudaStream_t as an integer handle."""
        p = _vp()
        _check(hlc_ctx_stream(self.h, ctypes.byref(p)), "hlc_ctx_stream")
        return p.value or 0

    def set_profiling(self, on=True):
        _check(hlc_ctx_set_profiling(self.h, int(bool(on))), "hlc_ctx_set_profiling")

    OPS = ("potrf", "trsm", "gemm", "trunc", "trunc_cluster")

    # ---- serving -------------------------------------------------------
    def serve_start(self, hbm_budget_bytes, max_slots):
        _check(hlc_serve_start(self.h, int(hbm_budget_bytes), int(max_slots)), "hlc_serve_start")

    def serve_submit(self, xy, z, th, **kw):
        xy = np.ascontiguousarray(xy, dtype=np.float64)
        z = np.ascontiguousarray(z, dtype=np.float64)
        p = params(**kw)
        rid = ctypes.c_uint64()
        _check(hlc_serve_submit(self.h, _ptr(xy), _ptr(z), xy.shape[0], ctypes.byref(th), ctypes.byref(p),
                                ctypes.byref(rid)), "hlc_serve_submit")
        return rid.value

    def serve_poll(self, rid):
        """None while pending, else the result dict (raises on a failed request)."""
        r = hlc_result()
        st = hlc_serve_poll(self.h, ctypes.c_uint64(rid), ctypes.byref(r))
        if st == HLC_PENDING:
            return None
        _check(st, "hlc_serve_poll")
        return r.as_dict()

    def serve_stop(self):
        _check(hlc_serve_stop(self.h), "hlc_serve_stop")

    def counters(self, reset=False):
        a = np.zeros(17)
        _check(hlc_ctx_counters(self.h, int(bool(reset)), _ptr(a)), "hlc_ctx_counters")
        out = {"launches": int(a[0])}
        for i, name in enumerate(self.OPS):
            out[name] = {"launches": int(a[1 + 3 * i]), "ms": float(a[2 + 3 * i]), "flops": float(a[3 + 3 * i])}
        out["persistent"] = int(a[16])
        return out


class HMat:
    def __init__(self, ctx, tree, h):
        self.ctx, self.tree, self.h = ctx, tree, h
        _LIVE["mats"].add(self)

    def free(self):
        if getattr(self, "h", None):
            hlc_hmat_free(self.h)
            self.h = None

    def __del__(self):
        self.free()

    def expand(self):
        n = self.tree.n
        out = np.zeros((n, n), order="F")
        _check(hlc_hmat_expand(self.ctx.h, self.h, _ptr(out)), "hlc_hmat_expand")
        return out

    def ranks(self):
        out = np.zeros(self.tree.nleaves, dtype=np.int32)
        _check(hlc_hmat_ranks(self.ctx.h, self.h, _ptr(out)), "hlc_hmat_ranks")
        return out

    def matvec(self, x, y=None):
        if y is None:
            x = np.ascontiguousarray(x, dtype=np.float64)
            y = np.empty_like(x)
        _check(hlc_matvec(self.ctx.h, self.h, _ptr(x), _ptr(y)), "hlc_matvec")
        return y

    def matvec_noalloc(self, x, y):
        """y = C~ x into the caller's device tensor y (x, y on the device)."""
        _check(hlc_matvec_noalloc(self.ctx.h, self.h, _ptr(x), _ptr(y)), "hlc_matvec_noalloc")
        return y


class Tree:
    """hlc_build_tree and the calls on a tree."""

    def __init__(self, ctx, xy, leaf=64, eta=2.0, eps=1e-6, precision=HLC_FP64, refine_tol=1e-12,
                 refine_maxit=100, kmax=64):
        self.ctx = ctx
        if not hasattr(xy, "data_ptr"):
            xy = np.ascontiguousarray(xy, dtype=np.float64)
        self._xy = xy
        self.n = int(xy.shape[0])
        self.p = params(leaf, eta, eps, precision, refine_tol, refine_maxit, kmax)
        h = _vp()
        _check(hlc_build_tree(ctx.h, _ptr(xy), self.n, ctypes.byref(self.p), ctypes.byref(h)), "hlc_build_tree")
        self.h = h
        _LIVE["trees"].add(self)
        info = self.info()
        self.nleaves = info["dense"] + info["lowrank"]

    def free(self):
        if getattr(self, "h", None):
            hlc_tree_free(self.h)
            self.h = None

    def __del__(self):
        self.free()

    def info(self):
        a = np.zeros(8, dtype=np.int64)
        _check(hlc_tree_info(self.h, _ptr(a)), "hlc_tree_info")
        return dict(n=int(a[0]), clusters=int(a[1]), leaf_clusters=int(a[2]), dense=int(a[3]),
                    lowrank=int(a[4]), depth=int(a[5]), plan_ops=int(a[6]), plan_waves=int(a[7]))

    def perm(self):
        p = np.zeros(self.n, dtype=np.int32)
        _check(hlc_tree_perm(self.h, _ptr(p)), "hlc_tree_perm")
        return p

    def leaf_blocks(self):
        out = np.zeros((self.nleaves, 5), dtype=np.int64)
        _check(hlc_tree_leaf_blocks(self.h, _ptr(out)), "hlc_tree_leaf_blocks")
        return out

    def assemble(self, th):
        h = _vp()
        _check(hlc_assemble(self.ctx.h, self.h, ctypes.byref(th), ctypes.byref(h)), "hlc_assemble")
        return HMat(self.ctx, self, h)

    def cholesky(self, C):
        h = _vp()
        _check(hlc_cholesky(self.ctx.h, C.h, ctypes.byref(h)), "hlc_cholesky")
        return HMat(self.ctx, self, h)

    def loglik(self, th, z):
        if not hasattr(z, "data_ptr"):
            z = np.ascontiguousarray(z, dtype=np.float64)
        r = hlc_result()
        _check(hlc_loglik(self.ctx.h, self.h, ctypes.byref(th), _ptr(z), ctypes.byref(r)), "hlc_loglik")
        return r.as_dict()
