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


HLC_ADM_STANDARD, HLC_ADM_MAXDIAM, HLC_ADM_WEAK = 0, 1, 2
HLC_SPLIT_GEOMETRIC, HLC_SPLIT_CARDINALITY = 0, 1


class hlc_params(ctypes.Structure):
    _fields_ = [("leaf", ctypes.c_int), ("eta", ctypes.c_double), ("eps", ctypes.c_double),
                ("precision", ctypes.c_int), ("refine_tol", ctypes.c_double), ("refine_maxit", ctypes.c_int),
                ("kmax", ctypes.c_int), ("admissibility", ctypes.c_int), ("split", ctypes.c_int),
                ("fixed_rank", ctypes.c_int)]


class hlc_result(ctypes.Structure):
    _fields_ = [("loglik", ctypes.c_double), ("logdet", ctypes.c_double), ("quad", ctypes.c_double),
                ("quad_factor", ctypes.c_double), ("refine_iters", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("est_rel_err", ctypes.c_double),
                ("bytes_C", ctypes.c_size_t), ("bytes_L", ctypes.c_size_t),
                ("max_rank_C", ctypes.c_int), ("max_rank_L", ctypes.c_int), ("ms_assemble", ctypes.c_double),
                ("ms_factor", ctypes.c_double), ("ms_solve", ctypes.c_double), ("ms_total", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class hlc_fit_opts(ctypes.Structure):
    _fields_ = [("step", ctypes.c_double * 3), ("size_tol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("free_mask", ctypes.c_int)]


class hlc_fit_result(ctypes.Structure):
    _fields_ = [("theta", hlc_theta), ("loglik", ctypes.c_double), ("iterations", ctypes.c_int),
                ("evaluations", ctypes.c_int), ("failed_evals", ctypes.c_int), ("converged", ctypes.c_int),
                ("traced", ctypes.c_int), ("ms_total", ctypes.c_double)]


OBJECTIVE = ctypes.CFUNCTYPE(ctypes.c_double, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p)


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
    "hlc_selftest_plans": (ctypes.c_int, [_i64, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_uint64, _vp, ctypes.c_int, ctypes.c_char_p,
                                          ctypes.c_int]),
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
    "hlc_serve_footprint": (ctypes.c_size_t, [_i64, ctypes.POINTER(hlc_params)]),
    "hlc_serve_admission_replay": (ctypes.c_int, [ctypes.c_size_t, ctypes.c_int, _i64, _vp, _vp, _vp,
                                                  ctypes.POINTER(ctypes.c_size_t)]),
    "hlc_tree_memory": (ctypes.c_int, [_vp, _vp]),
    "hlc_factor_apply": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp, _vp]),
    "hlc_nelder_mead": (ctypes.c_int, [ctypes.c_int, _vp, _vp, ctypes.c_double, ctypes.c_int, OBJECTIVE, _vp, _vp,
                                       _vp]),
    "hlc_default_fit_opts": (None, [ctypes.POINTER(hlc_fit_opts)]),
    "hlc_fit": (ctypes.c_int, [_vp, _vp, _vp, ctypes.POINTER(hlc_theta), ctypes.POINTER(hlc_fit_opts), _vp,
                               ctypes.c_int, ctypes.POINTER(hlc_fit_result)]),
    "hlc_sample": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(hlc_theta), _vp, _vp]),
    "hlc_diagnostics": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(hlc_theta), ctypes.c_int, ctypes.c_int,
                                       ctypes.c_uint64, _vp]),
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


def params(leaf=64, eta=2.0, eps=1e-6, precision=HLC_FP64, refine_tol=1e-12, refine_maxit=100, kmax=64,
           admissibility=HLC_ADM_STANDARD, split=HLC_SPLIT_GEOMETRIC, fixed_rank=0):
    p = hlc_params()
    hlc_default_params(ctypes.byref(p))
    p.leaf, p.eta, p.eps, p.precision = int(leaf), float(eta), float(eps), int(precision)
    p.refine_tol, p.refine_maxit, p.kmax = float(refine_tol), int(refine_maxit), int(kmax)
    p.admissibility, p.split, p.fixed_rank = int(admissibility), int(split), int(fixed_rank)
    return p


def theta(sigma2, ell, nu, nugget):
    return hlc_theta(float(sigma2), float(ell), float(nu), float(nugget))


def nelder_mead(f, x0, step, size_tol=1e-5, max_iter=200):
    """hlc_nelder_mead with a Python objective f(x: ndarray) -> float;
    returns (x, fmin, iterations)."""
    x = np.array(x0, dtype=np.float64)
    st = np.ascontiguousarray(step, dtype=np.float64)
    d = x.size

    def cb(p, _):
        return float(f(np.ctypeslib.as_array(p, shape=(d,)).copy()))

    c = OBJECTIVE(cb)
    fmin = ctypes.c_double()
    it = ctypes.c_int()
    _check(hlc_nelder_mead(d, _ptr(x), _ptr(st), float(size_tol), int(max_iter), c, None, ctypes.byref(fmin),
                           ctypes.byref(it)), "hlc_nelder_mead")
    return x, fmin.value, it.value


def fit_opts(step=None, size_tol=None, max_iter=None, free_mask=None):
    o = hlc_fit_opts()
    hlc_default_fit_opts(ctypes.byref(o))
    if step is not None:
        for i in range(3):
            o.step[i] = float(step[i])
    if size_tol is not None:
        o.size_tol = float(size_tol)
    if max_iter is not None:
        o.max_iter = int(max_iter)
    if free_mask is not None:
        o.free_mask = int(free_mask)
    return o


SELFTEST_PLAN_STATS = ("factor_ops", "factor_edges", "groups", "ready0", "fwd_ops", "fwd_joins", "bwd_ops",
                       "bwd_joins", "mv_ops", "model_makespan", "leaves", "rank_slots", "plan_ms", "factor_hash",
                       "solve_hash")


def selftest_plans(n, leaf=32, eta=2.0, kmax=64, ctas=16, seed=1, geometry=1):
    """hlc_selftest_plans (host only): the planner's dataflow invariants on a
    synthetic tree over [0, n) (geometry 1: a Morton-numbered grid, 0:
    intervals).  Returns (status, message, stats dict)."""
    stats = np.zeros(15, dtype=np.int64)
    msg = ctypes.create_string_buffer(512)
    st = hlc_selftest_plans(int(n), int(leaf), float(eta), int(geometry), int(kmax), int(ctas), int(seed),
                            _ptr(stats), 15, msg, 512)
    return st, msg.value.decode(), dict(zip(SELFTEST_PLAN_STATS, (int(v) for v in stats)))


def serve_footprint(n, **kw):
    """Bytes the request loop charges for one request of n points."""
    p = params(**kw)
    return int(hlc_serve_footprint(int(n), ctypes.byref(p)))


def admission_replay(budget, max_slots, footprints, durations):
    """Host-only replay of the serve loop's admission rule: returns the
    admission times of the requests (queued at time 0 in order) and the
    peak sum of footprints running at once."""
    fp = np.ascontiguousarray(footprints, dtype=np.uint64)
    du = np.ascontiguousarray(durations, dtype=np.float64)
    start = np.zeros(fp.size)
    peak = ctypes.c_size_t()
    _check(hlc_serve_admission_replay(int(budget), int(max_slots), fp.size, _ptr(fp), _ptr(du), _ptr(start),
                                      ctypes.byref(peak)), "hlc_serve_admission_replay")
    return start, int(peak.value)


class Context:
    """hlc_create / hlc_destroy."""

    def __init__(self, device=0):
        h = _vp()
        _check(hlc_create(ctypes.byref(h), int(device)), "hlc_create")
        self.h = h
        self._children = weakref.WeakSet()  # trees and matrices made on this context
        _LIVE["ctxs"].add(self)

    def close(self):
        """Destroy the context, after freeing the trees and matrices made on
        it (the C ABI requires them to go first)."""
        if getattr(self, "h", None):
            kids = list(getattr(self, "_children", ()))
            for obj in kids:
                if isinstance(obj, HMat):
                    obj.free()
            for obj in kids:
                if isinstance(obj, Tree):
                    obj.free()
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

    OPS = ("potrf", "trsm", "gemm", "trunc", "trunc_cluster", "chain")

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
        a = np.zeros(20)
        _check(hlc_ctx_counters(self.h, int(bool(reset)), _ptr(a)), "hlc_ctx_counters")
        out = {"launches": int(a[0])}
        for i, name in enumerate(self.OPS):
            out[name] = {"launches": int(a[1 + 3 * i]), "ms": float(a[2 + 3 * i]), "flops": float(a[3 + 3 * i])}
        out["persistent"] = int(a[19])
        return out


class HMat:
    def __init__(self, ctx, tree, h):
        self.ctx, self.tree, self.h = ctx, tree, h
        _LIVE["mats"].add(self)
        ctx._children.add(self)

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

    def factor_apply(self, x, trans=False, y=None):
        """y = L~ x (or L~^T x) with this factor (from Tree.cholesky)."""
        if y is None:
            x = np.ascontiguousarray(x, dtype=np.float64)
            y = np.empty_like(x)
        _check(hlc_factor_apply(self.ctx.h, self.h, int(bool(trans)), _ptr(x), _ptr(y)), "hlc_factor_apply")
        return y

    def matvec_noalloc(self, x, y):
        """y = C~ x into the caller's device tensor y (x, y on the device)."""
        _check(hlc_matvec_noalloc(self.ctx.h, self.h, _ptr(x), _ptr(y)), "hlc_matvec_noalloc")
        return y


class Tree:
    """hlc_build_tree and the calls on a tree."""

    def __init__(self, ctx, xy, leaf=64, eta=2.0, eps=1e-6, precision=HLC_FP64, refine_tol=1e-12,
                 refine_maxit=100, kmax=64, admissibility=HLC_ADM_STANDARD, split=HLC_SPLIT_GEOMETRIC,
                 fixed_rank=0):
        self.ctx = ctx
        if not hasattr(xy, "data_ptr"):
            xy = np.ascontiguousarray(xy, dtype=np.float64)
        self._xy = xy
        self.n = int(xy.shape[0])
        self.p = params(leaf, eta, eps, precision, refine_tol, refine_maxit, kmax, admissibility, split,
                        fixed_rank)
        h = _vp()
        _check(hlc_build_tree(ctx.h, _ptr(xy), self.n, ctypes.byref(self.p), ctypes.byref(h)), "hlc_build_tree")
        self.h = h
        _LIVE["trees"].add(self)
        ctx._children.add(self)
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

    def memory(self):
        a = np.zeros(6, dtype=np.int64)
        _check(hlc_tree_memory(self.h, _ptr(a)), "hlc_tree_memory")
        return dict(arena=int(a[0]), matrices=int(a[1]), tmp=int(a[2]), vectors=int(a[3]), plans=int(a[4]),
                    total=int(a[5]))

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

    def sample(self, th, xi, z=None):
        """z = L~(theta) xi, synthetic data from the H-Cholesky factor (Sec. 5.1)."""
        if not hasattr(xi, "data_ptr"):
            xi = np.ascontiguousarray(xi, dtype=np.float64)
        if z is None:
            z = np.empty(self.n) if not hasattr(xi, "data_ptr") else xi.new_empty(self.n)
        _check(hlc_sample(self.ctx.h, self.h, ctypes.byref(th), _ptr(xi), _ptr(z)), "hlc_sample")
        return z

    def fit(self, z, start, trace_cap=0, **opts):
        """Nelder-Mead identification of (nu, ell, sigma2) (hlc_fit); returns
        (result dict, trace array of {nu, ell, sigma2, loglik, status} rows)."""
        if not hasattr(z, "data_ptr"):
            z = np.ascontiguousarray(z, dtype=np.float64)
        o = fit_opts(**opts)
        tr = np.zeros((max(trace_cap, 0), 5))
        r = hlc_fit_result()
        _check(hlc_fit(self.ctx.h, self.h, _ptr(z), ctypes.byref(start), ctypes.byref(o),
                       _ptr(tr) if trace_cap > 0 else None, int(trace_cap), ctypes.byref(r)), "hlc_fit")
        out = {k: getattr(r, k) for k, _ in r._fields_ if k != "theta"}
        out.update(sigma2=r.theta.sigma2, ell=r.theta.ell, nu=r.theta.nu, nugget=r.theta.nugget)
        return out, tr[: r.traced]

    def diagnostics(self, th, iters=20, probes=16, seed=1):
        """hlc_diagnostics: dict of the norm and KLD estimates (-1: not computed)."""
        a = np.zeros(6)
        _check(hlc_diagnostics(self.ctx.h, self.h, ctypes.byref(th), int(iters), int(probes), int(seed), _ptr(a)),
               "hlc_diagnostics")
        return dict(err_C=a[0], norm_C=a[1], err_LLt=a[2], inv_err=a[3], kld=a[4], norm_Ch=a[5])

    def loglik(self, th, z):
        if not hasattr(z, "data_ptr"):
            z = np.ascontiguousarray(z, dtype=np.float64)
        r = hlc_result()
        _check(hlc_loglik(self.ctx.h, self.h, ctypes.byref(th), _ptr(z), ctypes.byref(r)), "hlc_loglik")
        return r.as_dict()
