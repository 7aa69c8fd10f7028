"""CPU oracle for the H-matrix Gaussian log-likelihood -- TEST INFRASTRUCTURE.

Plain FP64 C++ (``hlc_oracle.cpp``) written from arXiv:1709.08625 and loaded
through ctypes.  Only the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package; the product path never
does.  It shares no code with the CUDA library.

Passages followed (see the C++ file for the per-function citations):
eq. (1) dense likelihood, eq. (2) H-likelihood from the H-Cholesky factor,
eq. (3) Matern covariance, eq. (4)/Sec. 4.1 nugget, Sec. 2.2 + App. A cluster
tree, block-cluster tree and standard admissibility, App. B ACA and the
preconditioned solve, Remark A.1 QR+SVD recompression.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hlc_oracle.cpp")
_LIB = os.path.join(_HERE, "_hlc_oracle.so")

_dp = ctypes.POINTER(ctypes.c_double)
_lp = ctypes.POINTER(ctypes.c_long)
_ip = ctypes.POINTER(ctypes.c_int)

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (g++, OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
               _SRC, "-o", _LIB + ".tmp"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.orc_matern.argtypes = [_dp, ctypes.c_long, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_int, _dp]
        L.orc_dense_cov.argtypes = [_dp, _dp, ctypes.c_long] + [ctypes.c_double] * 4 + [_dp]
        L.orc_dense_cholesky.argtypes = [_dp, ctypes.c_long]
        L.orc_dense_cholesky.restype = ctypes.c_long
        L.orc_dense_loglik.argtypes = [_dp, _dp, _dp, ctypes.c_long] + [ctypes.c_double] * 4 + [_dp]
        L.orc_dense_loglik.restype = ctypes.c_long
        L.orc_dense_chol_apply.argtypes = [_dp, _dp, _dp, ctypes.c_long] + [ctypes.c_double] * 4 + [_dp]
        L.orc_dense_chol_apply.restype = ctypes.c_long
        L.orc_h_create.argtypes = [_dp, _dp, ctypes.c_long, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                   ctypes.c_int]
        L.orc_h_create.restype = ctypes.c_void_p
        L.orc_h_free.argtypes = [ctypes.c_void_p]
        L.orc_h_info.argtypes = [ctypes.c_void_p, _lp]
        L.orc_h_perm.argtypes = [ctypes.c_void_p, _ip]
        L.orc_h_clusters.argtypes = [ctypes.c_void_p, _lp, _dp, _ip, _ip]
        L.orc_h_clusters.restype = ctypes.c_long
        L.orc_h_leaf_blocks.argtypes = [ctypes.c_void_p, _lp]
        L.orc_h_leaf_blocks.restype = ctypes.c_long
        L.orc_h_assemble.argtypes = [ctypes.c_void_p] + [ctypes.c_double] * 5 + [ctypes.c_long]
        L.orc_h_cholesky.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_int]
        L.orc_h_cholesky.restype = ctypes.c_long
        L.orc_h_stats.argtypes = [ctypes.c_void_p, _lp]
        L.orc_h_ranks.argtypes = [ctypes.c_void_p, ctypes.c_int, _ip]
        L.orc_h_ranks.restype = ctypes.c_long
        L.orc_h_matvec.argtypes = [ctypes.c_void_p, _dp, _dp]
        L.orc_h_expand.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp]
        L.orc_h_lmatvec.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp, _dp]
        L.orc_h_loglik.argtypes = [ctypes.c_void_p, _dp, ctypes.c_double, ctypes.c_int, _dp]
        L.orc_h_aca_block.argtypes = [ctypes.c_void_p, ctypes.c_long, ctypes.c_long, ctypes.c_long,
                                      ctypes.c_long, ctypes.c_double, ctypes.c_long, _dp, _dp, ctypes.c_int]
        L.orc_h_aca_block.restype = ctypes.c_long
        L.orc_truncate.argtypes = [_dp, ctypes.c_long, _dp, ctypes.c_long, ctypes.c_long, ctypes.c_double]
        L.orc_truncate.restype = ctypes.c_long
        L.orc_h_set_theta.argtypes = [ctypes.c_void_p] + [ctypes.c_double] * 4
        L.orc_h_set_fixed_rank.argtypes = [ctypes.c_void_p, ctypes.c_long]
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def matern(h, sigma2, ell, nu, use_bessel=False):
    """Matern covariance, eq. (3), at distances h."""
    h = np.ascontiguousarray(h, dtype=np.float64).ravel()
    out = np.empty_like(h)
    st = lib().orc_matern(_d(h), h.size, sigma2, ell, nu, int(use_bessel), _d(out))
    if st != 0:
        raise ValueError("orc_matern: bad argument")
    return out


def dense_cov(xy, sigma2, ell, nu, nugget):
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    x = np.ascontiguousarray(xy[:, 0])
    y = np.ascontiguousarray(xy[:, 1])
    n = x.size
    C = np.empty((n, n), dtype=np.float64, order="F")
    st = lib().orc_dense_cov(_d(x), _d(y), n, sigma2, ell, nu, nugget, _d(C))
    if st != 0:
        raise ValueError("orc_dense_cov: bad argument")
    return C


def dense_cholesky(A):
    """Lower Cholesky factor of a symmetric matrix (hand-written, blocked)."""
    W = np.array(A, dtype=np.float64, order="F", copy=True)
    st = lib().orc_dense_cholesky(W.ctypes.data_as(_dp), W.shape[0])
    if st != 0:
        raise np.linalg.LinAlgError(f"not positive definite at pivot {-st - 1}")
    return np.tril(W)


def dense_loglik(xy, z, sigma2, ell, nu, nugget):
    """eq. (1) with a dense FP64 Cholesky: returns (loglik, logdet, quad)."""
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    x = np.ascontiguousarray(xy[:, 0])
    y = np.ascontiguousarray(xy[:, 1])
    z = np.ascontiguousarray(z, dtype=np.float64)
    out = np.zeros(3)
    st = lib().orc_dense_loglik(_d(x), _d(y), _d(z), x.size, sigma2, ell, nu, nugget, _d(out))
    if st == -2:
        raise np.linalg.LinAlgError("covariance not positive definite")
    if st != 0:
        raise ValueError("orc_dense_loglik: bad argument")
    return float(out[0]), float(out[1]), float(out[2])


def dense_chol_apply(xy, xi, sigma2, ell, nu, nugget):
    """z = L xi with C = L L^T (dense FP64)."""
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    x = np.ascontiguousarray(xy[:, 0])
    y = np.ascontiguousarray(xy[:, 1])
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    z = np.empty_like(xi)
    st = lib().orc_dense_chol_apply(_d(x), _d(y), _d(xi), x.size, sigma2, ell, nu, nugget, _d(z))
    if st != 0:
        raise np.linalg.LinAlgError("dense_chol_apply failed")
    return z


def truncate(U, V, eps):
    """Recompression of U V^T (Remark A.1); returns (U_k, V_k)."""
    U = np.array(U, dtype=np.float64, order="F", copy=True)
    V = np.array(V, dtype=np.float64, order="F", copy=True)
    m, K = U.shape
    n = V.shape[0]
    k = lib().orc_truncate(U.ctypes.data_as(_dp), m, V.ctypes.data_as(_dp), n, K, eps)
    Uk = U.ravel(order="F")[: m * k].reshape((m, k), order="F")
    Vk = V.ravel(order="F")[: n * k].reshape((n, k), order="F")
    return Uk, Vk


class HOracle:
    """Plain CPU H-matrix path: tree, assembly, H-Cholesky, likelihood."""

    def __init__(self, xy, leaf=32, eta=2.0, admissibility=0, split=0, fixed_rank=0):
        """admissibility: 0 standard min(diam) <= eta dist, 1 max(diam), 2 weak;
        split: 0 geometric midpoint, 1 cardinality (median); fixed_rank: 0
        adaptive, k > 0 at most k columns per low-rank block."""
        xy = np.ascontiguousarray(xy, dtype=np.float64)
        self._x = np.ascontiguousarray(xy[:, 0])
        self._y = np.ascontiguousarray(xy[:, 1])
        self.n = self._x.size
        self.h = lib().orc_h_create(_d(self._x), _d(self._y), self.n, int(leaf), float(eta), int(admissibility),
                                    int(split))
        if not self.h:
            raise ValueError("orc_h_create: bad argument")
        if fixed_rank:
            lib().orc_h_set_fixed_rank(self.h, int(fixed_rank))

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_h_free(self.h)
            self.h = None

    def info(self):
        a = np.zeros(6, dtype=np.int64)
        lib().orc_h_info(self.h, a.ctypes.data_as(_lp))
        return dict(n=int(a[0]), clusters=int(a[1]), leaf_clusters=int(a[2]), dense=int(a[3]),
                    lowrank=int(a[4]), depth=int(a[5]))

    def perm(self):
        p = np.zeros(self.n, dtype=np.int32)
        lib().orc_h_perm(self.h, p.ctypes.data_as(_ip))
        return p

    def clusters(self):
        nc = self.info()["clusters"]
        lohi = np.zeros((nc, 2), dtype=np.int64)
        bbox = np.zeros((nc, 4))
        lev = np.zeros(nc, dtype=np.int32)
        leaf = np.zeros(nc, dtype=np.int32)
        lib().orc_h_clusters(self.h, lohi.ctypes.data_as(_lp), _d(bbox), lev.ctypes.data_as(_ip),
                             leaf.ctypes.data_as(_ip))
        return lohi, bbox, lev, leaf

    def leaf_blocks(self):
        inf = self.info()
        nb = inf["dense"] + inf["lowrank"]
        out = np.zeros((nb, 5), dtype=np.int64)
        lib().orc_h_leaf_blocks(self.h, out.ctypes.data_as(_lp))
        return out

    def assemble(self, sigma2, ell, nu, nugget, eps, kmax=4096):
        st = lib().orc_h_assemble(self.h, sigma2, ell, nu, nugget, eps, int(kmax))
        if st != 0:
            raise ValueError("orc_h_assemble failed")
        self.eps = eps

    def cholesky(self, eps=None, accumulate=False):
        st = lib().orc_h_cholesky(self.h, float(self.eps if eps is None else eps), int(bool(accumulate)))
        if st == -2:
            raise np.linalg.LinAlgError("H-Cholesky: not positive definite")
        if st != 0:
            raise RuntimeError("orc_h_cholesky failed")

    def stats(self):
        a = np.zeros(4, dtype=np.int64)
        lib().orc_h_stats(self.h, a.ctypes.data_as(_lp))
        return dict(max_rank_C=int(a[0]), entries_C=int(a[1]), max_rank_L=int(a[2]), entries_L=int(a[3]))

    def ranks(self, which=0):
        nb = len(self.leaf_blocks())
        out = np.zeros(nb, dtype=np.int32)
        lib().orc_h_ranks(self.h, int(which), out.ctypes.data_as(_ip))
        return out

    def matvec(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.zeros_like(x)
        if lib().orc_h_matvec(self.h, _d(x), _d(y)) != 0:
            raise RuntimeError("not assembled")
        return y

    def lmatvec(self, x, trans=False):
        """L~ x (or L~^T x) with the H-Cholesky factor, user order."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.zeros_like(x)
        if lib().orc_h_lmatvec(self.h, int(bool(trans)), _d(x), _d(y)) != 0:
            raise RuntimeError("not factored")
        return y

    def expand(self, which=0):
        out = np.zeros((self.n, self.n), order="F")
        if lib().orc_h_expand(self.h, int(which), out.ctypes.data_as(_dp)) != 0:
            raise RuntimeError("not assembled / factored")
        return out

    def loglik(self, z, tol=1e-12, maxit=100):
        z = np.ascontiguousarray(z, dtype=np.float64)
        out = np.zeros(6)
        if lib().orc_h_loglik(self.h, _d(z), float(tol), int(maxit), _d(out)) != 0:
            raise RuntimeError("not factored")
        return dict(loglik=out[0], logdet=out[1], quad=out[2], quad_factor=out[3],
                    refine_iters=int(out[4]), rel_residual=out[5])

    def set_theta(self, sigma2, ell, nu, nugget):
        lib().orc_h_set_theta(self.h, sigma2, ell, nu, nugget)

    def aca_block(self, r0, m, c0, n, eps, kmax=4096, recompress=True):
        U = np.zeros((m, min(m, n, kmax)), order="F")
        V = np.zeros((n, min(m, n, kmax)), order="F")
        k = lib().orc_h_aca_block(self.h, r0, m, c0, n, eps, kmax, U.ctypes.data_as(_dp),
                                  V.ctypes.data_as(_dp), int(recompress))
        Uk = U.ravel(order="F")[: m * k].reshape((m, k), order="F")
        Vk = V.ravel(order="F")[: n * k].reshape((n, k), order="F")
        return Uk, Vk


def h_loglik(xy, z, sigma2, ell, nu, nugget, eps, leaf=32, eta=2.0, tol=1e-12, maxit=100, accumulate=False,
             admissibility=0, split=0, fixed_rank=0):
    """One oracle evaluation: tree, assembly, H-Cholesky, eq. (2) + preconditioned CG."""
    H = HOracle(xy, leaf=leaf, eta=eta, admissibility=admissibility, split=split, fixed_rank=fixed_rank)
    H.assemble(sigma2, ell, nu, nugget, eps)
    H.cholesky(eps, accumulate=accumulate)
    r = H.loglik(z, tol=tol, maxit=maxit)
    r.update(H.stats())
    return r
