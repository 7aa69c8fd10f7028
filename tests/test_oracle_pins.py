"""Pins of the CPU oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: closed
forms of eq. (3), library / arbitrary-precision Bessel values, brute-force
determinants, the Eckart-Young optimality of the recompression (Remark A.1),
exact invariants of eq. (1), and the partition properties of the cluster and
block-cluster trees (Sec. 2.2, App. A).
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1709_08625_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------
# Matern covariance, eq. (3)
# ----------------------------------------------------------------------------
H = np.array([0.0, 1e-9, 1e-4, 0.01, 0.05, 0.1, 0.3, 1.0, 3.0, 20.0])


def test_matern_half_integer_closed_forms():
    # nu = 1/2 -> sigma2 exp(-h/ell); nu = 3/2 -> sigma2 (1 + h/ell) exp(-h/ell)
    for s2, ell in [(1.0, 0.1), (2.5, 0.0864), (0.7, 1.3)]:
        x = H / ell
        b05 = oracle.matern(H, s2, ell, 0.5, use_bessel=True)
        b15 = oracle.matern(H, s2, ell, 1.5, use_bessel=True)
        np.testing.assert_allclose(b05, s2 * np.exp(-x), rtol=1e-13, atol=1e-300)
        np.testing.assert_allclose(b15, s2 * (1 + x) * np.exp(-x), rtol=1e-13, atol=1e-300)
        # the fast path uses the same closed forms
        np.testing.assert_allclose(oracle.matern(H, s2, ell, 0.5), b05, rtol=1e-13, atol=1e-300)
        np.testing.assert_allclose(oracle.matern(H, s2, ell, 1.5), b15, rtol=1e-13, atol=1e-300)


def test_bessel_half_identity_through_matern():
    # K_{1/2}(x) = sqrt(pi / (2x)) e^{-x}, recovered from the oracle's Bessel path
    x = np.array([1e-6, 0.01, 0.5, 1.0, 2.0, 10.0, 50.0])
    m = oracle.matern(x, 1.0, 1.0, 0.5, use_bessel=True)
    k = m * 2.0 ** (0.5 - 1.0) * math.gamma(0.5) / x ** 0.5
    np.testing.assert_allclose(k, np.sqrt(np.pi / (2 * x)) * np.exp(-x), rtol=1e-13)


@pytest.mark.parametrize("nu", [0.325, 1.0, 2.0, 0.7])
def test_matern_general_nu_vs_mpmath(nu):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    ell, s2 = 0.05, 1.3
    hs = np.array([1e-8, 1e-5, 1e-3, 0.01, 0.05, 0.2, 1.0, 5.0])
    got = oracle.matern(hs, s2, ell, nu)
    for h, g in zip(hs, got):
        x = mpmath.mpf(h) / ell
        ref = s2 / (mpmath.power(2, nu - 1) * mpmath.gamma(nu)) * mpmath.power(x, nu) * mpmath.besselk(nu, x)
        assert abs(g - float(ref)) <= 1e-13 * abs(float(ref)) + 1e-300, (nu, h, g, float(ref))


def test_bessel_recurrence_through_matern():
    # K_{nu+1}(x) = K_{nu-1}(x) + (2 nu / x) K_nu(x)
    def K(nu, x):
        m = oracle.matern(x, 1.0, 1.0, nu, use_bessel=True)
        return m * 2.0 ** (nu - 1.0) * math.gamma(nu) / x ** nu

    x = np.array([0.05, 0.3, 1.0, 4.0, 12.0])
    for nu in [1.325, 1.8, 2.5]:
        lhs = K(nu + 1, x)
        rhs = K(nu - 1, x) + 2 * nu / x * K(nu, x)
        np.testing.assert_allclose(lhs, rhs, rtol=1e-12)


def test_matern_limits():
    for nu in [0.325, 0.5, 1.0, 1.5, 2.0]:
        v = oracle.matern(np.array([0.0, 1e-200, 800.0]), 1.7, 0.1, nu)
        assert v[0] == 1.7 and v[1] == 1.7
        assert 0.0 <= v[2] < 1e-300
        # monotone decrease in h
        hh = np.linspace(0, 2, 200)
        vv = oracle.matern(hh, 1.0, 0.1, nu)
        assert np.all(np.diff(vv) <= 0)


# ----------------------------------------------------------------------------
# Dense eq. (1)
# ----------------------------------------------------------------------------
def leibniz_det(A):
    n = A.shape[0]
    tot = 0.0
    for perm in itertools.permutations(range(n)):
        inv = sum(1 for i in range(n) for j in range(i + 1, n) if perm[i] > perm[j])
        p = 1.0
        for i in range(n):
            p *= A[i, perm[i]]
        tot += (-1) ** inv * p
    return tot


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7])
def test_dense_logdet_vs_bruteforce(n):
    xy = inputs.points(n, 11 + n)
    z = inputs.normal(n, 21 + n)
    th = (1.3, 0.2, 0.5, 1e-2)
    C = oracle.dense_cov(xy, *th)
    L, logdet, quad = oracle.dense_loglik(xy, z, *th)
    det = leibniz_det(np.array(C))
    assert abs(logdet - math.log(det)) <= 1e-12 * max(1.0, abs(math.log(det)))
    # quadratic form by Cramer's rule on the brute-force determinant
    x = np.zeros(n)
    for i in range(n):
        Ci = np.array(C)
        Ci[:, i] = z
        x[i] = leibniz_det(Ci) / det
    assert abs(quad - z @ x) <= 1e-11 * abs(z @ x)
    assert abs(L - (-n / 2 * math.log(2 * math.pi) - logdet / 2 - quad / 2)) < 1e-12 * abs(L)


def test_dense_n1_n2_closed_forms():
    s2, ell, nu, tau2 = 1.7, 0.3, 1.5, 1e-3
    xy = np.array([[0.2, 0.4]])
    L, logdet, quad = oracle.dense_loglik(xy, np.array([0.9]), s2, ell, nu, tau2)
    ref = -0.5 * math.log(2 * math.pi) - 0.5 * math.log(s2 + tau2) - 0.81 / (2 * (s2 + tau2))
    assert abs(L - ref) < 1e-14
    xy = np.array([[0.2, 0.4], [0.5, 0.1]])
    h = math.hypot(0.3, 0.3)
    m = s2 * (1 + h / ell) * math.exp(-h / ell)
    _, logdet, _ = oracle.dense_loglik(xy, np.array([0.1, -0.2]), s2, ell, nu, tau2)
    assert abs(logdet - math.log((s2 + tau2) ** 2 - m * m)) < 1e-13


def test_dense_cholesky_vs_numpy_and_reconstruction():
    xy = inputs.points(300, 5)
    C = oracle.dense_cov(xy, 1.0, 0.1, 0.325, 1e-4)
    L = oracle.dense_cholesky(C)
    np.testing.assert_allclose(L @ L.T, C, atol=1e-13)
    np.testing.assert_allclose(L, np.linalg.cholesky(C), atol=1e-11)
    z = inputs.normal(300, 6)
    _, logdet, quad = oracle.dense_loglik(xy, z, 1.0, 0.1, 0.325, 1e-4)
    s, ld = np.linalg.slogdet(C)
    assert s > 0 and abs(logdet - ld) < 1e-9
    assert abs(quad - z @ np.linalg.solve(C, z)) < 1e-8 * abs(quad)


def test_dense_quad_of_factor_sample_is_norm_of_xi():
    # z = L xi  =>  z^T C^-1 z = |xi|^2 (exactly, up to rounding)
    xy = inputs.points(500, 7)
    xi = inputs.normal(500, 8)
    z = oracle.dense_chol_apply(xy, xi, 1.0, 0.1, 0.5, 1e-4)
    _, _, quad = oracle.dense_loglik(xy, z, 1.0, 0.1, 0.5, 1e-4)
    assert abs(quad - xi @ xi) < 1e-9 * (xi @ xi)


def test_dense_scaling_and_permutation_invariance():
    xy = inputs.points(400, 9)
    z = inputs.normal(400, 10)
    a = 3.7
    _, ld0, q0 = oracle.dense_loglik(xy, z, 1.0, 0.08, 1.5, 1e-4)
    _, ld1, q1 = oracle.dense_loglik(xy, z, a, 0.08, 1.5, a * 1e-4)
    assert abs(ld1 - (ld0 + 400 * math.log(a))) < 1e-9 * abs(ld0)
    assert abs(q1 - q0 / a) < 1e-10 * q0
    p = np.random.default_rng(3).permutation(400)
    L0 = oracle.dense_loglik(xy, z, 1.0, 0.08, 1.5, 1e-4)[0]
    L1 = oracle.dense_loglik(xy[p], z[p], 1.0, 0.08, 1.5, 1e-4)[0]
    assert abs(L0 - L1) < 1e-10 * abs(L0)


def test_dense_not_spd_detected():
    xy = np.array([[0.1, 0.1], [0.1, 0.1], [0.5, 0.2]])
    with pytest.raises(np.linalg.LinAlgError):
        oracle.dense_loglik(xy, np.ones(3), 1.0, 0.1, 0.5, 0.0)


def test_far_apart_points_closed_form():
    # spacing 0.05 with ell = 1e-4: covariance = (sigma2 + tau2) I to 1e-200
    g = np.linspace(0.0, 1.0, 21)
    xy = np.array([[a, b] for a in g for b in g])
    n = len(xy)
    z = inputs.normal(n, 12)
    s2, tau2 = 1.4, 2e-3
    ref = -n / 2 * math.log(2 * math.pi) - n / 2 * math.log(s2 + tau2) - (z @ z) / (2 * (s2 + tau2))
    assert abs(oracle.dense_loglik(xy, z, s2, 1e-4, 0.5, tau2)[0] - ref) < 1e-10 * abs(ref)
    r = oracle.h_loglik(xy, z, s2, 1e-4, 0.5, tau2, 1e-6, leaf=16)
    assert abs(r["loglik"] - ref) < 1e-10 * abs(ref)


# ----------------------------------------------------------------------------
# Recompression (Remark A.1) and ACA (App. B)
# ----------------------------------------------------------------------------
def test_truncation_exact_low_rank():
    rng = np.random.default_rng(0)
    U = rng.standard_normal((80, 5)) @ rng.standard_normal((5, 12))
    V = rng.standard_normal((60, 12))
    Uk, Vk = oracle.truncate(U, V, 1e-10)
    assert Uk.shape[1] == 5
    np.testing.assert_allclose(Uk @ Vk.T, U @ V.T, atol=1e-11 * np.abs(U @ V.T).max())


def test_truncation_is_eckart_young():
    rng = np.random.default_rng(1)
    m, n, K = 70, 50, 30
    Q1, _ = np.linalg.qr(rng.standard_normal((m, K)))
    Q2, _ = np.linalg.qr(rng.standard_normal((n, K)))
    s = 10.0 ** -np.arange(K) * 0.5 ** 0.5
    U = Q1 * s
    V = Q2
    for eps in [3e-3, 3e-6, 3e-9]:
        Uk, Vk = oracle.truncate(U, V, eps)
        k = int(np.sum(s > eps * s[0]))
        assert Uk.shape[1] == k
        A = U @ V.T
        uu, ss, vt = np.linalg.svd(A)
        best = (uu[:, :k] * ss[:k]) @ vt[:k]
        np.testing.assert_allclose(Uk @ Vk.T, best, atol=1e-13 * ss[0])


def test_aca_far_block_accuracy_and_rank():
    xy = inputs.points(4000, 1)
    Hh = oracle.HOracle(xy, leaf=64)
    Hh.set_theta(1.0, 0.1, 0.5, 1e-4)
    blocks = Hh.leaf_blocks()
    lr = blocks[blocks[:, 4] == 1]
    sizes = (lr[:, 1] - lr[:, 0]) * (lr[:, 3] - lr[:, 2])
    perm = Hh.perm()
    for q in np.argsort(-sizes)[:6]:
        r0, r1, c0, c1, _ = lr[q]
        M = oracle.dense_cov(xy[perm[np.r_[r0:r1, c0:c1]]], 1.0, 0.1, 0.5, 0.0)[: r1 - r0, r1 - r0:]
        for eps in [1e-5, 1e-7]:
            U, V = Hh.aca_block(r0, r1 - r0, c0, c1 - c0, eps)
            err = np.linalg.norm(M - U @ V.T) / np.linalg.norm(M)
            assert err <= 10 * eps, (q, eps, err)
            sv = np.linalg.svd(M, compute_uv=False)
            k_exact = int(np.sum(sv > eps * sv[0]))
            assert abs(U.shape[1] - k_exact) <= 2, (U.shape[1], k_exact)


# ----------------------------------------------------------------------------
# Cluster tree and block-cluster tree (Sec. 2.2, App. A)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("n,leaf", [(777, 16), (3000, 32)])
def test_cluster_tree_properties(n, leaf):
    xy = inputs.points(n, 40 + n)
    Hh = oracle.HOracle(xy, leaf=leaf)
    perm = Hh.perm()
    assert sorted(perm) == list(range(n))
    pts = xy[perm]
    lohi, bbox, lev, isleaf = Hh.clusters()
    by = {(int(a), int(b)): i for i, (a, b) in enumerate(lohi)}
    for i, (lo, hi) in enumerate(lohi):
        p = pts[lo:hi]
        np.testing.assert_array_equal(bbox[i], [p[:, 0].min(), p[:, 1].min(), p[:, 0].max(), p[:, 1].max()])
        if isleaf[i]:
            assert hi - lo <= leaf or np.ptp(p, axis=0).max() == 0
            continue
        # two children partition the parent at the midpoint of the longest axis
        kids = [j for j, (a, b) in enumerate(lohi) if lev[j] == lev[i] + 1 and a >= lo and b <= hi]
        assert len(kids) == 2
        k0, k1 = sorted(kids, key=lambda j: lohi[j][0])
        assert lohi[k0][0] == lo and lohi[k0][1] == lohi[k1][0] and lohi[k1][1] == hi
        ext = bbox[i, 2:] - bbox[i, :2]
        ax = 0 if ext[0] >= ext[1] else 1
        mid = 0.5 * (bbox[i, ax] + bbox[i, 2 + ax])
        assert np.all(pts[lohi[k0][0]:lohi[k0][1], ax] <= mid)
        assert np.all(pts[lohi[k1][0]:lohi[k1][1], ax] > mid)
    assert by[(0, n)] == 0


def test_morton_order_of_root_before_bisection():
    # Within every leaf cluster, points keep the Morton order of the global
    # bounding-box quantisation (the bisection partitions stably).
    xy = inputs.points(2000, 3)
    Hh = oracle.HOracle(xy, leaf=32)
    perm = Hh.perm()
    lo = xy.min(axis=0)
    hi = xy.max(axis=0)
    q = np.floor((xy - lo) / (hi - lo) * 4294967295.0).astype(np.uint64)
    key = np.zeros(len(xy), dtype=np.uint64)
    for b in range(32):
        key |= ((q[:, 0] >> np.uint64(b)) & np.uint64(1)) << np.uint64(2 * b)
        key |= ((q[:, 1] >> np.uint64(b)) & np.uint64(1)) << np.uint64(2 * b + 1)
    lohi, _, _, isleaf = Hh.clusters()
    for (a, b), lf in zip(lohi, isleaf):
        if lf:
            k = key[perm[a:b]]
            assert np.all(k[1:] >= k[:-1])


@pytest.mark.parametrize("n,leaf,eta", [(600, 16, 2.0), (2500, 32, 2.0), (2500, 32, 0.7)])
def test_block_tree_partitions_lower_triangle(n, leaf, eta):
    xy = inputs.points(n, 60 + n)
    Hh = oracle.HOracle(xy, leaf=leaf, eta=eta)
    perm = Hh.perm()
    pts = xy[perm]
    cover = np.zeros((n, n), dtype=np.int32)
    for r0, r1, c0, c1, t in Hh.leaf_blocks():
        assert r0 >= c0
        cover[r0:r1, c0:c1] += 1
        R, S = pts[r0:r1], pts[c0:c1]
        diam = lambda P: np.hypot(*np.ptp(P, axis=0))
        gap = np.maximum(0, np.maximum(R.min(0) - S.max(0), S.min(0) - R.max(0)))
        dist = np.hypot(*gap)
        adm = dist > 0 and min(diam(R), diam(S)) <= eta * dist
        assert bool(adm) == (t == 1)
        if t == 0 and r0 != c0:
            assert (r1 - r0 <= leaf) or (c1 - c0 <= leaf)
    low = np.tril(np.ones((n, n), dtype=bool))
    assert np.all(cover[low] == 1)
    # upper triangle only covered by diagonal blocks
    assert np.all(cover[~low] <= 1)


# ----------------------------------------------------------------------------
# H-matrix approximation, H-Cholesky and eq. (2)
# ----------------------------------------------------------------------------
def _power_norm(apply, n, it=30, seed=0):
    x = np.random.default_rng(seed).standard_normal(n)
    lam = 0.0
    for _ in range(it):
        y = apply(x)
        lam = np.linalg.norm(y)
        if lam == 0:
            return 0.0
        x = y / lam
    return lam


@pytest.mark.parametrize("eps", [1e-4, 1e-6, 1e-8])
def test_h_approximation_error_is_order_eps(eps):
    xy = inputs.points(1500, 70)
    C = oracle.dense_cov(xy, 1.0, 0.1, 0.5, 1e-4)
    Hh = oracle.HOracle(xy, leaf=32)
    Hh.assemble(1.0, 0.1, 0.5, 1e-4, eps)
    Ct = Hh.expand(0)
    nC = _power_norm(lambda v: C @ v, 1500)
    e1 = _power_norm(lambda v: (C - Ct) @ v, 1500) / nC
    assert e1 <= 5 * eps
    # the H-matvec is the product with the expanded matrix
    x = inputs.normal(1500, 71)
    np.testing.assert_allclose(Hh.matvec(x), Ct @ x, rtol=0, atol=1e-12 * np.abs(Ct @ x).max())
    Hh.cholesky(eps)
    Lt = Hh.expand(1)
    e2 = _power_norm(lambda v: Ct @ v - Lt @ (Lt.T @ v), 1500) / nC
    assert e2 <= 20 * eps, e2


def test_h_loglik_vs_dense_n2000():
    # The small workload: n=2000, nu=1/2, ell=0.1, eps=1e-7, z = L xi.
    w = inputs.WORKLOADS["n2000_nu0.5_eps1e-7"]
    xy = inputs.workload_points("n2000_nu0.5_eps1e-7")
    xi = inputs.workload_normal("n2000_nu0.5_eps1e-7")
    th = (w["sigma2"], w["ell"], w["nu"], w["nugget"])
    z = oracle.dense_chol_apply(xy, xi, *th)
    Ld, ldd, qd = oracle.dense_loglik(xy, z, *th)
    assert abs(qd - xi @ xi) < 1e-8 * (xi @ xi)
    r = oracle.h_loglik(xy, z, *th, w["eps"], leaf=w["leaf"], eta=w["eta"])
    assert abs(r["loglik"] - Ld) / 2000 <= 1e-6
    assert abs(r["logdet"] - ldd) / 2000 <= 1e-6
    assert r["rel_residual"] <= 1e-12


def test_h_loglik_scaling_invariance():
    xy = inputs.points(1200, 80)
    z = inputs.normal(1200, 81)
    a = 2.5
    r0 = oracle.h_loglik(xy, z, 1.0, 0.05, 1.5, 1e-4, 1e-8, leaf=32)
    r1 = oracle.h_loglik(xy, z, a, 0.05, 1.5, a * 1e-4, 1e-8, leaf=32)
    assert abs(r1["logdet"] - (r0["logdet"] + 1200 * math.log(a))) < 1e-8 * abs(r0["logdet"])
    assert abs(r1["quad"] - r0["quad"] / a) < 1e-9 * r0["quad"]


def test_paper_table5_storage_order_of_magnitude():
    # Table 5 prints the storage of C~ at eps = 1e-5 for nu=0.33, ell=0.65:
    # 5.1 kB per degree of freedom at n = 32,000 (HLIBpro, leaf size unstated).
    with open(os.path.join(GOLDEN, "table5_storage.json")) as f:
        g = json.load(f)
    row = g["rows"][0]
    n = 8000  # a quarter of the table's n; kB/dof grows only like log n
    xy = inputs.points(n, 90)
    Hh = oracle.HOracle(xy, leaf=64)
    Hh.assemble(1.0, g["ell"], g["nu"], 1e-4, g["eps"])
    kb = Hh.stats()["entries_C"] * 8 / n / 1000.0
    assert row["kb_per_dof"] / 4 <= kb <= row["kb_per_dof"] * 2, kb


def test_paper_table5_inverse_error_order_of_magnitude():
    # Table 5 prints ||I - (L~ L~^T)^-1 C~||_2 = 2.4e-3 at n = 32,000 for
    # nu=0.33, ell=0.65, sigma2=1, block accuracy 1e-5 for C~ and L~ (growing
    # slowly with n).  The oracle at n = 2000 (nugget 1e-4) lands within a
    # factor 10 of it.  The expansions are in caller order, where L~ is a
    # permuted triangle, so the inverse goes through a Cholesky of L~ L~^T.
    import scipy.linalg as sl

    with open(os.path.join(GOLDEN, "table5_storage.json")) as f:
        g = json.load(f)
    target = g["rows"][0]["inv_err"]
    n = 2000
    xy = inputs.points(n, 95)
    Hh = oracle.HOracle(xy, leaf=64)
    Hh.assemble(1.0, g["ell"], g["nu"], 1e-4, g["eps"])
    Hh.cholesky(g["eps"])
    Ct, Lt = Hh.expand(0), Hh.expand(1)
    cf = sl.cho_factor(Lt @ Lt.T)

    def a(v):
        return v - sl.cho_solve(cf, Ct @ v)

    def at(v):
        return v - Ct @ sl.cho_solve(cf, v)

    v = np.random.default_rng(0).standard_normal(n)
    v /= np.linalg.norm(v)
    lam = 0.0
    for _ in range(40):
        y = at(a(v))
        lam = np.linalg.norm(y)
        v = y / lam
    err = math.sqrt(lam)
    assert target / 10 <= err <= target * 10, err


def test_h_loglik_permutation_invariance():
    # The tree depends on the point set, not on its order: permuting the
    # locations (and z with them) gives the same likelihood.
    n = 1500
    xy = inputs.points(n, 96)
    z = inputs.normal(n, 97)
    p = np.random.default_rng(98).permutation(n)
    r0 = oracle.h_loglik(xy, z, 1.0, 0.08, 0.5, 1e-4, 1e-7, leaf=32)
    r1 = oracle.h_loglik(xy[p], z[p], 1.0, 0.08, 0.5, 1e-4, 1e-7, leaf=32)
    assert abs(r1["loglik"] - r0["loglik"]) <= 1e-9 * abs(r0["loglik"])
    assert abs(r1["logdet"] - r0["logdet"]) <= 1e-9 * abs(r0["logdet"])


# ----------------------------------------------------------------------------
# Products with the H-Cholesky factor (synthetic data Z = L~ xi, Sec. 5.1)
# ----------------------------------------------------------------------------
def test_factor_product_equals_dense_cholesky_of_tree_ordered_matrix():
    # At an accuracy below rounding every low-rank block is exact, so the
    # H-Cholesky factor is the dense Cholesky factor of the covariance in
    # tree order: L~ x (user order) = P L_p P^T x with L_p = chol(P^T C P).
    n = 400
    xy = inputs.points(n, 4100)
    th = (1.0, 0.1, 0.5, 1e-2)
    H = oracle.HOracle(xy, leaf=32)
    H.assemble(*th, 1e-15)
    H.cholesky(1e-15)
    perm = H.perm()
    C = oracle.dense_cov(xy, *th)
    Lp = np.linalg.cholesky(C[np.ix_(perm, perm)])
    x = inputs.normal(n, 4101)
    for trans in (False, True):
        A = Lp.T if trans else Lp
        ref = np.zeros(n)
        ref[perm] = A @ x[perm]
        got = H.lmatvec(x, trans=trans)
        assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)


def test_factor_product_reproduces_covariance():
    # L~ (L~^T x) = C~ x to the accuracy of the factorisation (order eps)
    n, eps = 2500, 1e-8
    xy = inputs.points(n, 4102)
    H = oracle.HOracle(xy, leaf=32)
    H.assemble(1.0, 0.08, 1.5, 1e-4, eps)
    H.cholesky(eps)
    x = inputs.normal(n, 4103)
    y = H.lmatvec(H.lmatvec(x, trans=True))
    ref = H.matvec(x)
    assert np.linalg.norm(y - ref) <= 50 * eps * np.linalg.norm(ref)
    # and against the expanded factor (the lower triangle of the blocks)
    Le = H.expand(1)
    np.testing.assert_allclose(H.lmatvec(x), Le @ x, rtol=0, atol=1e-12 * np.abs(Le @ x).max())


# ----------------------------------------------------------------------------
# Variants of the block structure and of the rank (Sec. 2.2, App. A,
# Tables 2 and 3)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("n,leaf", [(777, 16), (3001, 32)])
def test_cardinality_split_halves_at_the_median(n, leaf):
    # "two (equal sized) sub-sets": each split puts floor(size/2) points,
    # those with the smallest coordinates along the longest bbox axis, left
    xy = inputs.points(n, 4200 + n)
    xy[10:40, 0] = xy[5, 0]  # ties on the split coordinate
    Hh = oracle.HOracle(xy, leaf=leaf, split=1)
    perm = Hh.perm()
    assert sorted(perm) == list(range(n))
    pts = xy[perm]
    lohi, bbox, lev, isleaf = Hh.clusters()
    nsplit = 0
    for i, (lo, hi) in enumerate(lohi):
        if isleaf[i]:
            assert hi - lo <= leaf
            continue
        nsplit += 1
        kids = [j for j, (a, b) in enumerate(lohi) if lev[j] == lev[i] + 1 and a >= lo and b <= hi]
        k0, k1 = sorted(kids, key=lambda j: lohi[j][0])
        assert lohi[k0][1] - lo == (hi - lo) // 2
        ext = bbox[i, 2:] - bbox[i, :2]
        ax = 0 if ext[0] >= ext[1] else 1
        assert pts[lo:lohi[k0][1], ax].max() <= pts[lohi[k1][0]:hi, ax].min()
    assert nsplit > 0


@pytest.mark.parametrize("adm,eta", [(1, 2.0), (1, 4.0), (2, 2.0)])
def test_block_tree_admissibility_variants(adm, eta):
    n, leaf = 2500, 32
    xy = inputs.points(n, 4300)
    Hh = oracle.HOracle(xy, leaf=leaf, eta=eta, admissibility=adm)
    pts = xy[Hh.perm()]
    cover = np.zeros((n, n), dtype=np.int32)
    nlr = 0
    for r0, r1, c0, c1, t in Hh.leaf_blocks():
        cover[r0:r1, c0:c1] += 1
        R, S = pts[r0:r1], pts[c0:c1]
        diam = lambda P: np.hypot(*np.ptp(P, axis=0))
        gap = np.maximum(0, np.maximum(R.min(0) - S.max(0), S.min(0) - R.max(0)))
        dist = np.hypot(*gap)
        if adm == 1:
            assert bool(dist > 0 and max(diam(R), diam(S)) <= eta * dist) == (t == 1)
        else:  # weak: every block of two distinct clusters is low-rank
            assert (t == 1) == (r0 != c0)
        nlr += t == 1
    low = np.tril(np.ones((n, n), dtype=bool))
    assert np.all(cover[low] == 1) and nlr > 0
    # max-diam is stricter than the standard rule: fewer low-rank leaves
    if adm == 1:
        std = oracle.HOracle(xy, leaf=leaf, eta=eta)
        assert (std.leaf_blocks()[:, 4] == 1).sum() >= nlr


@pytest.mark.parametrize("adm,split", [(1, 0), (2, 0), (0, 1), (2, 1)])
def test_variant_h_loglik_vs_dense(adm, split):
    # every variant approximates the same eq. (1)
    n = 1500
    xy = inputs.points(n, 4400)
    th = (1.0, 0.1, 0.5, 1e-4)
    z = oracle.dense_chol_apply(xy, inputs.normal(n, 4401), *th)
    Ld = oracle.dense_loglik(xy, z, *th)[0]
    r = oracle.h_loglik(xy, z, *th, 1e-8, leaf=32, admissibility=adm, split=split)
    assert abs(r["loglik"] - Ld) / n <= 1e-6


def test_fixed_rank_caps_ranks_and_error_falls_with_k():
    # Tables 2 and 3: fixed rank k, no nugget; ranks never exceed k and the
    # approximation error falls as k grows
    n = 1200
    xy = inputs.points(n, 4500)
    th = (1.0, 0.25, 0.5, 0.0)
    C = oracle.dense_cov(xy, *th)
    errs = []
    for k in (4, 8, 16):
        Hh = oracle.HOracle(xy, leaf=32, fixed_rank=k)
        Hh.assemble(*th, 1e-14)
        r = Hh.ranks(0)
        assert r.max() <= k
        errs.append(np.linalg.norm(C - Hh.expand(0), 2))
    assert errs[0] > errs[1] > errs[2]
    # a cap above every adaptive rank changes nothing
    Ha = oracle.HOracle(xy, leaf=32)
    Ha.assemble(*th, 1e-6)
    Hk = oracle.HOracle(xy, leaf=32, fixed_rank=int(Ha.ranks(0).max()) + 5)
    Hk.assemble(*th, 1e-6)
    np.testing.assert_array_equal(Ha.expand(0), Hk.expand(0))


# ----------------------------------------------------------------------------
# Accumulated updates (accumulate=1): the same factorisation with the updates
# of a low-rank block truncated together before the block is next used
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("eps", [1e-5, 1e-7])
def test_accumulated_updates_factor_error_is_order_eps(eps):
    n = 1500
    xy = inputs.points(n, 4600)
    Hh = oracle.HOracle(xy, leaf=32)
    Hh.assemble(1.0, 0.08, 0.5, 1e-4, eps)
    Ct = Hh.expand(0)
    Hh.cholesky(eps, accumulate=True)
    Lt = Hh.expand(1)
    nC = _power_norm(lambda v: Ct @ v, n)
    e2 = _power_norm(lambda v: Ct @ v - Lt @ (Lt.T @ v), n) / nC
    assert e2 <= 20 * eps, e2
    # the factor is lower triangular with a positive diagonal
    assert np.allclose(np.triu(Lt[np.ix_(Hh.perm(), Hh.perm())], 1), 0.0)


def test_accumulated_updates_loglik_vs_dense_n2000():
    w = inputs.WORKLOADS["n2000_nu0.5_eps1e-7"]
    xy = inputs.workload_points("n2000_nu0.5_eps1e-7")
    xi = inputs.workload_normal("n2000_nu0.5_eps1e-7")
    th = (w["sigma2"], w["ell"], w["nu"], w["nugget"])
    z = oracle.dense_chol_apply(xy, xi, *th)
    Ld, ldd, _ = oracle.dense_loglik(xy, z, *th)
    r = oracle.h_loglik(xy, z, *th, w["eps"], leaf=w["leaf"], eta=w["eta"], accumulate=True)
    assert abs(r["loglik"] - Ld) / 2000 <= 1e-6
    assert abs(r["logdet"] - ldd) / 2000 <= 1e-6
