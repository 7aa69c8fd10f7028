"""Accuracy diagnostics of Sec. 3 (hlc_diagnostics) against dense
references at n = 2000: the power-iteration norms of C - C~, C~ - L~ L~^T,
I - (L~ L~^T)^-1 C~ (Table 5's last column) and the probe estimate of the
KLD, with C~ and L~ the GPU's own (expanded) and C the dense oracle."""
import numpy as np
import pytest

import oracle
from paper_1709_08625_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hlc():
    from paper_1709_08625_gb300 import build

    build.build()
    from paper_1709_08625_gb300 import hlc as h

    return h


@pytest.mark.parametrize("nu,eps,nugget", [(0.5, 1e-4, 0.05), (1.5, 1e-5, 0.05), (0.325, 1e-5, 1e-2)])
def test_diagnostics_vs_dense(hlc, nu, eps, nugget):
    n = 2000
    xy = inputs.points(n, 6500)
    th = (1.0, 0.1, nu, nugget)
    ctx = hlc.Context(0)
    t = ctx.build_tree(xy, leaf=32, eps=eps)
    d = t.diagnostics(hlc.theta(*th), iters=40, probes=64, seed=3)
    C = t.assemble(hlc.theta(*th))
    L = t.cholesky(C)
    Ch, Lh = C.expand(), L.expand()
    Cx = oracle.dense_cov(xy, *th)
    ref = dict(err_C=np.linalg.norm(Cx - Ch, 2), norm_C=np.linalg.norm(Cx, 2),
               err_LLt=np.linalg.norm(Ch - Lh @ Lh.T, 2), norm_Ch=np.linalg.norm(Ch, 2),
               inv_err=np.linalg.norm(np.eye(n) - np.linalg.solve(Lh @ Lh.T, Ch), 2))
    # power iteration approaches each norm from below
    for k, v in ref.items():
        assert d[k] <= v * (1 + 1e-6) + 1e-300, (k, d[k], v)
        assert d[k] >= 0.8 * v, (k, d[k], v)
    # KLD(C, C~) = 1/2 sum (delta_i - log(1 + delta_i)), delta = eig of
    # C~^-1/2 (C - C~) C~^-1/2; the estimate is 1/4 |L~^-1 (C - C~) L~^-T|_F^2
    # by 64 Gaussian probes (relative spread ~ sqrt(2/64))
    Lc = np.linalg.cholesky(Ch)
    Bm = np.linalg.solve(Lc, np.linalg.solve(Lc, (Cx - Ch).T).T)
    delta = np.linalg.eigvalsh(0.5 * (Bm + Bm.T))
    kld = 0.5 * np.sum(delta - np.log1p(delta))
    assert d["kld"] > 0
    assert 0.5 * kld <= d["kld"] <= 1.6 * kld, (d["kld"], kld)
    ctx.close()


def test_diagnostics_large_n_skips_exact_parts(hlc):
    # above 131,072 locations the O(n^2) parts are not computed (-1)
    n = 140000
    ctx = hlc.Context(0)
    t = ctx.build_tree(inputs.points(n, 6600), leaf=64, eps=1e-5)
    d = t.diagnostics(hlc.theta(1.0, 0.05, 0.5, 1e-4), iters=3, probes=2)
    assert d["err_C"] == -1 and d["norm_C"] == -1 and d["kld"] == -1
    # the 2-norm of the nonsymmetric I - (L L^T)^-1 C~ may exceed its spectral
    # radius by up to the condition of L~: only finite and positive here
    assert 0 < d["inv_err"] < np.inf and 0 < d["err_LLt"] < np.inf and d["norm_Ch"] > 1
    ctx.close()
