"""Products with the H-Cholesky factor on the GPU (hlc_factor_apply,
hlc_sample: synthetic data Z = L~ xi of Sec. 5.1) and the per-result error
estimate est_rel_err, against the CPU oracle."""
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


@pytest.fixture(scope="module")
def ctx(hlc):
    c = hlc.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("n,leaf,nu", [(3000, 32, 0.5), (5000, 64, 1.5), (1, 64, 0.5), (97, 64, 0.325)])
def test_factor_apply_vs_oracle(ctx, hlc, n, leaf, nu):
    eps = 1e-8
    xy = inputs.points(n, 5200 + n)
    th = (1.0, 0.08, nu, 1e-4)
    t = ctx.build_tree(xy, leaf=leaf, eps=eps)
    C = t.assemble(hlc.theta(*th))
    L = t.cholesky(C)
    H = oracle.HOracle(xy, leaf=leaf)
    H.assemble(*th, eps)
    H.cholesky(eps)
    x = inputs.normal(n, 5201)
    for trans in (False, True):
        y = L.factor_apply(x, trans=trans)
        ref = H.lmatvec(x, trans=trans)
        # the two factors agree to a few hundred eps (test_cholesky_reproduces_matrix)
        assert np.linalg.norm(y - ref) <= 500 * eps * np.linalg.norm(ref)
    # L~ (L~^T x) = C~ x to the accuracy of the factorisation
    y = L.factor_apply(L.factor_apply(x, trans=True))
    ref = C.matvec(x)
    assert np.linalg.norm(y - ref) <= 50 * eps * np.linalg.norm(ref)


def test_sample_then_loglik(ctx, hlc):
    # z = L~ xi: the factor's quadratic form v^T v (L~ v = z) is |xi|^2 up to
    # rounding, and the refined z^T C~^-1 z agrees to the factor's accuracy
    n, eps = 6000, 1e-7
    xy = inputs.points(n, 5300)
    th = hlc.theta(1.0, 0.0864, 0.5, 1e-4)
    xi = inputs.normal(n, 5301)
    t = ctx.build_tree(xy, leaf=64, eps=eps)
    z = t.sample(th, xi)
    H = oracle.HOracle(xy, leaf=64)
    H.assemble(1.0, 0.0864, 0.5, 1e-4, eps)
    H.cholesky(eps)
    zo = H.lmatvec(xi)
    assert np.linalg.norm(z - zo) <= 500 * eps * np.linalg.norm(zo)
    r = t.loglik(th, z)
    assert abs(r["quad_factor"] - xi @ xi) <= 1e-9 * (xi @ xi)
    assert abs(r["quad"] - xi @ xi) / n <= 1e-6


def test_sample_device_tensors(ctx, hlc):
    torch = pytest.importorskip("torch")
    n = 2000
    xy = inputs.points(n, 5400)
    xi = inputs.normal(n, 5401)
    th = hlc.theta(1.0, 0.1, 0.5, 1e-4)
    t = ctx.build_tree(xy, leaf=32, eps=1e-8)
    z_host = t.sample(th, xi)
    z_dev = t.sample(th, torch.tensor(xi, device="cuda"))
    assert np.array_equal(z_dev.cpu().numpy(), z_host)


@pytest.mark.parametrize("eps", [1e-4, 1e-5])
def test_est_rel_err_vs_dense(ctx, hlc, eps):
    # est_rel_err estimates |I - (L~ L~^T)^-1 C~|_2 from the CG's Lanczos
    # coefficients.  Dense reference from the GPU's own C~ and L~: the
    # operator is similar to a symmetric one, its eigenvalues are real, and
    # the Ritz values lie inside its spectrum, so the estimate cannot exceed
    # the spectral radius rho; with the CG iterations these tolerances need
    # it comes within a factor 2 of it.
    n = 2000
    xy = inputs.points(n, 5500)
    z = inputs.normal(n, 5501)
    th = hlc.theta(1.0, 0.1, 0.5, 1e-4)
    t = ctx.build_tree(xy, leaf=32, eps=eps)
    r = t.loglik(th, z)
    C = t.assemble(th)
    L = t.cholesky(C)
    Ce, Le = C.expand(), L.expand()
    A = np.eye(n) - np.linalg.solve(Le @ Le.T, Ce)
    rho = np.max(np.abs(np.linalg.eigvals(A)))
    assert r["refine_iters"] >= 2
    assert r["est_rel_err"] <= 1.01 * rho
    assert r["est_rel_err"] >= 0.5 * rho, (r["est_rel_err"], rho, r["refine_iters"])
    # the 2-norm of Table 5's column is at least the spectral radius
    assert np.linalg.norm(A, 2) >= rho * (1 - 1e-9)
