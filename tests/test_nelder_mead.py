"""The simplex method of the identification (App. B: Nelder-Mead), pinned on
the CPU against SciPy's Nelder-Mead (the same published method: reflection 1,
expansion 2, contraction 1/2, shrink 1/2) and against known minima."""
import numpy as np
import pytest

scipy_optimize = pytest.importorskip("scipy.optimize")


@pytest.fixture(scope="module")
def hlc():
    from paper_1709_08625_gb300 import build

    build.build()
    from paper_1709_08625_gb300 import hlc as h

    return h


def rosen(x):
    return float(np.sum(100.0 * (x[1:] - x[:-1] ** 2) ** 2 + (1 - x[:-1]) ** 2))


def quad3(x):
    c = np.array([0.5, 0.0864, 1.0])
    w = np.array([3.0, 50.0, 1.0])
    return float(np.sum(w * (x - c) ** 2))


@pytest.mark.parametrize("f,x0,step", [(rosen, [-1.2, 1.0], [0.1, 0.1]),
                                       (quad3, [0.6, 0.1, 1.2], [0.02, 0.04, 0.01]),
                                       (rosen, [0.0, 0.0, 0.0], [0.5, 0.5, 0.5])])
@pytest.mark.parametrize("iters", [1, 5, 40])
def test_trajectory_matches_scipy(hlc, f, x0, step, iters):
    # with the same initial simplex, k iterations of both give the same best
    # vertex (no size stop: tolerance 0); SciPy counts its iterations from 1,
    # so its maxiter = k + 1 runs k steps
    x0 = np.array(x0, dtype=float)
    x, fx, it = hlc.nelder_mead(f, x0, step, size_tol=0.0, max_iter=iters)
    sim = np.vstack([x0] + [x0 + s * e for s, e in zip(step, np.eye(len(x0)))])
    r = scipy_optimize.minimize(f, x0, method="Nelder-Mead",
                                options=dict(initial_simplex=sim, maxiter=iters + 1, maxfev=10 ** 9, xatol=0.0,
                                             fatol=0.0, adaptive=False))
    assert it == iters
    # the reflected / expanded points are formed in a different but equal
    # algebraic form (c + a (c - x) against (1 + a) c - a x): equal to rounding
    np.testing.assert_allclose(x, r.x, rtol=1e-10, atol=1e-13)
    assert fx == pytest.approx(r.fun, rel=1e-9, abs=1e-300)


def test_converges_to_known_minima(hlc):
    x, fx, it = hlc.nelder_mead(rosen, [-1.2, 1.0], [0.1, 0.1], size_tol=1e-10, max_iter=2000)
    np.testing.assert_allclose(x, [1.0, 1.0], atol=1e-6)
    assert it < 2000
    x, fx, it = hlc.nelder_mead(quad3, [0.6, 0.1, 1.2], [0.02, 0.04, 0.01], size_tol=1e-9, max_iter=2000)
    np.testing.assert_allclose(x, [0.5, 0.0864, 1.0], atol=1e-6)


def test_size_tolerance_stops_early_and_nan_is_worst(hlc):
    calls = []

    def f(x):
        calls.append(x.copy())
        return np.nan if x[0] < -5 else quad3(x)

    x, fx, it = hlc.nelder_mead(f, [0.6, 0.1, 1.2], [0.02, 0.04, 0.01], size_tol=1e-3, max_iter=500)
    assert it < 500 and np.isfinite(fx)
    # a NaN vertex never becomes the best
    x, fx, it = hlc.nelder_mead(lambda x: np.nan if x[0] > 0.3 else (x[0] - 0.2) ** 2, [0.0], [0.35],
                                size_tol=1e-8, max_iter=300)
    assert x[0] == pytest.approx(0.2, abs=1e-6)


def test_default_fit_options_are_the_listing_settings(hlc):
    o = hlc.fit_opts()
    assert list(o.step) == [0.02, 0.04, 0.01]
    assert o.size_tol == 1e-5 and o.max_iter == 200 and o.free_mask == 7
