"""Parameter identification on synthetic data, the experiment of Sec. 5.

1. Z0 = L~ xi on n0 uniform locations in [0,1]^2 with the GPU H-Cholesky
   factor of C(theta*) (Sec. 5.1; hlc_sample), xi ~ N(0, I) seeded.
2. A random subsample of n of the n0 locations and their values (Sec. 5.1:
   every replicate is sampled from the same Z0).
3. The three-parameter Nelder-Mead fit of (nu, ell, sigma2) on the subsample
   from a start away from theta* (App. B settings; hlc_fit).

    python -m paper_1709_08625_gb300.identify --n0 524288 --n 65536

prints one JSON record.  theta* defaults to the paper's (ell, nu, sigma2) =
(0.0864, 0.5, 1.0) with the nugget 1e-4 of the App. B listing.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import hlc, inputs


def run(n0=524288, n=65536, seed=0, true=(1.0, 0.0864, 0.5), nugget=1e-4, start=None, eps=1e-6, leaf=64,
        precision="mixed", max_iter=200, size_tol=1e-5, device=0, trace=False, gen_precision=None):
    """Returns a dict: the true and identified theta, the fit's record and
    the wall times of the generation and the fit.  gen_precision: precision
    of the factor that draws Z0 (default: the fit's)."""
    modes = {"fp64": hlc.HLC_FP64, "mixed": hlc.HLC_MIXED, "mixed_svd64": hlc.HLC_MIXED_SVD64}
    prec = modes[precision]
    gprec = modes[gen_precision or precision]
    s2, ell, nu = true
    if start is None:
        start = (1.2 * s2, 1.25 * ell, 0.8 * nu)
    rng = np.random.default_rng(seed)
    xy0 = inputs.points(n0, seed + 1)
    xi = inputs.normal(n0, seed + 2)
    ctx = hlc.Context(device)
    try:
        t0 = time.perf_counter()
        tree0 = ctx.build_tree(xy0, leaf=leaf, eps=eps, precision=gprec)
        z0 = tree0.sample(hlc.theta(s2, ell, nu, nugget), xi)
        tree0.free()
        t_gen = time.perf_counter() - t0
        idx = np.sort(rng.choice(n0, size=n, replace=False)) if n < n0 else np.arange(n0)
        xy, z = xy0[idx], z0[idx]
        t0 = time.perf_counter()
        tree = ctx.build_tree(xy, leaf=leaf, eps=eps, precision=prec)
        st = hlc.theta(start[0], start[1], start[2], nugget)
        l_start = tree.loglik(st, z)["loglik"]
        r, tr = tree.fit(z, st, trace_cap=4 * max_iter + 16 if trace else 0, max_iter=max_iter,
                         size_tol=size_tol)
        t_fit = time.perf_counter() - t0
        # the likelihood at the true theta, for comparison with the maximum
        # found (on a ridge of nearly equal likelihood, sigma2 / ell^(2 nu)
        # is what the data fix best)
        l_true = tree.loglik(hlc.theta(s2, ell, nu, nugget), z)["loglik"]
        out = dict(n0=n0, n=n, seed=seed, eps=eps, leaf=leaf, precision=precision,
                   gen_precision=gen_precision or precision, nugget=nugget,
                   true=dict(sigma2=s2, ell=ell, nu=nu), start=dict(sigma2=start[0], ell=start[1], nu=start[2]),
                   estimate=dict(sigma2=r["sigma2"], ell=r["ell"], nu=r["nu"]), loglik_start=l_start,
                   loglik_true=l_true, fit=r,
                   microergodic=dict(true=s2 / ell ** (2 * nu), estimate=r["sigma2"] / r["ell"] ** (2 * r["nu"])),
                   seconds_generate=t_gen, seconds_fit=t_fit,
                   ms_per_eval=r["ms_total"] / max(r["evaluations"], 1))
        if trace:
            out["trace"] = tr.tolist()
        return out
    finally:
        ctx.close()


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--n0", type=int, default=524288)
    p.add_argument("--n", type=int, default=65536)
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--eps", type=float, default=1e-6)
    p.add_argument("--precision", default="mixed", choices=["fp64", "mixed", "mixed_svd64"])
    p.add_argument("--max-iter", type=int, default=200)
    a = p.parse_args()
    from . import build

    build.build()
    print(json.dumps(run(n0=a.n0, n=a.n, seed=a.seed, eps=a.eps, precision=a.precision, max_iter=a.max_iter)))


if __name__ == "__main__":
    main()
