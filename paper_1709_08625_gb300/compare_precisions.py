"""One named workload in several precisions: a warm evaluation (it builds the
plans and workspaces) and then a timed one per precision, printed as one
JSON line per workload with the mixed-vs-FP64 differences of L and log det
per location.

Usage: python -m paper_1709_08625_gb300.compare_precisions [--precisions mixed,fp64] [--n N] WORKLOAD...

Workloads are the names of inputs.WORKLOADS (e.g. n65536_nu1.5_eps1e-6,
n524288_nu0.5_eps1e-7).  The rank capacity is 128 for nu > 1 (smooth
kernels reach ranks above 64 at eps = 1e-6) and 64 otherwise.
"""
import argparse
import json
import time

from . import build, inputs

KEYS = ("loglik", "logdet", "quad", "refine_iters", "est_rel_err", "ms_assemble", "ms_factor", "ms_solve",
        "max_rank_C", "max_rank_L", "bytes_C", "bytes_L")


def run(names, precisions=("mixed", "fp64"), device=0, first=0):
    from . import hlc

    modes = {"mixed": hlc.HLC_MIXED, "fp64": hlc.HLC_FP64, "mixed_svd64": hlc.HLC_MIXED_SVD64}
    c = hlc.Context(device)
    out = []
    try:
        for name in names:
            w = inputs.WORKLOADS[name]
            xy, z = inputs.workload_points(name), inputs.workload_normal(name)
            if first > 0:  # a smaller case: the workload's first locations
                xy, z = xy[:first], z[:first]
            n = len(z)
            th = hlc.theta(w["sigma2"], w["ell"], w["nu"], w["nugget"])
            res = {"workload": name, "n": n}
            for pn in precisions:
                t0 = time.perf_counter()
                try:
                    t = c.build_tree(xy, leaf=w["leaf"], eta=w["eta"], eps=w["eps"], precision=modes[pn],
                                     kmax=128 if w["nu"] > 1 else 64)
                    try:
                        t.loglik(th, z)
                        first_s = time.perf_counter() - t0
                        r = t.loglik(th, z)
                    finally:
                        t.free()
                    res[pn] = {k: r[k] for k in KEYS}
                    res[pn]["first_call_s"] = first_s
                except hlc.HlcError as e:
                    res[pn] = {"err": str(e)}
            if "loglik" in res.get("mixed", {}) and "loglik" in res.get("fp64", {}):
                res["dL_per_n"] = abs(res["mixed"]["loglik"] - res["fp64"]["loglik"]) / n
                res["dlogdet_per_n"] = abs(res["mixed"]["logdet"] - res["fp64"]["logdet"]) / n
            out.append(res)
            print(json.dumps(res), flush=True)
    finally:
        c.close()
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("workloads", nargs="+", choices=sorted(inputs.WORKLOADS))
    ap.add_argument("--precisions", default="mixed,fp64")
    ap.add_argument("--n", type=int, default=0, help="take the workload's first N locations (0: all)")
    a = ap.parse_args(argv)
    build.build()
    run(a.workloads, tuple(p for p in a.precisions.split(",") if p), first=a.n)


if __name__ == "__main__":
    main()
