#!/usr/bin/env python
"""Throughput of the H-matrix Gaussian log-likelihood on GB300.

One step = one likelihood evaluation (arXiv:1709.08625, eq. 2) at
n = 524,288 uniform locations in [0,1]^2 on an existing tree: Matern assembly
(dense leaves + ACA + recompression), H-Cholesky, log det, forward solve and
the FP64 preconditioned-CG quadratic form.  theta varies by +-5 % (sigma2,
ell) from step to step.  The working set (tens of GB of H-matrix storage) is
far larger than L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU runs (torchrun, one rank per GPU) are replicas: every rank runs its
own evaluations on its own GPU; value = evaluations of all ranks / max time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "loglik evals/s at n=512k (mixed vs FP64, |ΔL|/n≤1e-6); serve p50/p99 ms"
UNIT = "evals/s"
WORKLOAD = "n524288_nu0.5_eps1e-5"
SAMPLE_N = 32768  # oracle sample: the first SAMPLE_N locations of the workload (~Table 5's smallest n)
FP32_LANES_PER_SM = 128
NUM_SMS = 152
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one k_factor
# launch of the mixed-precision workload, from one ncu capture of the kernel
# as it is now (one pass, the first of the two factorisations):
#   python -m paper_1709_08625_gb300.compare_precisions --precisions mixed n524288_nu0.5_eps1e-5 &&
#   ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum --clock-control none -k regex:k_factor -c 1 \
#       python -m paper_1709_08625_gb300.compare_precisions --precisions mixed n524288_nu0.5_eps1e-5
# None where no capture of the current kernel exists.
K_FACTOR_TRAFFIC = {"n524288_nu0.5_eps1e-5": 144.41e9 + 156.48e9}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default=WORKLOAD)
    p.add_argument("--precision", default="mixed", choices=["mixed", "mixed_svd64", "fp64"])
    p.add_argument("--no-fp64-check", action="store_true")
    p.add_argument("--fp64-steps", type=int, default=2, help="timed FP64 evaluations (after one warm-up)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--kmax", type=int, default=64)
    p.add_argument("--no-serve", action="store_true")
    p.add_argument("--no-profiled-pass", action="store_true",
                   help="skip the pass that times every op launch by type (e.g. for an ncu launch list)")
    p.add_argument("--serve-requests", type=int, default=16)
    p.add_argument("--serve-n", type=int, nargs=2, default=[10000, 65536])
    p.add_argument("--sample-n", type=int, default=SAMPLE_N,
                   help="locations in the oracle's bounded sample of the workload")
    return p.parse_args()


# --------------------------------------------------------------------------
# distributed plumbing (replicas)
# --------------------------------------------------------------------------
def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, 0, None
    import torch
    import torch.distributed as dist

    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    backend = "nccl" if torch.cuda.is_available() else "gloo"
    if backend == "nccl":
        torch.cuda.set_device(local)
    dist.init_process_group(backend=backend)
    return rank, ws, local, dist


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, v):
    if dist is None:
        return v
    import torch

    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            if len(r) >= 9:
                for nm, v in zip(names, r[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# CPU baseline: the oracle on a bounded sample of the workload
# --------------------------------------------------------------------------
def oracle_sample(name, n_sample):
    """One oracle evaluation (tree, assembly, H-Cholesky, log det, solve and
    PCG) on the first n_sample locations of the workload, timed as it runs;
    nothing is rescaled."""
    import oracle
    from paper_1709_08625_gb300 import inputs

    w = inputs.WORKLOADS[name]
    xy = inputs.workload_points(name)[:n_sample]
    z = inputs.workload_normal(name)[:n_sample]
    t0 = time.perf_counter()
    r = oracle.h_loglik(xy, z, w["sigma2"], w["ell"], w["nu"], w["nugget"], w["eps"], leaf=w["leaf"], eta=w["eta"])
    dt = time.perf_counter() - t0
    return {"value": 1.0 / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"one CPU H-oracle evaluation (tree, assembly, H-Cholesky, log det, solve, PCG) on the first "
                      f"{n_sample} locations of the {name} workload, same theta, eps and leaf; measured at "
                      f"n={n_sample}, not rescaled", "n": n_sample, "seconds": dt, "loglik": r["loglik"]}


def run_reference(args, rank, ws, dist):
    if rank != 0:
        return 0
    import oracle

    oracle.build()
    times = []
    last = None
    for _ in range(args.warmup):
        oracle_sample(args.workload, args.sample_n)
    for _ in range(args.steps):
        last = oracle_sample(args.workload, args.sample_n)
        times.append(last["seconds"])
    ms = 1000.0 * statistics.mean(times)
    v = 1000.0 / ms
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload, "n": args.sample_n, "measured_at_n": args.sample_n,
                      "note": f"the oracle is timed on the first {args.sample_n} locations of the workload (one "
                              "evaluation per step); value and ms_per_step are that measurement, not rescaled"},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": last["cores"], "kind": "oracle",
                            "sample": last["sample"]},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


# --------------------------------------------------------------------------
# served stream: p50 / p99 latency under Poisson arrivals
# --------------------------------------------------------------------------
def serve_stream(hlc, inputs, dev, n_lo, n_hi, n_req, slots, seed=5000):
    """Requests with n log-uniform in [n_lo, n_hi], sigma2 ~ U[0.5, 2],
    ell ~ U[0.02, 0.2], nu ~ U[0.3, 2.0], nugget 1e-4, z ~ N(0, 1), mixed
    precision with FP64 refinement.  A closed-loop pass (all requests at once)
    measures the capacity; the timed pass submits the same requests as Poisson
    arrivals at 0.8 x that capacity.  Latency = submission to completion,
    tree build included, as the library records it."""
    import numpy as np

    rng = np.random.default_rng(seed)
    reqs = []
    for q in range(n_req):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        th = hlc.theta(float(rng.uniform(0.5, 2.0)), float(rng.uniform(0.02, 0.2)), float(rng.uniform(0.3, 2.0)),
                       1e-4)
        reqs.append((inputs.points(n, seed + 1 + q), inputs.normal(n, seed + 1001 + q), th))
    kw = dict(leaf=64, eps=1e-6, kmax=128, precision=hlc.HLC_MIXED)
    ctx = hlc.Context(dev)
    ctx.serve_start(96 << 30, slots)

    errors = []

    def drain(ids, t_limit=900.0):
        done, failed = {}, 0
        t0 = time.perf_counter()
        while len(done) + failed < len(ids) and time.perf_counter() - t0 < t_limit:
            for i in ids:
                if i in done or i < 0:
                    continue
                try:
                    r = ctx.serve_poll(i)
                except hlc.HlcError as e:
                    errors.append(hlc.ERRORS.get(e.status, e.status))
                    failed += 1
                    ids[ids.index(i)] = -1
                    continue
                if r is not None:
                    done[i] = r
            time.sleep(0.002)
        return done, failed

    t0 = time.perf_counter()
    ids = [ctx.serve_submit(xy, z, th, **kw) for xy, z, th in reqs]
    drain(ids)
    capacity = n_req / (time.perf_counter() - t0)
    rate = 0.8 * capacity
    gaps = rng.exponential(1.0 / rate, n_req)
    errors.clear()  # count the timed pass only
    t0 = time.perf_counter()
    ids, due = [], t0
    for (xy, z, th), g in zip(reqs, gaps):
        due += g
        while time.perf_counter() < due:
            time.sleep(0.001)
        ids.append(ctx.serve_submit(xy, z, th, **kw))
    done, failed = drain(ids)
    span = time.perf_counter() - t0
    ctx.serve_stop()
    ctx.close()
    lat = sorted(r["ms_total"] for r in done.values())

    def pct(p):
        if not lat:
            return None
        return lat[min(len(lat) - 1, int(math.ceil(p / 100.0 * len(lat))) - 1)]

    return {"p50_ms": pct(50), "p99_ms": pct(99), "evals_per_s": len(lat) / span, "requests": n_req,
            "completed": len(lat), "failed": failed, "errors": errors, "n_range": [n_lo, n_hi], "slots": slots,
            "arrival_rate_per_s": rate, "closed_loop_capacity_per_s": capacity,
            "note": "Poisson arrivals at 0.8 x closed-loop capacity; mixed precision, eps 1e-6, leaf 64"}


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------
def run_ours(args, rank, ws, local, dist):
    import numpy as np
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_1709_08625_gb300 import hlc, inputs

    dev = local
    torch.cuda.set_device(dev)
    w = inputs.WORKLOADS[args.workload]
    n = w["n"]
    xy = inputs.workload_points(args.workload)
    z_host = inputs.workload_normal(args.workload)
    prec = {"mixed": hlc.HLC_MIXED, "mixed_svd64": hlc.HLC_MIXED_SVD64, "fp64": hlc.HLC_FP64}[args.precision]
    ctx = hlc.Context(dev)
    t0 = time.perf_counter()
    tree = ctx.build_tree(xy, leaf=w["leaf"], eta=w["eta"], eps=w["eps"], precision=prec, kmax=args.kmax)
    tree_s = time.perf_counter() - t0
    z_dev = torch.tensor(z_host, device=f"cuda:{dev}")
    z_pin = torch.tensor(z_host).pin_memory()
    stream = torch.cuda.ExternalStream(ctx.stream(), device=f"cuda:{dev}")

    def theta(k):
        j = inputs.theta_jitter(w, k)
        return hlc.theta(j["sigma2"], j["ell"], w["nu"], w["nugget"])  # nu fixed: same kernel class

    first = time.perf_counter()
    for k in range(args.warmup):
        tree.loglik(theta(k), z_dev)
    warm_s = time.perf_counter() - first

    # ---- timed region: device time on the library stream --------------------
    ctx.set_profiling(False)
    ctx.counters(reset=True)
    clocks = ClockSampler(dev)
    clocks.start()
    barrier(dist)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    results = []
    for k in range(args.steps):
        results.append(tree.loglik(theta(1000 + k), z_dev))
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(dist)
    clk = clocks.stop()
    ms_total = ev0.elapsed_time(ev1)
    cnt = ctx.counters(reset=True)
    ms_total = max_over_ranks(dist, ms_total)
    value = ws * args.steps / (ms_total / 1000.0)

    # ---- profiled pass (one step): every op launch timed with CUDA events ---
    # (the waves' launches by op type, for the per-type breakdown)
    prof, prof_ms = {}, None
    if not args.no_profiled_pass:
        ctx.set_profiling(True)
        torch.cuda.synchronize()
        pe0 = torch.cuda.Event(enable_timing=True)
        pe1 = torch.cuda.Event(enable_timing=True)
        pe0.record(stream)
        tree.loglik(theta(1000), z_dev)
        pe1.record(stream)
        torch.cuda.synchronize()
        prof = ctx.counters(reset=True)
        ctx.set_profiling(False)
        prof_ms = pe0.elapsed_time(pe1)

    # ---- the dominant kernel: one H-Cholesky (k_factor) timed alone ---------
    # algorithmic flops counted by its ops, over the CUDA-event time of the
    # hlc_cholesky call on the library stream
    Cm = tree.assemble(theta(1000))
    torch.cuda.synchronize()
    ctx.counters(reset=True)
    fe0 = torch.cuda.Event(enable_timing=True)
    fe1 = torch.cuda.Event(enable_timing=True)
    fe0.record(stream)
    Lm = tree.cholesky(Cm)
    fe1.record(stream)
    torch.cuda.synchronize()
    fcnt = ctx.counters(reset=True)
    factor_ms = fe0.elapsed_time(fe1)
    factor_flops = sum(fcnt[k]["flops"] for k in ("potrf", "trsm", "gemm", "trunc", "trunc_cluster"))
    factor_kernel = "k_factor" if fcnt["persistent"] >= 1 else "wave launches"
    Lm.free()
    Cm.free()

    # ---- end to end through the public API with host buffers ---------------
    # (a step is ~50 s at the default workload: one step per rank suffices)
    e2e_steps = min(args.steps, 1) if args.steps > 0 else 0
    t0 = time.perf_counter()
    e2e_res = results[-1] if results else None
    for k in range(e2e_steps):
        e2e_res = tree.loglik(theta(1000 + k), z_pin.numpy())
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(dist, time.perf_counter() - t0)
    e2e_value = ws * e2e_steps / e2e_s if e2e_steps else None
    info = tree.info()
    iters = e2e_res["refine_iters"]
    # bytes read back per evaluation: scalars of the solve, status words and
    # the two rank arrays for the storage statistics
    d2h = 8 * (8 + 3 * iters) + 8 * 3 + 2 * 4 * info["lowrank"]

    out = {}
    if rank == 0:
        # per op type, from the profiled pass (every launch timed)
        ops = {k: v for k, v in prof.items() if isinstance(v, dict)}
        sm_mhz = clk.get("sm_max_mhz") or 2070.0
        if args.precision != "fp64":
            # FP32 SIMT: the mixed factorisation's panels, products and cores
            peak = NUM_SMS * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
        else:
            peak = 1.25  # nominal FP64 rate of GB300
        unit = "TFLOP/s"
        achieved = factor_flops / (factor_ms / 1000.0) / 1e12 if factor_ms > 0 else 0.0
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32+f64",
            "data": "synthetic: seeded uniform locations in [0,1]^2, z ~ N(0,1); theta +-5 % per step",
            "config": {"workload": args.workload, "n": n, "nu": w["nu"], "ell": w["ell"], "sigma2": w["sigma2"],
                       "nugget": w["nugget"], "eps": w["eps"], "leaf": w["leaf"], "eta": w["eta"],
                       "precision": args.precision, "kmax": args.kmax,
                       "l2": "no flush: H-matrix working set of several GB > 129 MB L2",
                       "parallelism": f"replicas x{ws}", "tree_build_s": tree_s, "warmup_s": warm_s,
                       "plan_ops": info["plan_ops"], "plan_waves": info["plan_waves"]},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": d2h,
                    "steps": e2e_steps},
            "gpu_launches": int(cnt["launches"]),
            "roofline": {"bound": "alu", "kernel": factor_kernel, "achieved": achieved, "peak": peak, "unit": unit,
                         "frac": achieved / peak if peak else None,
                         "traffic": K_FACTOR_TRAFFIC.get(args.workload) if args.precision == "mixed" else None,
                         "launch_ms": factor_ms, "launch_gflop": factor_flops / 1e9,
                         "note": "one H-Cholesky at the workload: algorithmic flops counted by its ops (POTRF "
                                 "n^3/3, TRSM n^2 c, GEMM 2mkc, truncation 2K^2(m+n) + 2Kk(m+n) per batch) over "
                                 "the CUDA-event time of the hlc_cholesky call on the library stream",
                         "peak_note": ("FP32 SIMT: 152 SMs x 128 lanes x 2 flop x max SM clock (derived)"
                                       if peak > 2 else "nominal FP64 rate of GB300"),
                         "profiled_ms_per_step": prof_ms,
                         "per_op_type_profiled_pass": {k: v for k, v in ops.items()}},
            "clocks": clk,
            "result": {k: results[-1][k] for k in ("loglik", "logdet", "quad", "refine_iters", "rel_residual",
                                                   "est_rel_err",
                                                   "max_rank_C", "max_rank_L", "bytes_C", "bytes_L",
                                                   "ms_assemble", "ms_factor", "ms_solve")},
        }
    # ---- FP64 comparison at the same theta ---------------------------------
    # warm: one evaluation builds the FP64 tree's plans, workspaces and graphs
    # (and tunes the solve kernel's grid), then fp64_steps timed evaluations
    # on the library stream
    if rank == 0 and not args.no_fp64_check and args.precision != "fp64":
        del tree
        t64 = ctx.build_tree(xy, leaf=w["leaf"], eta=w["eta"], eps=w["eps"], precision=hlc.HLC_FP64,
                             kmax=args.kmax)
        t64.loglik(theta(1000 + args.steps - 1), z_dev)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        r64s = [t64.loglik(theta(1000 + k), z_dev) for k in range(args.fp64_steps)]
        f1.record(stream)
        torch.cuda.synchronize()
        ms64 = f0.elapsed_time(f1) / max(args.fp64_steps, 1)
        # the mixed result at the same theta (the first timed step)
        r64, rm = r64s[0], results[0]
        out["fp64"] = {"value": 1000.0 / ms64, "unit": UNIT, "steps": args.fp64_steps, "warmup": 1,
                       "ms_per_step": ms64, "loglik": r64["loglik"], "ms_factor": r64["ms_factor"],
                       "ms_solve": r64["ms_solve"], "refine_iters": r64["refine_iters"]}
        out["parity"] = {"dL_per_n_mixed_vs_fp64": abs(rm["loglik"] - r64["loglik"]) / n,
                         "dlogdet_per_n": abs(rm["logdet"] - r64["logdet"]) / n,
                         "dquad_per_n": abs(rm["quad"] - r64["quad"]) / n, "bar": 1e-6,
                         "est_rel_err_mixed": rm["est_rel_err"], "est_rel_err_fp64": r64["est_rel_err"],
                         "speedup_mixed_vs_fp64": ms64 / (ms_total / args.steps)}
        del t64
    if rank == 0 and not args.no_serve:
        out["serve"] = serve_stream(hlc, inputs, dev, args.serve_n[0], args.serve_n[1], args.serve_requests, 3)
    if rank == 0:
        if not args.no_cpu_baseline:
            import oracle

            oracle.build()
            cb = oracle_sample(args.workload, args.sample_n)
            out["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample", "n", "seconds")}
            # the same sample on the GPU (a tree of the first sample_n
            # locations, same precision), for a comparison at equal n
            ts = ctx.build_tree(xy[: args.sample_n], leaf=w["leaf"], eta=w["eta"], eps=w["eps"], precision=prec,
                                kmax=args.kmax)
            zs = z_dev[: args.sample_n].contiguous()
            th_w = hlc.theta(w["sigma2"], w["ell"], w["nu"], w["nugget"])  # the oracle's theta
            for _ in range(2):
                ts.loglik(th_w, zs)
            torch.cuda.synchronize()
            s0 = torch.cuda.Event(enable_timing=True)
            s1 = torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            rs = ts.loglik(th_w, zs)
            s1.record(stream)
            torch.cuda.synchronize()
            gms = s0.elapsed_time(s1)
            out["cpu_baseline"]["gpu_same_sample"] = {
                "value": 1000.0 / gms, "unit": UNIT, "ms": gms,
                "dL_per_n_vs_oracle": abs(rs["loglik"] - cb["loglik"]) / args.sample_n,
                "speedup_vs_oracle": cb["seconds"] * 1000.0 / gms}
            del ts
        print(json.dumps(out), flush=True)
    ctx.close()
    return 0


def main():
    args = parse()
    rank, ws, local, dist = dist_setup(args)
    try:
        if args.impl == "reference":
            return run_reference(args, rank, ws, dist)
        return run_ours(args, rank, ws, local, dist)
    finally:
        if dist is not None:
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
