"""Summary of a dataflow factorisation timeline (HLC_FACTOR_TRACE=<path>).

Usage: python -m paper_1709_08625_gb300.factor_trace <path> [--top N]

Reads the file the library writes after a dependency-driven H-Cholesky and
prints where the time went: per op type the count, the run time (ready to
done) and the wait for producers (taken to ready); the share of CTA time
spent running ops; and the critical path, followed back from the last op to
finish through the producer whose signal released each op, split into run
time per op type, signal latency (producer done to consumer ready) and
ticket delay (the consumer's producers were done before any CTA took it).
"""
import argparse
import sys

import numpy as np

NAMES = {0: "potrf", 1: "trsm", 2: "gemm", 3: "trunc", 4: "trunc_group"}
TRACE = np.dtype([("t_take", "<u8"), ("t_ready", "<u8"), ("t_done", "<u8"), ("cta", "<u4"), ("releaser", "<i4")])


def load(path):
    with open(path, "rb") as f:
        if f.read(8) != b"HLCFTR01":
            raise ValueError(f"{path}: not a factorisation trace")
        nops = int(np.frombuffer(f.read(8), "<i8")[0])
        meta = np.frombuffer(f.read(24 * nops), "<i4").reshape(nops, 6)
        tr = np.frombuffer(f.read(TRACE.itemsize * nops), TRACE)
    if tr.shape[0] != nops:
        raise ValueError(f"{path}: truncated")
    return meta, tr


def summarise(meta, tr, top=10, out=sys.stdout):
    t0 = tr["t_take"].min()
    take = (tr["t_take"] - t0).astype(np.float64) * 1e-6  # ms
    ready = (tr["t_ready"] - t0).astype(np.float64) * 1e-6
    done = (tr["t_done"] - t0).astype(np.float64) * 1e-6
    run = done - ready
    wait = ready - take
    span = done.max()
    ncta = int(tr["cta"].max()) + 1
    typ = meta[:, 0]
    p = lambda *a: print(*a, file=out)
    p(f"ops {len(tr)}, CTAs {ncta}, makespan {span:.2f} ms")
    p(f"CTA time running ops {run.sum() / (span * ncta):.1%}, waiting for producers {wait.sum() / (span * ncta):.1%}")
    p(f"{'type':12s} {'ops':>9s} {'run ms':>10s} {'share':>6s} {'us/op':>8s} {'wait ms':>10s} {'us/op':>8s}")
    for t in sorted(NAMES):
        s = typ == t
        if not s.any():
            continue
        p(f"{NAMES[t]:12s} {s.sum():9d} {run[s].sum():10.1f} {run[s].sum() / run.sum():6.1%} "
          f"{1e3 * run[s].mean():8.2f} {wait[s].sum():10.1f} {1e3 * wait[s].mean():8.2f}")
    # critical path through the releasing producers
    path = []
    i = int(np.argmax(done))
    while i >= 0 and len(path) < len(tr):
        path.append(i)
        i = int(tr["releaser"][i])
    path = np.array(path[::-1])
    rel = tr["releaser"][path]
    crun = run[path]
    prev_done = np.where(rel >= 0, done[np.maximum(rel, 0)], 0.0)
    ticket = np.maximum(take[path] - prev_done, 0.0)
    signal = ready[path] - np.maximum(take[path], prev_done)
    p(f"critical path: {len(path)} ops, {span:.2f} ms = run {crun.sum():.2f} + signal {signal.sum():.2f} "
      f"+ ticket {ticket.sum():.2f} ms (first op ready at {ready[path[0]]:.2f} ms)")
    for t in sorted(NAMES):
        s = typ[path] == t
        if s.any():
            p(f"  {NAMES[t]:12s} {s.sum():7d} ops  run {crun[s].sum():9.2f} ms  {1e3 * crun[s].mean():8.2f} us/op")
    # the longest ops on the path
    order = np.argsort(-crun)[:top]
    p(f"longest ops on the critical path (type: sizes, run us):")
    for k in order:
        o = path[k]
        p(f"  {NAMES.get(int(typ[o]), typ[o])}: {meta[o, 1:].tolist()} {1e3 * run[o]:.1f}")
    # truncations by size class
    s = (typ == 3) | ((typ == 4) & (meta[:, 1] == 0))
    if s.any():
        mn = meta[s, 2] + meta[s, 3]
        K = meta[s, 4]
        p("truncations by rows m + n and term columns: count, mean run us")
        for lo, hi in ((0, 256), (256, 1024), (1024, 4096), (4096, 1 << 30)):
            for klo, khi in ((0, 33), (33, 65), (65, 1 << 30)):
                q = (mn >= lo) & (mn < hi) & (K >= klo) & (K < khi)
                if q.any():
                    p(f"  m+n [{lo}, {hi}) cols [{klo}, {khi}): {q.sum():8d} {1e3 * run[s][q].mean():9.1f}")
    # ops running over time
    edges = np.linspace(0.0, span, 21)
    busy = []
    for a, b in zip(edges[:-1], edges[1:]):
        ov = np.clip(np.minimum(done, b) - np.maximum(ready, a), 0.0, None).sum()
        busy.append(ov / (b - a))
    p("mean ops running per 5 % of the makespan: " + " ".join(f"{x:.0f}" for x in busy))
    return dict(makespan_ms=span, path_ops=len(path), path_run_ms=float(crun.sum()),
                path_signal_ms=float(signal.sum()), path_ticket_ms=float(ticket.sum()))


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("path")
    ap.add_argument("--top", type=int, default=10)
    a = ap.parse_args(argv)
    meta, tr = load(a.path)
    summarise(meta, tr, a.top)


if __name__ == "__main__":
    main()
