"""The factorisation timeline reader (HLC_FACTOR_TRACE) on a hand-made
trace: file layout, per-type sums and the critical path."""
import io

import numpy as np

from paper_1709_08625_gb300 import factor_trace as ft


def write_trace(path, meta, rows):
    tr = np.array(rows, dtype=ft.TRACE)
    with open(path, "wb") as f:
        f.write(b"HLCFTR01")
        f.write(np.int64(len(rows)).tobytes())
        f.write(np.asarray(meta, dtype="<i4").tobytes())
        f.write(tr.tobytes())


def test_trace_summary(tmp_path):
    ms = 1_000_000  # ns per ms
    # op 0: potrf, no producer, ready at 0, done at 10 ms (CTA 0)
    # op 1: trsm released by 0, taken at 5, ready at 11, done at 20 (CTA 1)
    # op 2: gemm, no producer, 0 .. 4 (CTA 1)
    # op 3: trunc released by 1, taken at 25 (ticket delay 5), done at 40 (CTA 0)
    meta = [[0, 0, 64, 0, 0, 0], [1, 0, 64, 8, 0, 0], [2, 0, 64, 8, 8, 0], [3, 0, 100, 200, 40, 7]]
    rows = [(0, 0, 10 * ms, 0, -1), (5 * ms, 11 * ms, 20 * ms, 1, 0), (0, 0, 4 * ms, 1, -1),
            (25 * ms, 25 * ms, 40 * ms, 0, 1)]
    p = tmp_path / "t.bin"
    write_trace(p, meta, rows)
    m, tr = ft.load(p)
    assert m.shape == (4, 6) and tr["releaser"].tolist() == [-1, 0, -1, 1]
    out = io.StringIO()
    r = ft.summarise(m, tr, out=out)
    assert r["makespan_ms"] == 40.0
    assert r["path_ops"] == 3  # 0 -> 1 -> 3
    assert r["path_run_ms"] == 10.0 + 9.0 + 15.0
    assert r["path_signal_ms"] == 1.0  # op 1 ready 1 ms after op 0 finished
    assert r["path_ticket_ms"] == 5.0  # op 3 taken 5 ms after op 1 finished
    text = out.getvalue()
    assert "potrf" in text and "trunc" in text and "critical path: 3 ops" in text


def test_trace_rejects_other_files(tmp_path):
    p = tmp_path / "x.bin"
    p.write_bytes(b"NOTATRACE" + bytes(64))
    try:
        ft.load(p)
    except ValueError:
        return
    raise AssertionError("accepted a file without the trace header")
