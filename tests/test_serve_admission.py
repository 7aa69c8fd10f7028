"""The serve loop's admission rule, replayed on the host (no GPU).

Requests are admitted in arrival order when a slot is free and their
estimated device footprint fits in what is left of the budget; a request
larger than the whole budget runs alone.  The replay runs the same rule
object the slot workers use, against fake footprints and durations.
"""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def hlc():
    from paper_1709_08625_gb300 import build

    build.build()
    from paper_1709_08625_gb300 import hlc as h

    return h


def _check_schedule(start, fp, du, budget, slots):
    # at every admission time, what runs (admitted, not finished) fits
    n = len(fp)
    for i in range(n):
        t = start[i]
        running = [j for j in range(n) if start[j] <= t < start[j] + du[j] or j == i]
        assert len(running) <= slots
        tot = sum(fp[j] for j in running)
        assert tot <= budget or len(running) == 1, (i, tot, budget)
    # arrival order is kept
    assert np.all(np.diff(start) >= 0)


@pytest.mark.parametrize("seed", range(6))
def test_admission_never_exceeds_budget(hlc, seed):
    rng = np.random.default_rng(seed)
    n = 200
    budget = 64 << 30
    fp = rng.integers(1 << 28, 40 << 30, n).astype(np.uint64)
    du = rng.exponential(1.0, n)
    for slots in (1, 3, 8):
        start, peak = hlc.admission_replay(budget, slots, fp, du)
        assert peak <= budget
        _check_schedule(start, fp.astype(float), du, budget, slots)


def test_oversized_request_runs_alone(hlc):
    budget = 10 << 30
    fp = np.array([4 << 30, 30 << 30, 4 << 30, 4 << 30], dtype=np.uint64)
    du = np.array([1.0, 2.0, 1.0, 1.0])
    start, peak = hlc.admission_replay(budget, 4, fp, du)
    # the 30 GB request waits for the first to finish, then runs alone
    assert start[1] == pytest.approx(1.0)
    assert start[2] == pytest.approx(3.0) and start[3] == pytest.approx(3.0)
    assert peak == 30 << 30


def test_slots_limit_concurrency(hlc):
    fp = np.full(10, 1 << 20, dtype=np.uint64)
    du = np.ones(10)
    start, peak = hlc.admission_replay(1 << 40, 3, fp, du)
    np.testing.assert_allclose(start, [0, 0, 0, 1, 1, 1, 2, 2, 2, 3])
    assert peak == 3 << 20


def test_footprint_grows_with_n_and_kmax(hlc):
    a = hlc.serve_footprint(65536, kmax=64)
    b = hlc.serve_footprint(131072, kmax=64)
    c = hlc.serve_footprint(65536, kmax=128)
    assert 2 * a < b * 1.3 and b > 2 * a * 0.9
    assert c > 1.7 * a
    assert hlc.serve_footprint(0) == 0


def test_replay_rejects_bad_arguments(hlc):
    with pytest.raises(hlc.HlcError):
        hlc.admission_replay(0, 1, [1], [1.0])
    with pytest.raises(hlc.HlcError):
        hlc.admission_replay(10, 0, [1], [1.0])
    with pytest.raises(hlc.HlcError):
        hlc.admission_replay(10, 1, [1], [-1.0])
