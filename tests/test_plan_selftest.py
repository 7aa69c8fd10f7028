"""The planner's dataflow programs on the host (hlc_selftest_plans, no GPU):
on synthetic trees over index intervals, every plan stays inside its
buffers, every dependency edge points forward with matching predecessor
counts, group truncations are consecutive parts with edges on the first, the
ready list is the ops without producers, joined products write their TRSM's
rows and run once, and a model of the factorisation kernel's ready-queue
protocol (as few as 9 CTAs for 8-part groups) runs every op after its
producers and finishes."""
import pytest


@pytest.fixture(scope="module")
def hlc():
    from paper_1709_08625_gb300 import build

    build.build()
    from paper_1709_08625_gb300 import hlc as h

    return h


# geometry 1: a Morton-numbered square grid (the block structure of spread
# points); geometry 0: index intervals (sparser, deeper trees)
@pytest.mark.parametrize("n,leaf,eta,kmax,ctas,seed,geometry", [
    (2000, 32, 2.0, 64, 16, 1, 1),
    (16384, 64, 2.0, 64, 304, 2, 1),
    (12000, 64, 2.0, 64, 9, 3, 1),      # the fewest CTAs the kernel accepts with groups of 8
    (3001, 16, 4.0, 32, 12, 5, 1),      # ragged sizes, weaker admissibility
    (40000, 64, 1.0, 128, 64, 4, 0),
    (20000, 64, 2.0, 64, 9, 6, 0),
])
def test_plan_invariants(hlc, n, leaf, eta, kmax, ctas, seed, geometry):
    st, msg, s = hlc.selftest_plans(n, leaf, eta, kmax, ctas, seed, geometry=geometry)
    assert st == hlc.HLC_OK, msg
    assert s["factor_ops"] > 0 and s["factor_edges"] >= s["factor_ops"] - 1
    assert s["ready0"] >= 1
    # one neighbour product joins the TRSM of (almost) every diagonal leaf
    assert s["fwd_joins"] == s["bwd_joins"] > 0
    assert s["model_makespan"] > 0
    if n >= 12000:
        assert s["groups"] > 0  # targets above 4096 rows run as 8-part groups


def test_model_with_different_durations_and_grids(hlc):
    # the same plans under other op durations and grid sizes
    for seed, ctas in ((11, 9), (12, 10), (13, 152)):
        st, msg, _ = hlc.selftest_plans(8192, 64, 2.0, 64, ctas, seed)
        assert st == hlc.HLC_OK, msg


def test_arguments_are_checked(hlc):
    assert hlc.selftest_plans(1000, 32, 2.0, 64, 8, 1)[0] == hlc.HLC_ERR_ARG   # groups of 8 need > 8 CTAs
    assert hlc.selftest_plans(1000, 0, 2.0, 64, 16, 1)[0] == hlc.HLC_ERR_ARG
    assert hlc.selftest_plans(1000, 32, 2.0, 0, 16, 1)[0] == hlc.HLC_ERR_ARG
    assert hlc.selftest_plans(1, 32, 2.0, 64, 16, 1)[0] == hlc.HLC_ERR_ARG
