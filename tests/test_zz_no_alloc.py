"""hlc_matvec_noalloc: the matvec from a fixed buffer, without allocating.

It must give hlc_matvec's result bit for bit, call after call, and refuse
what it cannot serve (host pointers, a tree whose matvec plan does not exist
yet).  The file runs last in a full session and also passes on its own.
"""
import numpy as np
import pytest

from paper_1709_08625_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hlc():
    from paper_1709_08625_gb300 import build

    build.build()
    from paper_1709_08625_gb300 import hlc as h

    return h


def test_noalloc_matvec_matches_matvec_on_consecutive_calls(hlc):
    torch = pytest.importorskip("torch")
    n = 5000
    ctx = hlc.Context(0)
    try:
        t = ctx.build_tree(inputs.points(n, 7001), leaf=64, eps=1e-7, kmax=64)
        C = t.assemble(hlc.theta(1.0, 0.08, 0.5, 1e-4))
        x = inputs.normal(n, 7002)
        xd = torch.tensor(x, device="cuda:0")
        yd = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda:0")
        # no matvec plan on this tree yet: refused, nothing run
        with pytest.raises(hlc.HlcError) as e:
            C.matvec_noalloc(xd, yd)
        assert e.value.status == hlc.HLC_ERR_STATE
        ref = C.matvec(x)  # the existing entry point; builds the plan
        assert hlc.hlc_matvec_noalloc_capacity() == 8 << 20
        outs = []
        for call in range(2):
            yd.fill_(float("nan"))
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info(0)[0]
            C.matvec_noalloc(xd, yd)
            torch.cuda.synchronize()
            if call == 1:  # the first call may load the module and its buffer
                assert torch.cuda.mem_get_info(0)[0] == free0
            outs.append(yd.cpu().numpy())
        for y in outs:
            assert np.array_equal(y, ref)
        # host pointers are refused
        with pytest.raises(hlc.HlcError) as e:
            C.matvec_noalloc(x, np.empty_like(x))
        assert e.value.status == hlc.HLC_ERR_ARG
    finally:
        ctx.close()
