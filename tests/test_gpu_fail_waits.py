"""The bounded-wait error path of the fast product, driven by the test hook
hub_test_fail_waits: pass 1 takes the exit a given-up mbarrier wait takes (device error flag
set, kernel returns) after its bulk copies have landed, so no wait runs out and no copy is in
flight; the small-sector Lanczos takes its given-up-barrier exit before any barrier.  The flag must surface as HUB_ERR_TIMEOUT from hub_check and hub_lanczos_ground, be
cleared once reported, and leave the handle usable."""
import numpy as np
import pytest

from paper_1307_7542_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def hub(cuda_ok):
    import __graft_entry__
    __graft_entry__.build()
    from paper_1307_7542_gb300 import hub as H
    return H


@pytest.mark.parametrize("small", [False, True])
def test_timeout_flag_reaches_the_caller(hub, small):
    """small: hub_lanczos_ground runs the single-launch small-sector solver, whose CTAs take
    the same exit before their first grid barrier; else the double-float driver."""
    w = W.ring8()
    m = hub.Hubbard(8, 4, 4, w["bonds"], w["t"], w["U"], w["eps"])
    if not small:
        hub.hub_set_small_dim(m.h, 0)
    try:
        x = torch.from_numpy(W.normal(5, m.D)).cuda()
        y_ref = m.apply(x)
        r_ref = m.ground(x, maxit=300, tol=1e-12)
        hub.hub_check(m.h)

        hub.hub_test_fail_waits(m.h, True)
        m.apply(x)                                    # enqueued; the flag is read by hub_check
        with pytest.raises(hub.HubError) as e:
            hub.hub_check(m.h)
        assert e.value.code == hub.HUB_ERR_TIMEOUT
        hub.hub_check(m.h)                            # reported once, then cleared
        with pytest.raises(hub.HubError) as e:
            m.ground(x, maxit=50, tol=1e-12)
        assert e.value.code == hub.HUB_ERR_TIMEOUT
        hub.hub_check(m.h)

        hub.hub_test_fail_waits(m.h, False)           # the handle works as before
        assert torch.equal(m.apply(x), y_ref)
        r = m.ground(x, maxit=300, tol=1e-12)
        assert r["E0"] == r_ref["E0"] and r["iters"] == r_ref["iters"]
    finally:
        m.close()
