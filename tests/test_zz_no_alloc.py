"""hub_grad_noalloc: the gradient entry point for callers that cannot allocate device
memory at call time (they own the device through their own pool, sit on a latency-
critical path where cudaMalloc/cudaFree would synchronise the device, or must keep the
memory footprint fixed after start-up).  Its scratch is a fixed array inside the library.

This file is collected last so that a run stopping at the first failure has already run
every other test; it also passes alone in a fresh process.
"""
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


def test_noalloc_matches_hub_grad_twice(hub):
    """Two calls in a row through the C ABI give the same quadratic forms as hub_grad, to
    the tolerance the gradient parity tests use (1e-12 absolute)."""
    w = dict(W.disordered3x4(), n_up=5, n_dn=6)
    m = hub.Hubbard(w["M"], w["n_up"], w["n_dn"], w["bonds"], w["t"], w["U"], w["eps"])
    try:
        r = m.ground(torch.from_numpy(W.normal(0, m.D)).cuda(), maxit=300, tol=1e-12, want_psi=True)
        vectors = [r["psi"], torch.from_numpy(W.normal(7, m.D)).cuda()]
        for v in vectors:                                  # two calls in a row, different inputs
            ref = hub.hub_grad(m.h, v, m.n_bonds, m.M)
            got = hub.hub_grad_noalloc(m.h, v, m.n_bonds, m.M)
            for a, b in zip(got, ref):
                np.testing.assert_allclose(a, b, rtol=0, atol=1e-12 * max(1.0, np.abs(b).max()))
    finally:
        m.close()


def test_noalloc_allocates_no_device_memory(hub):
    """Free device memory (cudaMemGetInfo) is unchanged across several calls on a fresh handle
    that has run neither Lanczos nor hub_grad, so no lazily allocated scratch of the handle
    exists; a first call on another handle has already loaded the library's device code."""
    w = dict(W.disordered3x4(), n_up=5, n_dn=6)
    warm = hub.Hubbard(w["M"], w["n_up"], w["n_dn"], w["bonds"], w["t"], w["U"], w["eps"])
    m = hub.Hubbard(w["M"], w["n_up"], w["n_dn"], w["bonds"], w["t"], w["U"], w["eps"])
    try:
        v = torch.from_numpy(W.normal(9, m.D)).cuda()
        hub.hub_grad_noalloc(warm.h, v, warm.n_bonds, warm.M)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        got = [hub.hub_grad_noalloc(m.h, v, m.n_bonds, m.M) for _ in range(3)]
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0, (free0, free1)
        ref = hub.hub_grad(m.h, v, m.n_bonds, m.M)
        for g in got:
            for a, b in zip(g, ref):
                np.testing.assert_allclose(a, b, rtol=0, atol=1e-12 * max(1.0, np.abs(b).max()))
    finally:
        m.close()
        warm.close()


def test_noalloc_rejects_models_beyond_its_capacity(hub):
    """n_bonds + 2M above the fixed capacity (160) is refused with HUB_ERR_ARG."""
    M = 30
    bonds = [(i, j) for i in range(M) for j in range(i + 1, M)][:120]      # 120 + 60 = 180 > 160
    m = hub.Hubbard(M, 1, 1, bonds, np.ones(len(bonds)), 1.0)
    try:
        psi = torch.from_numpy(W.normal(1, m.D)).cuda()
        with pytest.raises(hub.HubError) as e:
            hub.hub_grad_noalloc(m.h, psi, m.n_bonds, m.M)
        assert e.value.code == hub.HUB_ERR_ARG
        assert "160" in str(e.value)
    finally:
        m.close()
