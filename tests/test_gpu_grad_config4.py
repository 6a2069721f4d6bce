"""Gradients of E0 on the disordered 3x4 open lattice, (N_up, N_dn) = (6, 6), D = 853,776
(t_b = 1 + U[-0.1, 0.1], U_i ~ U[2, 8], eps_i ~ U[-0.5, 0.5]): all 41 derivatives.

dE0/dt_b = <-sum_s (c+_i c_j + h.c.)>, dE0/dU_i = <n_i,up n_i,dn>, dE0/deps_i = <n_i>
(Hellmann-Feynman, with H = -sum_b t_b ... + sum_i U_i n_up n_dn + sum_i eps_i n_i) from
hub_grad are checked against
  * central finite differences (h = 1e-4) of GPU Lanczos energies, every parameter, and
  * the oracle's expectation values on the oracle's own Lanczos ground state (two-spin
    basis, CPU): no GPU vector enters the reference,
after checking that the ground state is non-degenerate (gap > 1e-6), so that psi and the
derivatives are defined.
"""
import numpy as np
import pytest

from helpers import oracle_model
from oracle import hub_oracle as O
from paper_1307_7542_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def hub(cuda_ok):
    import __graft_entry__
    __graft_entry__.build()
    from paper_1307_7542_gb300 import hub as H
    return H


@pytest.fixture(scope="module")
def config4(hub):
    """GPU model, start vector, converged ground state and hub_grad's 41 derivatives."""
    w = dict(W.disordered3x4(), n_up=6, n_dn=6)
    m = hub.Hubbard(w["M"], 6, 6, w["bonds"], w["t"], w["U"], w["eps"])
    x0 = torch.from_numpy(W.normal(0, m.D)).cuda()
    r = m.ground(x0, maxit=600, tol=1e-14, want_psi=True)
    assert r["status"] in (0, 1), r
    g = m.grad(r["psi"])
    ev, res = hub.hub_lanczos_spectrum(m.h, x0, 300, 2)
    yield dict(w=w, m=m, x0=x0, E0=r["E0"], psi=r["psi"], grad=g, spectrum=(ev, res))
    m.close()


def test_config4_gap(config4):
    """The two lowest eigenvalues are separated by more than 1e-6 (non-degenerate ground state)."""
    ev, res = config4["spectrum"]
    assert len(ev) == 2
    assert abs(ev[0] - config4["E0"]) < 1e-9
    assert ev[1] - ev[0] > 1e-6


def test_config4_grad_vs_finite_differences_all_parameters(config4):
    """All 17 + 12 + 12 derivatives against (E0(theta + h) - E0(theta - h)) / 2h, h = 1e-4:
    the difference quotient's error is O(h^2) ~ 1e-8 plus Lanczos noise / h ~ 1e-9."""
    w, m, x0 = config4["w"], config4["m"], config4["x0"]
    dt, dU, de = config4["grad"]
    h = 1e-4

    def E(t, U, eps):
        m.set_params(t, U, eps)
        r = m.ground(x0, maxit=600, tol=1e-14)
        assert r["status"] in (0, 1)
        return r["E0"]

    worst = 0.0
    try:
        for name, base, g in (("t", w["t"], dt), ("U", w["U"], dU), ("eps", w["eps"], de)):
            for k in range(len(base)):
                p, q = base.copy(), base.copy()
                p[k] += h
                q[k] -= h
                args_p = {"t": w["t"], "U": w["U"], "eps": w["eps"], name: p}
                args_q = {"t": w["t"], "U": w["U"], "eps": w["eps"], name: q}
                fd = (E(**args_p) - E(**args_q)) / (2 * h)
                worst = max(worst, abs(fd - g[k]))
                assert abs(fd - g[k]) < 1e-6, (name, k, fd, g[k])
    finally:
        m.set_params(w["t"], w["U"], w["eps"])
    print(f"max |FD - hub_grad| over 41 parameters: {worst:.2e}")


@pytest.mark.slow
def test_config4_grad_vs_oracle_ground_state(hub, config4):
    """hub_grad on the GPU ground state against the oracle's expectation values on the
    oracle's own ground state.  Both sides run their plain Lanczos from the same start
    vector for a fixed 300 iterations, so that the eigenvectors, not only E0, converge: an
    expectation value taken on a vector with residual r is off by O(r / gap), and the
    residuals are checked below 1e-8 (oracle products on both vectors)."""
    w, m = config4["w"], config4["m"]
    om = oracle_model(w)
    B = O.basis(12, 6, 6)
    r = O.lanczos(om, B, W.normal(0, B.shape[0]), maxit=300, tol=0.0, want_psi=True, fixed_iters=True)
    psi_o = r["psi"]
    rg = m.ground(config4["x0"], maxit=300, tol=0.0, want_psi=True)
    psi_g = rg["psi"].cpu().numpy()
    res_o = np.linalg.norm(O.apply(om, B, psi_o) - r["E0"] * psi_o)
    res_g = np.linalg.norm(O.apply(om, B, psi_g) - rg["E0"] * psi_g)
    assert res_o < 1e-8 and res_g < 1e-8, (res_o, res_g)
    ot, oU, oe = O.expectations(om, B, psi_o)
    dt, dU, de = m.grad(rg["psi"])
    assert abs(r["E0"] - rg["E0"]) <= 1e-10 * abs(r["E0"])
    overlap = abs(float(np.dot(psi_o, psi_g)))
    assert 1.0 - overlap < 1e-12, overlap
    # |<psi'|A|psi'> - <psi|A|psi>| <= 2 |A| |psi' - psi| with |psi' - psi| <= r / gap; the
    # one-site and one-bond operators A here have norm at most 2
    ev, _ = config4["spectrum"]
    atol = 4.0 * 2.0 * max(res_o, res_g) / (ev[1] - ev[0]) + 1e-11
    for a, b in ((dt, ot), (dU, oU), (de, oe)):
        np.testing.assert_allclose(a, b, rtol=0, atol=atol)
    diff = max(np.max(np.abs(dt - ot)), np.max(np.abs(dU - oU)), np.max(np.abs(de - oe)))
    print(f"max |hub_grad - oracle| = {diff:.2e} (bound {atol:.1e}), 1 - overlap = {1 - overlap:.1e}, "
          f"residuals {res_g:.1e} (GPU), {res_o:.1e} (oracle)")
