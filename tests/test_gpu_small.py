"""The single-launch small-sector Lanczos (one cooperative kernel per batch of iterations,
grid barriers between the phases of an iteration, FP64 throughout) against the oracle's
Lanczos, the dense Hamiltonian and the multi-kernel drivers it stands in for: E0 within
1e-10 relative of the oracle, the same psi, the same stopping rule, breakdowns, refusals,
determinism, and the dispatch by sector size."""
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


def _disordered(M, nu, nd, seed, bonds=None):
    bonds = W.ring_bonds(M) if bonds is None else bonds
    nb = len(bonds)
    t = W.uniform(seed, nb, 0.5, 1.5)
    U = W.uniform(seed + 1, M, 1.0, 6.0)
    eps = W.uniform(seed + 2, M, -0.5, 0.5)
    return dict(M=M, n_up=nu, n_dn=nd, bonds=np.asarray(bonds, dtype=np.int32), t=t, U=U, eps=eps)


def _uniform(M, nu, nd, bonds=None):
    bonds = W.ring_bonds(M) if bonds is None else bonds
    return dict(M=M, n_up=nu, n_dn=nd, bonds=np.asarray(bonds, dtype=np.int32), t=np.ones(len(bonds)),
                U=np.full(M, 4.0), eps=np.zeros(M))


def _model(hub, w):
    return hub.Hubbard(w["M"], w["n_up"], w["n_dn"], w["bonds"], w["t"], w["U"], w["eps"])


def _launches(hub, m, x0, **kw):
    hub.hub_profile(m.h, True)
    r = m.ground(x0, **kw)
    n = hub.hub_profile_read(m.h, hub.HUB_PROF_APPLY)[2]
    hub.hub_profile(m.h, False)
    return r, n


# ring 8 (uniform: the double-float driver otherwise) and a disordered 8-site ring (FP64 driver
# otherwise) run as one thread-block cluster; 9 sites, (4,3) and (5,4), as a cooperative grid
# with the vector staged in shared memory; 10 and 11 sites: vectors beyond the staging size
CASES = {
    "ring8_cluster": lambda: _uniform(8, 4, 4),
    "disordered8_cluster": lambda: _disordered(8, 4, 3, 40),
    "disordered9_staged": lambda: _disordered(9, 4, 3, 40),
    "disordered9_54_staged": lambda: _disordered(9, 5, 4, 45),
    "ring10_unstaged": lambda: _uniform(10, 5, 5),
    "disordered11_unstaged": lambda: _disordered(11, 5, 4, 50),
}


@pytest.mark.parametrize("case", list(CASES))
def test_small_matches_multi_kernel_drivers(hub, case):
    """Same x0, same stopping rule: E0 within 1e-11 relative, iteration counts within two, the
    same normalised psi (overlap 1 - 1e-9), and far fewer kernel launches."""
    w = CASES[case]()
    m = _model(hub, w)
    try:
        x0 = torch.from_numpy(W.normal(7, m.D)).cuda()
        r1, n1 = _launches(hub, m, x0, maxit=500, tol=1e-12, want_psi=True)
        hub.hub_set_small_dim(m.h, 0)
        r2, n2 = _launches(hub, m, x0, maxit=500, tol=1e-12, want_psi=True)
        assert r1["status"] == 0 and r2["status"] == 0
        assert abs(r1["E0"] - r2["E0"]) <= 1e-11 * abs(r2["E0"])
        assert abs(r1["iters"] - r2["iters"]) <= 2
        assert abs(torch.linalg.norm(r1["psi"]).item() - 1.0) < 1e-12
        assert 1.0 - abs(torch.dot(r1["psi"], r2["psi"]).item()) < 1e-9
        # one launch per batch of eight iterations (two batches may run past the stop), plus psi
        assert n1 <= r1["iters"] // 8 + 4 and n2 > 3 * r2["iters"]
    finally:
        m.close()


def test_small_against_oracle_lanczos(hub):
    """Disordered 7-site ring, (4,3): E0 and psi from the same x0 as the oracle's plain Lanczos,
    and E0 against the dense ground state."""
    w = _disordered(7, 4, 3, 60)
    m = _model(hub, w)
    om = oracle_model(w)
    try:
        B = O.basis(7, 4, 3)
        x0 = W.normal(3, B.shape[0])
        r = m.ground(torch.from_numpy(x0).cuda(), maxit=400, tol=1e-12, want_psi=True)
        ro = O.lanczos(om, B, x0, maxit=400, tol=1e-12, want_psi=True)
        assert r["status"] == 0 and ro["converged"]
        assert abs(r["E0"] - ro["E0"]) <= 1e-10 * abs(ro["E0"])
        assert 1.0 - abs(r["psi"].cpu().numpy() @ ro["psi"]) < 1e-9
        w0 = np.linalg.eigvalsh(O.dense_fock(om, 4, 3))[0]
        assert abs(r["E0"] - w0) <= 1e-10 * abs(w0)
    finally:
        m.close()


def test_small_fixed_iterations_coefficients(hub):
    """tol = 0: exactly maxit iterations in one launch; alpha_j and beta_j agree with the FP64
    multi-kernel driver's (the same recurrence, products rounded in another order)."""
    w = _disordered(9, 4, 4, 70)
    m = _model(hub, w)
    try:
        x0 = torch.from_numpy(W.normal(8, m.D)).cuda()
        r1, n1 = _launches(hub, m, x0, maxit=40, tol=0.0)
        a1, b1 = (np.array(c) for c in hub.hub_lanczos_coeffs(m.h))
        hub.hub_set_small_dim(m.h, 0)
        r2 = m.ground(x0, maxit=40, tol=0.0)
        a2, b2 = (np.array(c) for c in hub.hub_lanczos_coeffs(m.h))
        assert r1["iters"] == 40 and r2["iters"] == 40 and n1 == 1
        scale = np.max(np.abs(a2))
        assert np.max(np.abs(a1 - a2)) < 1e-10 * scale and np.max(np.abs(b1 - b2)) < 1e-10 * scale
        assert abs(r1["E0"] - r2["E0"]) <= 1e-12 * abs(r2["E0"])
    finally:
        m.close()


def test_small_breakdowns(hub):
    """One state: breakdown at the first step, E0 = the diagonal.  Two sites, one electron:
    the Krylov space has dimension two, breakdown at the second step, E0 = -|t|."""
    m = hub.Hubbard(5, 5, 0, W.ring_bonds(5), 1.0, 3.0)
    try:
        r = m.ground(torch.ones(1, dtype=torch.float64, device="cuda"), maxit=50, tol=1e-13)
        assert r["status"] == 1 and r["iters"] == 1 and r["E0"] == 0.0
    finally:
        m.close()
    m = hub.Hubbard(2, 1, 0, np.array([[0, 1]], dtype=np.int32), 0.7, 2.0)
    try:
        r = m.ground(torch.tensor([1.0, 0.3], dtype=torch.float64, device="cuda"), maxit=50, tol=1e-15,
                     want_psi=True)
        assert r["status"] == 1 and r["iters"] == 2
        assert abs(r["E0"] + 0.7) < 1e-14
        psi = r["psi"].cpu().numpy()
        assert abs(abs(psi[0]) - np.sqrt(0.5)) < 1e-14 and abs(abs(psi[1]) - np.sqrt(0.5)) < 1e-14
    finally:
        m.close()


def test_small_refusals_and_reuse(hub):
    """A zero start vector is refused (HUB_ERR_ARG) without disturbing later calls; a negative
    bound is refused; the default start vector (x0 = NULL) is the multi-kernel driver's."""
    w = _uniform(8, 4, 4)
    m = _model(hub, w)
    try:
        with pytest.raises(hub.HubError) as e:
            m.ground(torch.zeros(m.D, dtype=torch.float64, device="cuda"), maxit=50, tol=1e-12)
        assert e.value.code == hub.HUB_ERR_ARG
        with pytest.raises(hub.HubError) as e:
            hub.hub_set_small_dim(m.h, -1)
        assert e.value.code == hub.HUB_ERR_ARG
        r1 = m.ground(None, maxit=300, tol=1e-12)
        hub.hub_set_mode(m.h, hub.HUB_MODE_FP64)
        hub.hub_set_small_dim(m.h, 0)
        r2 = m.ground(None, maxit=300, tol=1e-12)
        assert r1["status"] == 0 and r2["status"] == 0
        assert abs(r1["E0"] - r2["E0"]) <= 1e-11 * abs(r2["E0"])
    finally:
        m.close()


@pytest.mark.parametrize("M,nu,nd", [(10, 5, 4), (8, 4, 3)])
def test_small_deterministic(hub, M, nu, nd):
    """Fixed-order reductions: two runs give bit-identical coefficients, E0 and psi (a
    cooperative grid and a cluster)."""
    w = _disordered(M, nu, nd, 80)
    m = _model(hub, w)
    try:
        x0 = torch.from_numpy(W.normal(9, m.D)).cuda()
        runs = []
        for _ in range(2):
            r = m.ground(x0, maxit=300, tol=1e-12, want_psi=True)
            runs.append((r, [np.array(c) for c in hub.hub_lanczos_coeffs(m.h)]))
        (r1, c1), (r2, c2) = runs
        assert r1["E0"] == r2["E0"] and r1["iters"] == r2["iters"]
        assert all(np.array_equal(a, b) for a, b in zip(c1, c2))
        assert torch.equal(r1["psi"], r2["psi"])
    finally:
        m.close()


def test_small_dispatch_by_dimension(hub):
    """Sectors above the bound run the multi-kernel driver: with the bound one below the
    dimension the launch count grows with the iterations; at the dimension it does not."""
    w = _uniform(8, 4, 4)
    m = _model(hub, w)
    try:
        x0 = torch.from_numpy(W.normal(0, m.D)).cuda()
        hub.hub_set_small_dim(m.h, m.D - 1)
        r1, n1 = _launches(hub, m, x0, maxit=300, tol=1e-12)
        hub.hub_set_small_dim(m.h, m.D)
        r2, n2 = _launches(hub, m, x0, maxit=300, tol=1e-12)
        assert n1 > 3 * r1["iters"] and n2 <= r2["iters"] // 8 + 3
        assert abs(r1["E0"] - r2["E0"]) <= 1e-11 * abs(r2["E0"])
    finally:
        m.close()
