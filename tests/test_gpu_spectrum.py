"""GPU parity of the low-lying spectrum (Sec. IV): hub_lanczos_spectrum (plain Lanczos on the
GPU, Cullum-Willoughby filtering of the tridiagonal on the host) against the exact lowest
distinct eigenvalues (dense diagonalisation, or ARPACK on the oracle's apply)."""
import numpy as np
import pytest

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


def _distinct(w, tol=1e-8):
    out = []
    for x in np.sort(w):
        if not out or x - out[-1] > tol:
            out.append(x)
    return np.array(out)


@pytest.mark.parametrize("small", [False, True])
def test_spectrum_ring8_fast_path(hub, small):
    """Ring M = 8, (4,4), U = 4 (double-float driver, or the single-launch small-sector
    solver): the five lowest distinct eigenvalues agree with ARPACK on the oracle's apply to
    1e-9; their residual estimates are small (an eigenvalue converges as the square of its
    residual, so 1e-4 suffices for 1e-9)."""
    from scipy.sparse.linalg import LinearOperator, eigsh
    M = 8
    bonds = W.ring_bonds(M)
    om = O.Model(M, bonds, 1.0, 4.0)
    B = O.basis(M, 4, 4)
    op = LinearOperator((B.size, B.size), matvec=lambda v: O.apply(om, B, np.ascontiguousarray(v, dtype=np.float64)),
                        dtype=np.float64)
    ref = _distinct(eigsh(op, k=24, which="SA", tol=1e-13, v0=W.normal(3, B.size))[0])[:5]
    m = hub.Hubbard(M, 4, 4, bonds, 1.0, 4.0)
    if not small:
        hub.hub_set_small_dim(m.h, 0)
    e, r = hub.hub_lanczos_spectrum(m.h, torch.from_numpy(W.normal(2, m.D)).cuda(), 400, 5)
    m.close()
    assert e.size == 5
    assert np.max(np.abs(e - ref)) < 1e-9 * np.max(np.abs(ref))
    assert np.all(r < 1e-4)          # eigenvalue error ~ residual^2 / gap


@pytest.mark.parametrize("small", [False, True])
def test_spectrum_disordered_fp64_path(hub, small):
    """Disordered open chain M = 7, (3,2), per-bond t, per-site U and eps (FP64 driver, or the
    single-launch small-sector solver): the six lowest distinct eigenvalues equal those of the
    dense Hamiltonian."""
    M, nu, nd = 7, 3, 2
    bonds = W.chain_bonds(M)
    r = W.uniform(31, 3 * M)
    t = 1.0 + 0.3 * (r[: M - 1] - 0.5)
    U, eps = 2.0 + 4.0 * r[M: 2 * M], 0.4 * (r[2 * M:] - 0.5)
    om = O.Model(M, bonds, t, U, eps)
    ref = _distinct(np.linalg.eigvalsh(O.dense_fock(om, nu, nd)))[:6]
    m = hub.Hubbard(M, nu, nd, bonds, t, U, eps)
    if not small:
        hub.hub_set_small_dim(m.h, 0)
    e, res = hub.hub_lanczos_spectrum(m.h, None, 2 * m.D, 6)
    m.close()
    assert np.max(np.abs(e - ref)) < 1e-9 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.slow
def test_spectrum_4x4_full_size(hub):
    """4x4 periodic lattice, half filling, U = 4, full size: the lowest filtered value equals
    the converged ground-state energy, the next ones lie above it in ascending order."""
    w = W.square4x4(4.0)
    m = hub.Hubbard(16, 8, 8, w["bonds"], w["t"], w["U"], w["eps"])
    g = m.ground(None, maxit=400, tol=1e-12)
    e, r = hub.hub_lanczos_spectrum(m.h, None, 300, 3)
    m.close()
    assert e.size == 3
    assert abs(e[0] - g["E0"]) < 1e-10 * abs(g["E0"])
    assert np.all(np.diff(e) > 0)
    assert r[0] < 1e-4


def _ritz_checks(hub, m, x0, maxit, levels, ref_vals, ref_vecs):
    for i in levels:
        psi = torch.empty(m.D, dtype=torch.float64, device="cuda")
        theta = hub.hub_lanczos_ritz(m.h, x0, maxit, float(ref_vals[i]), psi)
        assert abs(theta - ref_vals[i]) < 1e-9 * max(1.0, abs(ref_vals[i]))
        p = psi.cpu().numpy()
        assert abs(np.linalg.norm(p) - 1.0) < 1e-12
        assert 1.0 - abs(float(p @ ref_vecs[:, i])) < 1e-8, i
        r = (m.apply(psi) - theta * psi).norm().item()
        assert r < 1e-6, (i, r)


@pytest.mark.parametrize("small", [False, True])
def test_ritz_vectors_disordered_fp64_path(hub, small):
    """Excited-state eigenvectors (Sec. IV) on the FP64 driver (or the single-launch
    small-sector solver): the Ritz vectors of the second and third levels of a disordered
    7-site chain, (3,2), match the dense eigenvectors."""
    M, nu, nd = 7, 3, 2
    bonds = W.chain_bonds(M)
    r = W.uniform(31, 3 * M)
    t = 1.0 + 0.3 * (r[: M - 1] - 0.5)
    U, eps = 2.0 + 4.0 * r[M: 2 * M], 0.4 * (r[2 * M:] - 0.5)
    om = O.Model(M, bonds, t, U, eps)
    w, V = np.linalg.eigh(O.dense_fock(om, nu, nd))
    assert min(w[2] - w[1], w[1] - w[0], w[3] - w[2]) > 1e-3
    m = hub.Hubbard(M, nu, nd, bonds, t, U, eps)
    if not small:
        hub.hub_set_small_dim(m.h, 0)
    x0 = torch.from_numpy(W.normal(4, m.D)).cuda()
    _ritz_checks(hub, m, x0, 150, [0, 1, 2], w, V)
    m.close()


@pytest.mark.parametrize("small", [False, True])
def test_ritz_vectors_chain8_fast_path(hub, small):
    """Excited-state eigenvectors on the double-float driver (or the single-launch
    small-sector solver): open chain M = 8, (4,4), U = 4; the two lowest levels against ARPACK
    eigenvectors of the oracle's apply."""
    from scipy.sparse.linalg import LinearOperator, eigsh
    M = 8
    bonds = W.chain_bonds(M)
    om = O.Model(M, bonds, 1.0, 4.0)
    B = O.basis(M, 4, 4)
    op = LinearOperator((B.size, B.size), matvec=lambda v: O.apply(om, B, np.ascontiguousarray(v, dtype=np.float64)),
                        dtype=np.float64)
    w, V = eigsh(op, k=6, which="SA", tol=1e-14, v0=W.normal(3, B.size))
    order = np.argsort(w)
    w, V = w[order], V[:, order]
    levels = [i for i in range(2) if min(abs(w[i] - w[j]) for j in range(len(w)) if j != i) > 1e-3]
    assert levels
    m = hub.Hubbard(M, 4, 4, bonds, 1.0, 4.0)
    if not small:
        hub.hub_set_small_dim(m.h, 0)
    x0 = torch.from_numpy(W.normal(2, m.D)).cuda()
    _ritz_checks(hub, m, x0, 200, levels, w, V)
    m.close()
