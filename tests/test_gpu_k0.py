"""GPU parity of the k = 0 translation sector (Sec. V) through the C ABI.

The oracle builds the k = 0 Bloch states of the paper's combined representatives in the full
two-spin basis and applies the full H (oracle/hub_oracle_k0.py).  The library works in row
form with the columns of Table I, X[i, (j, n)] = sqrt(P_i) <R_i (x) T^n R_j | Psi>; the tests
sample the oracle's translation-invariant vectors on the rows of the up representatives in
that column order (oracle ``row_form_rep``) to compare.  Integer data (representatives,
periods, dimension) bit for bit; products per entry within 1e-13 (|H||Psi|); energies within
1e-10 relative.
"""
import math

import numpy as np
import pytest

from helpers import assert_entrywise
from oracle import hub_oracle as O
from oracle import hub_oracle_k0 as K
from paper_1307_7542_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def hub(cuda_ok):
    import __graft_entry__
    __graft_entry__.build()
    from paper_1307_7542_gb300 import hub as H
    return H


def ring(M, nnn=False):
    b = [(i, (i + 1) % M) for i in range(M)]
    if nnn:
        b += [(i, (i + 2) % M) for i in range(M)]
    return np.array(b, dtype=np.int32)


# (M, N_up, N_dn, next-nearest bonds, t, U, eps)
CASES = [
    (4, 2, 1, False, 1.0, 4.0, 0.0),
    (4, 2, 0, False, 1.0, 4.0, 0.0),     # a cycle with no k = 0 state
    (6, 3, 3, False, 1.0, 4.0, 0.0),
    (6, 4, 2, False, 0.7, 2.5, 0.3),     # short rows and cycles with no k = 0 state
    (6, 3, 3, True, 1.0, 4.0, -0.2),
    (7, 3, 4, False, 1.0, 3.0, 0.0),
    (8, 4, 4, False, 1.0, 4.0, 0.0),
    (8, 4, 2, True, 0.9, 6.0, 0.1),
    (9, 3, 3, False, 1.0, 8.0, 0.0),
    (10, 5, 5, False, 1.0, 4.0, 0.0),
    (12, 6, 6, False, 1.0, 4.0, 0.0),    # 924 columns: four 256-column tiles, ragged tail
    (12, 4, 5, True, 1.1, 2.0, 0.05),
    (6, 0, 2, False, 1.0, 4.0, 0.0),     # one row of period 1
    (5, 5, 2, False, 1.0, 4.0, 0.0),     # full up filling
    (8, 4, 3, True, (1.0, 0.6), 4.0, 0.0),   # two hopping amplitudes: the FP64 kernel
]


def _t(M, nnn, t):
    """Per-bond t: a scalar for every bond, or (nearest, next-nearest)."""
    if np.ndim(t) == 0:
        return float(t)
    return np.r_[np.full(M, t[0]), np.full(M, t[1])] if nnn else np.full(M, t[0])


# (case, omega): k = 0 for every case, k = pi (omega = -1) for the even rings
SECTOR_CASES = [(c, 1) for c in CASES] + [(c, -1) for c in CASES if c[0] % 2 == 0]


def _ids(sc):
    (M, nu, nd, nnn, *_), om = sc
    return f"M{M}-{nu}-{nd}{'-nnn' if nnn else ''}-{'k0' if om == 1 else 'kpi'}"


def _models(hub, M, nu, nd, nnn, t, U, eps, omega=1):
    bonds = ring(M, nnn)
    t = _t(M, nnn, t)
    om = O.Model(M, bonds, t, U, eps)
    m = hub.Hubbard(M, nu, nd, bonds, t, U, np.full(M, eps) if eps else None)
    m.set_symmetry(hub.HUB_SYM_K0 if omega == 1 else hub.HUB_SYM_KPI)
    return om, m


@pytest.mark.parametrize("sc", SECTOR_CASES, ids=_ids)
def test_k0_tables_bitexact(hub, sc):
    """Rows, columns and dimension of the k = 0 (k = pi) space; the up representatives and
    their periods equal the oracle's cycle enumeration, bit for bit."""
    (M, nu, nd, nnn, t, U, eps), omega = sc
    om, m = _models(hub, M, nu, nd, nnn, t, U, eps, omega)
    tb = K.spin_tables(M, nu)
    is_rep = tb["state"] == tb["rep"]
    reps, per = m.k_reps()
    m.close()
    assert np.array_equal(reps.astype(np.uint64), tb["state"][is_rep])
    assert np.array_equal(per.astype(np.int64), tb["period"][is_rep])
    assert (m.k_rows, m.k_cols) == (int(is_rep.sum()), math.comb(M, nd))
    assert m.k_dim == K.k0_dimension(M, nu, nd, omega)
    bits, sign = K.rep_columns(M, nd)
    om, m = _models(hub, M, nu, nd, nnn, t, U, eps, omega)
    cb, cs = m.k_columns()
    m.close()
    assert np.array_equal(cb.astype(np.uint64), bits) and np.array_equal(cs, sign.astype(np.int32))


@pytest.mark.parametrize("sc", SECTOR_CASES, ids=_ids)
def test_k0_apply_parity(hub, sc):
    """H on random k = 0 (k = pi) states: the library's row-form product equals the oracle's
    full two-spin product sampled on the representative rows, per entry within
    1e-13 |H||Psi|."""
    (M, nu, nd, nnn, t, U, eps), omega = sc
    om, m = _models(hub, M, nu, nd, nnn, t, U, eps, omega)
    B = O.basis(M, nu, nd)
    V = K.bloch_matrix(M, nu, nd, B, omega)
    if V.shape[1] == 0:
        m.close()
        return
    for seed in (1, 2):
        psi = np.asarray(V @ W.normal(seed, V.shape[1]))
        X, _, _ = K.row_form_rep(M, nu, nd, B, psi)
        Yref, _, _ = K.row_form_rep(M, nu, nd, B, O.apply(om, B, psi))
        bound, _, _ = K.row_form_rep(M, nu, nd, B, O.apply(om, B, np.abs(psi), absolute=True))
        y = m.apply(torch.from_numpy(X.ravel()).cuda()).cpu().numpy()
        assert_entrywise(y, Yref.ravel(), np.abs(bound).ravel())
    m.close()


@pytest.mark.parametrize("M,nu,nd,nnn,omega", [(6, 4, 2, False, 1), (8, 4, 4, True, 1), (8, 4, 4, False, -1),
                                               (10, 5, 4, False, 1)])
def test_k0_apply_wide_range(hub, M, nu, nd, nnn, omega):
    """Integer-pipe sums on vectors spanning 10^-300 .. 10^300 with zeros and subnormal
    entries: per entry within 1e-13 |H||Psi| of the oracle."""
    om, m = _models(hub, M, nu, nd, nnn, 1.0, 4.0, 0.0, omega)
    B = O.basis(M, nu, nd)
    V = K.bloch_matrix(M, nu, nd, B, omega)
    n = V.shape[1]
    phi = W.normal(11, n) * 10.0 ** W.uniform(12, n, -300.0, 300.0)
    phi[W.uniform(13, n) < 0.2] = 0.0
    phi[:3] = [5e-321, -2e-310, 1e-308]
    psi = np.asarray(V @ phi)
    X, _, _ = K.row_form_rep(M, nu, nd, B, psi)
    Yref, _, _ = K.row_form_rep(M, nu, nd, B, O.apply(om, B, psi))
    bound, _, _ = K.row_form_rep(M, nu, nd, B, O.apply(om, B, np.abs(psi), absolute=True))
    y = m.apply(torch.from_numpy(X.ravel()).cuda()).cpu().numpy()
    m.close()
    assert_entrywise(y, Yref.ravel(), np.abs(bound).ravel())


@pytest.mark.parametrize("M,omega", [(12, 1), (14, -1)])
def test_k0_clean_and_general_integer_kernels_agree(hub, M, omega):
    """The integer-pipe product has two kernels: one for vectors of zeros and normal numbers
    (checked on the device before each product), one that also handles subnormal, Inf and NaN
    entries.  Putting a subnormal (1e-310) where the vector had a zero sends the product to the
    second kernel; every entry the subnormal cannot reach at the 1e-300 level is bit-identical
    to the first kernel's product of the vector with the zero."""
    m = hub.Hubbard(M, M // 2, M // 2, ring(M), 1.0, 4.0)
    m.set_symmetry(hub.HUB_SYM_K0 if omega == 1 else hub.HUB_SYM_KPI)
    x = m.k_project(torch.from_numpy(W.normal(5, m.D)).cuda())
    p = int(torch.argmax(x.abs()).item())
    x[p] = 0.0
    y_clean = m.apply(x)
    x2 = x.clone()
    x2[p] = 1e-310
    y_gen = m.apply(x2)
    m.close()
    keep = y_clean.abs() > 1e-200
    assert bool(keep.float().mean() > 0.99)
    assert torch.equal(y_clean[keep], y_gen[keep])


@pytest.mark.parametrize("M,omega", [(14, 1), (16, -1)])
def test_k0_integer_path_matches_fp64_kernel(hub, M, omega):
    """Full-size rings: the integer-pipe product (default) against the FP64 kernel
    (HUB_MODE_FP64) on the same projected random array, per entry within 1e-13 of the
    entry's |H||x| scale, and the same Lanczos energy to 1e-12."""
    m = hub.Hubbard(M, M // 2, M // 2, ring(M), 1.0, 4.0)
    m.set_symmetry(hub.HUB_SYM_K0 if omega == 1 else hub.HUB_SYM_KPI)
    x = m.k_project(torch.from_numpy(W.normal(3, m.D)).cuda())
    y_int = m.apply(x)
    e_int = m.ground(None, maxit=300, tol=1e-12)["E0"]
    hub.hub_set_mode(m.h, hub.HUB_MODE_FP64)
    y_f64 = m.apply(x)
    e_f64 = m.ground(None, maxit=300, tol=1e-12)["E0"]
    scale = m.apply(x.abs())          # >= the |H||x| scale entrywise only up to signs of H
    m.close()
    err = (y_int - y_f64).abs()
    bound = 1e-13 * (scale.abs() + 4.0 * M * x.abs().max())
    assert bool((err <= bound).all())
    assert abs(e_int - e_f64) < 1e-12 * abs(e_f64)


@pytest.mark.parametrize("M,nu,nd,omega", [(4, 2, 0, 1), (6, 4, 2, 1), (8, 4, 2, 1), (8, 4, 4, 1), (9, 3, 3, 1),
                                         (4, 2, 0, -1), (6, 4, 2, -1), (8, 4, 4, -1), (6, 2, 1, -1)])
def test_k0_projection(hub, M, nu, nd, omega):
    """hub_k_project is the orthogonal projection onto the sector in row form: it keeps
    row-form states of the sector, is idempotent bit for bit, leaves x - Px orthogonal to the
    sector, and its trace (projecting every unit array) is the sector's dimension."""
    om, m = _models(hub, M, nu, nd, False, 1.0, 4.0, 0.0, omega)
    B = O.basis(M, nu, nd)
    V = K.bloch_matrix(M, nu, nd, B, omega)
    X, _, _ = K.row_form_rep(M, nu, nd, B, np.asarray(V @ W.normal(5, V.shape[1])))
    px = m.k_project(torch.from_numpy(X.ravel()).cuda()).cpu().numpy()
    assert np.max(np.abs(px - X.ravel())) < 1e-14 * np.max(np.abs(X))
    x = torch.from_numpy(W.normal(6, m.D)).cuda()
    p1 = m.k_project(x)
    p2 = m.k_project(p1.clone())
    assert torch.equal(p1, p2)
    r = (x - p1).cpu().numpy()
    for seed in (7, 8):
        Z, _, _ = K.row_form_rep(M, nu, nd, B, np.asarray(V @ W.normal(seed, V.shape[1])))
        assert abs(float(r @ Z.ravel())) < 1e-13 * np.linalg.norm(r) * np.linalg.norm(Z)
    eye = torch.eye(m.D, dtype=torch.float64, device="cuda")
    tr = sum(float(m.k_project(eye[k].contiguous())[k]) for k in range(m.D))
    assert abs(tr - K.k0_dimension(M, nu, nd, omega)) < 1e-12 * m.D
    m.close()


@pytest.mark.parametrize("sc", [c for c in SECTOR_CASES if c[0][0] <= 10], ids=_ids)
def test_k0_ground_energy(hub, sc):
    """Lowest eigenvalue of the sector by the library's Lanczos in it equals the lowest
    eigenvalue of V^T H V, within 1e-10 relative; the row-form ground state matches the
    oracle's eigenvector sampled on the rows (when that level is simple)."""
    (M, nu, nd, nnn, t, U, eps), omega = sc
    om, m = _models(hub, M, nu, nd, nnn, t, U, eps, omega)
    B = O.basis(M, nu, nd)
    V = K.bloch_matrix(M, nu, nd, B, omega)
    if V.shape[1] == 0:
        m.close()
        return
    w, Z = np.linalg.eigh(K.k0_matrix(om, B, V))
    g = m.ground(None, maxit=min(400, 3 * m.k_dim + 5), tol=1e-13, want_psi=True)
    assert abs(g["E0"] - w[0]) < 1e-10 * max(1.0, abs(w[0]))
    if w.size > 1 and w[1] - w[0] > 1e-6:
        ref, _, _ = K.row_form_rep(M, nu, nd, B, np.asarray(V @ Z[:, 0]))
        p = g["psi"].cpu().numpy()
        assert 1.0 - abs(float(p @ ref.ravel())) < 1e-9
    m.close()


@pytest.mark.parametrize("M,nu,nd,nnn,omega", [(8, 4, 4, False, 1), (6, 4, 2, False, 1), (9, 3, 3, True, 1),
                                               (8, 4, 4, False, -1), (8, 3, 4, True, -1)])
def test_k0_spectrum(hub, M, nu, nd, nnn, omega):
    """hub_lanczos_spectrum in a momentum sector: its lowest distinct eigenvalues."""
    om, m = _models(hub, M, nu, nd, nnn, 1.0, 4.0, 0.0, omega)
    B = O.basis(M, nu, nd)
    w = np.linalg.eigvalsh(K.k0_matrix(om, B, K.bloch_matrix(M, nu, nd, B, omega)))
    ref = []
    for x in w:
        if not ref or x - ref[-1] > 1e-8:
            ref.append(x)
    n = min(4, len(ref))
    e, _ = hub.hub_lanczos_spectrum(m.h, None, min(3000, 4 * m.k_dim + 20), n)
    m.close()
    assert np.max(np.abs(e[:n] - np.array(ref[:n]))) < 1e-9 * max(1.0, abs(ref[0]))


def test_k0_hermitian_and_free_ring_at_M14(hub):
    """M = 14, (7, 7): U = 0 k = 0 ground energy equals the best momentum-0 filling of the
    one-particle levels; at U = 4 the product is symmetric on projected random arrays."""
    M = 14
    bonds = ring(M)
    m = hub.Hubbard(M, 7, 7, bonds, 1.0, 0.0)
    m.set_symmetry(hub.HUB_SYM_K0)
    g = m.ground(None, maxit=300, tol=1e-13)
    ref = K.ring_free_k0_levels(M, 7, 7)[0]
    assert abs(g["E0"] - ref) < 1e-10 * abs(ref)
    m.set_params(1.0, 4.0)
    m.set_symmetry(hub.HUB_SYM_K0)
    a = m.k_project(torch.from_numpy(W.normal(1, m.D)).cuda())
    b = m.k_project(torch.from_numpy(W.normal(2, m.D)).cuda())
    lhs, rhs = float(a @ m.apply(b)), float(m.apply(a) @ b)
    assert abs(lhs - rhs) < 1e-12 * (float(a.norm()) * float(m.apply(b).norm()))
    m.close()


def test_k0_table4_M14(hub):
    """Table IV: the 14-site ring at half filling, U = 4, t = 1.  The ground state lies at
    k = 0 (seven electrons of each spin); the k = 0 Lanczos energy equals the printed value
    within 5e-10 and the full-sector energy of the library within 1e-10 relative."""
    M = 14
    from conftest import golden
    printed = {int(r[0]): float(r[2]) for r in golden("table4_E0.txt")}[M]
    m = hub.Hubbard(M, 7, 7, ring(M), 1.0, 4.0)
    full = m.ground(None, maxit=400, tol=1e-13)["E0"]
    m.set_symmetry(hub.HUB_SYM_K0)
    assert m.k_dim * 14 >= m.count_up * m.count_dn
    k0 = m.ground(None, maxit=400, tol=1e-13)["E0"]
    m.set_symmetry(hub.HUB_SYM_NONE)
    again = m.ground(None, maxit=400, tol=1e-13)["E0"]
    m.close()
    assert abs(k0 - printed) < 5e-10
    assert abs(k0 - full) < 1e-10 * abs(full)
    assert again == full


@pytest.mark.slow
def test_k0_M16_variational(hub):
    """M = 16, (8, 8), U = 4: the k = 0 and k = pi energies are not below the full-sector
    energy (subspaces); with eight electrons of each spin the ground state lies at k = pi,
    where the 16-fold smaller space reaches the full-sector energy (Table IV)."""
    M = 16
    m = hub.Hubbard(M, 8, 8, ring(M), 1.0, 4.0)
    full = m.ground(None, maxit=400, tol=1e-12)["E0"]
    m.set_symmetry(hub.HUB_SYM_K0)
    k0 = m.ground(None, maxit=400, tol=1e-12)["E0"]
    m.set_symmetry(hub.HUB_SYM_KPI)
    kpi = m.ground(None, maxit=400, tol=1e-12)["E0"]
    m.close()
    assert k0 >= full - 1e-10 * abs(full)
    assert kpi >= full - 1e-10 * abs(full)
    assert abs(kpi - full) < 1e-10 * abs(full)


def test_k0_errors(hub):
    """Refusals: bonds not invariant under T, site-dependent U or eps; calls that have no
    k = 0 form; the k = 0 queries outside the sector.  New parameters leave the sector."""
    M = 6
    m = hub.Hubbard(M, 3, 3, W.chain_bonds(M), 1.0, 4.0)          # open chain
    with pytest.raises(hub.HubError) as e:
        m.set_symmetry(hub.HUB_SYM_K0)
    assert e.value.code == hub.HUB_ERR_ARG
    with pytest.raises(hub.HubError) as e:
        hub.hub_k_dims(m.h)
    assert e.value.code == hub.HUB_ERR_STATE
    m.set_params(np.ones(M - 1), 4.0)
    m.close()
    m = hub.Hubbard(M, 3, 3, ring(M), 1.0, np.arange(M, dtype=np.float64))
    with pytest.raises(hub.HubError) as e:
        m.set_symmetry(hub.HUB_SYM_K0)
    assert e.value.code == hub.HUB_ERR_ARG
    m.set_params(1.0, 4.0, np.linspace(0, 1, M))
    with pytest.raises(hub.HubError) as e:
        m.set_symmetry(hub.HUB_SYM_K0)
    assert e.value.code == hub.HUB_ERR_ARG
    m.set_params(1.0, 4.0)
    m.set_symmetry(hub.HUB_SYM_K0)
    psi = torch.zeros(m.D, dtype=torch.float64, device="cuda")
    with pytest.raises(hub.HubError) as e:
        m.grad(psi)
    assert e.value.code == hub.HUB_ERR_STATE
    with pytest.raises(hub.HubError) as e:
        hub.hub_set_symmetry(m.h, 7)
    assert e.value.code == hub.HUB_ERR_ARG
    with pytest.raises(hub.HubError) as e:
        hub.Hubbard(5, 2, 2, ring(5), 1.0, 4.0).set_symmetry(hub.HUB_SYM_KPI)   # odd M
    assert e.value.code == hub.HUB_ERR_ARG
    m.set_params(1.0, 5.0)                                     # leaves the k = 0 sector
    assert m.D == m.count_up * m.count_dn
    with pytest.raises(hub.HubError) as e:
        hub.hub_k_dims(m.h)
    assert e.value.code == hub.HUB_ERR_STATE
    m.close()


def test_k_sector_host_apply_and_ritz(hub):
    """Inside a momentum sector: hub_apply_host (host arrays) equals hub_apply, and
    hub_lanczos_ritz returns the eigenvector (row form) and value of the lowest simple excited
    k = 0 level."""
    M, nu, nd = 8, 4, 4
    om, m = _models(hub, M, nu, nd, False, 1.0, 4.0, 0.0, 1)
    x = m.k_project(torch.from_numpy(W.normal(9, m.D)).cuda())
    y_dev = m.apply(x).cpu().numpy()
    xh = x.cpu().numpy().copy()
    yh = np.empty_like(xh)
    hub.hub_apply_host(m.h, xh, yh)
    assert np.array_equal(yh, y_dev)
    B = O.basis(M, nu, nd)
    V = K.bloch_matrix(M, nu, nd, B)
    w, Z = np.linalg.eigh(K.k0_matrix(om, B, V))
    lvl = next(l for l in range(1, w.size - 1) if min(w[l] - w[l - 1], w[l + 1] - w[l]) > 1e-3)
    assert lvl <= 4
    psi = torch.empty(m.D, dtype=torch.float64, device="cuda")
    theta = hub.hub_lanczos_ritz(m.h, None, 200, float(w[lvl]), psi)
    ref, _, _ = K.row_form_rep(M, nu, nd, B, np.asarray(V @ Z[:, lvl]))
    m.close()
    assert abs(theta - w[lvl]) < 1e-9 * abs(w[lvl])
    assert 1.0 - abs(float(psi.cpu().numpy() @ ref.ravel())) < 1e-8


# ------------------------------------------------------------------ several translations (torus)

def torus_bonds(Lx, Ly):
    b = set()
    for y in range(Ly):
        for x in range(Lx):
            s = x + Lx * y
            for dx, dy in ((1, 0), (0, 1)):
                s2 = (x + dx) % Lx + Lx * ((y + dy) % Ly)
                b.add((min(s, s2), max(s, s2)))
    return np.array(sorted(b), dtype=np.int32)


# (Lx, Ly, N_up, N_dn, characters, t, U, eps)
TORUS = [
    (3, 3, 2, 2, (1, 1), 1.0, 4.0, 0.0),
    (3, 3, 3, 2, (1, 1), 0.8, 2.0, 0.1),
    (4, 2, 3, 3, (-1, 1), 1.0, 4.0, 0.0),
    (4, 2, 4, 2, (-1, -1), 1.0, 3.0, 0.0),     # stabilisers with sign -1, empty orbits
    (4, 2, 2, 2, (1, -1), 0.7, 5.0, -0.2),
    (2, 2, 2, 2, (-1, 1), 1.0, 4.0, 0.0),
    (4, 3, 3, 3, (-1, 1), 1.0, 4.0, 0.0),       # 220 x 220 strings: several column tiles
]


@pytest.mark.parametrize("case", TORUS, ids=lambda c: f"{c[0]}x{c[1]}-{c[2]}-{c[3]}-{c[4]}")
def test_torus_sector_parity(hub, case):
    """Momentum sectors of the torus (hub_set_translations): representatives, orbit sizes,
    columns and dimension bit-exact against the oracle's group construction; products of
    random states of the sector per entry within 1e-13 |H||Psi|; the lowest eigenvalue of the
    sector by the library's Lanczos against dense V^T H V."""
    Lx, Ly, nu, nd, chars, t, U, eps = case
    M = Lx * Ly
    gens = K.torus_translations(Lx, Ly)
    bonds = torus_bonds(Lx, Ly)
    om = O.Model(M, bonds, t, U, eps)
    m = hub.Hubbard(M, nu, nd, bonds, t, U, np.full(M, eps) if eps else None)
    m.set_translations(gens, chars)
    B = O.basis(M, nu, nd)
    V = K.bloch_matrix_group(M, nu, nd, B, gens, list(chars))
    assert m.k_dim == V.shape[1]
    X0, reps, per = K.row_form_group(M, nu, nd, B, np.zeros(B.shape[0]), gens)
    r, p = m.k_reps()
    assert np.array_equal(r.astype(np.uint64), reps) and np.array_equal(p.astype(np.int64), per)
    cb, cs = m.k_columns()
    ob, osg = K.group_columns(M, nd, gens)
    assert np.array_equal(cb.astype(np.uint64), ob) and np.array_equal(cs, osg.astype(np.int32))
    for seed in (1, 2):
        psi = np.asarray(V @ W.normal(seed, V.shape[1]))
        X, _, _ = K.row_form_group(M, nu, nd, B, psi, gens)
        Yref, _, _ = K.row_form_group(M, nu, nd, B, O.apply(om, B, psi), gens)
        bound, _, _ = K.row_form_group(M, nu, nd, B, O.apply(om, B, np.abs(psi), absolute=True), gens)
        y = m.apply(torch.from_numpy(X.ravel()).cuda()).cpu().numpy()
        assert_entrywise(y, Yref.ravel(), np.abs(bound).ravel())
    w = np.linalg.eigvalsh(K.k0_matrix(om, B, V))
    g = m.ground(None, maxit=min(400, 3 * m.k_dim + 5), tol=1e-13)
    m.close()
    assert abs(g["E0"] - w[0]) < 1e-10 * max(1.0, abs(w[0]))


def test_torus_translation_errors(hub):
    """Refusals: a generator that is not a permutation, one that does not map bonds onto
    bonds, non-commuting generators, -1 on a generator of odd order."""
    M = 9
    gens = K.torus_translations(3, 3)
    m = hub.Hubbard(M, 2, 2, torus_bonds(3, 3), 1.0, 4.0)
    for perms, chars in [([[0] * M], [1]), ([list(range(1, M)) + [0]], [1]), (gens, [-1, 1]),
                         ([gens[0], [1, 0, 2, 4, 3, 5, 7, 6, 8]], [1, 1])]:
        with pytest.raises(hub.HubError) as e:
            m.set_translations(perms, chars)
        assert e.value.code == hub.HUB_ERR_ARG
    m.close()


@pytest.mark.slow
def test_torus_4x4_sectors_reach_the_ground_state(hub):
    """4x4 torus, half filling, U = 4: the four real-momentum sectors (each about 16 times
    smaller than the sector) lie above the full-sector E0, and the lowest of them equals it."""
    w = W.square4x4(4.0)
    m = hub.Hubbard(16, 8, 8, w["bonds"], w["t"], w["U"], w["eps"])
    full = m.ground(None, maxit=400, tol=1e-12)["E0"]
    gens = K.torus_translations(4, 4)
    energies = []
    for chars in ((1, 1), (-1, 1), (1, -1), (-1, -1)):
        m.set_translations(gens, chars)
        assert 0.9 * m.count_up * m.count_dn <= 16 * m.k_dim <= 1.1 * m.count_up * m.count_dn
        energies.append(m.ground(None, maxit=400, tol=1e-12)["E0"])
    m.close()
    assert min(energies) >= full - 1e-10 * abs(full)
    assert abs(min(energies) - full) < 1e-10 * abs(full)
