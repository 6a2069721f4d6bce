"""Pins of the k = 0 oracle (Sec. V, translation symmetry) against what the paper prints
and what the mathematics fixes: Tables I and II, brute-force counts of representatives,
the character formula for the dimension of the k = 0 space, the complete U = 0 spectrum
from one-particle momenta, and the spectrum of H on the range of the projector
(1/M) sum_r T^r built from the brute-force translation matrix.  The same pins hold the
k = pi sector (omega = e^{ik} = -1, even M) of the oracle."""
import os
from itertools import product

import numpy as np
import pytest

from oracle import hub_oracle as O
from oracle import hub_oracle_k0 as K

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def ring(M, nnn=False):
    b = [(i, (i + 1) % M) for i in range(M)]
    if nnn:
        b += [(i, (i + 2) % M) for i in range(M)]
    return b


def test_table2_per_rep_trans_esign():
    """Table II: period index, representative index, translation and phase of every string
    of M = 4, N = 2."""
    tb = K.spin_tables(4, 2)
    for s, per, rep, tr, sg in _rows("k0_table2_M4_N2.txt"):
        i = int(np.flatnonzero(tb["state"] == int(s, 2))[0])
        assert (tb["per_index"][i] + 1, tb["rep_index"][i] + 1, tb["trans"][i], int(tb["esign"][i])) == \
            (int(per), int(rep), int(tr), int(sg)), s
    # the paper's example of a phase after one period: T^2 |0101> = -|0101>
    i = int(np.flatnonzero(tb["state"] == 0b0101)[0])
    assert tb["period"][i] == 2 and tb["esignb"][i] == -1


def test_table1_combined_representatives():
    """Table I: the combined representatives of M = 4, (N_up, N_dn) = (2, 1), in order."""
    cr = K.combined_reps(4, 2, 1)
    rows = _rows("k0_table1_M4_up2_dn1.txt")
    assert len(rows) == cr["n"].shape[0]
    for j, (ru, rd, n, tn, idx) in enumerate(rows):
        assert int(idx) == j + 1
        assert (int(cr["up"][j]), int(cr["dn_rep"][j]), int(cr["n"][j]), int(cr["dn"][j])) == \
            (int(ru, 2), int(rd, 2), int(n), int(tn, 2))
    assert not cr["null"].any()


@pytest.mark.parametrize("M", range(1, 15))
def test_nstate_counts_the_cycles(M):
    """Eq. count6 (reading 1) equals the number of cycles of each period found by
    enumerating all strings; the printed form agrees whenever a period has at most one
    smaller admissible period dividing it."""
    for N in range(M + 1):
        tb = K.spin_tables(M, N)
        reps = tb["state"] == tb["rep"]
        counted = {int(p): int(np.count_nonzero(tb["period"][reps] == p)) for p in np.unique(tb["period"])}
        formula = {z: c for z, c in K.spin_nstate(M, N).items() if c}
        assert formula == counted, (M, N)
        assert set(counted) <= set(K.spin_periods(M, N))
        printed = K.spin_nstate_printed(M, N)
        per = K.spin_periods(M, N)
        for z in per:
            if sum(1 for i in per if i < z and z % i == 0) <= 1:
                assert printed[z] == K.spin_nstate(M, N)[z], (M, N, z)
    if M == 8:
        assert K.spin_nstate_printed(8, 4)[8] != K.spin_nstate(8, 4)[8]


SECTORS = [(4, 2, 1), (4, 2, 2), (4, 2, 0), (5, 2, 3), (6, 3, 3), (6, 2, 1), (6, 4, 2), (6, 3, 1), (8, 4, 4),
           (8, 4, 2), (8, 6, 2), (9, 3, 3), (6, 6, 6), (6, 0, 0), (6, 2, 0)]


@pytest.mark.parametrize("M,nu,nd", [s for s in SECTORS if s[0] % 2 == 0])
def test_k_pi_dimension_and_invariance(M, nu, nd):
    """k = pi: dim = (1/M) sum_r (-1)^r tr T^r, the Bloch columns are orthonormal and
    T V = -V."""
    B = O.basis(M, nu, nd)
    assert K.k0_dimension(M, nu, nd, -1) == K.character_dimension(M, nu, nd, B, -1)
    V = K.bloch_matrix(M, nu, nd, B, -1)
    assert V.shape[1] == K.k0_dimension(M, nu, nd, -1)
    if V.shape[1] == 0:
        return
    assert abs((V.T @ V).toarray() - np.eye(V.shape[1])).max() < 1e-14
    T = K.translation_matrix(M, nu, nd, B)
    assert abs(T @ V + V).max() == 0.0


@pytest.mark.parametrize("M,nu,nd", SECTORS)
def test_dimension_is_the_character_count(M, nu, nd):
    """dim k = 0 = (1/M) sum_r tr T^r (brute force on the full basis); the Bloch columns
    are orthonormal and invariant under T.  Sectors (4,2,0), (6,4,2), (8,4,2)
    and (6,2,0) have combined representatives whose Bloch sum vanishes (reading 2)."""
    B = O.basis(M, nu, nd)
    assert K.k0_dimension(M, nu, nd) == K.character_dimension(M, nu, nd, B)
    V = K.bloch_matrix(M, nu, nd, B)
    assert V.shape == (B.shape[0], K.k0_dimension(M, nu, nd))
    assert abs((V.T @ V).toarray() - np.eye(V.shape[1])).max() < 1e-14
    T = K.translation_matrix(M, nu, nd, B)
    assert abs(T @ V - V).max() == 0.0
    if (M, nu, nd) in [(4, 2, 0), (6, 4, 2), (8, 4, 2), (6, 2, 0)]:
        assert K.combined_reps(M, nu, nd)["null"].any()
    if nu == nd:
        assert not K.combined_reps(M, nu, nd)["null"].any()


@pytest.mark.parametrize("M,nu,nd,omega", [(6, 3, 3, 1), (6, 2, 1, 1), (6, 4, 2, 1), (5, 2, 3, 1), (8, 4, 2, 1),
                                         (7, 3, 2, 1), (6, 3, 3, -1), (6, 4, 2, -1), (8, 4, 4, -1), (4, 2, 0, -1)])
def test_free_ring_k0_spectrum(M, nu, nd, omega):
    """U = 0: every eigenvalue of H in the k = 0 (k = pi) basis is a sum of one-particle
    energies -2t cos(2 pi m / M) whose momenta add to 0 (pi) mod 2 pi, and all such sums
    appear."""
    m = O.Model(M, ring(M), 1.0, 0.0)
    B = O.basis(M, nu, nd)
    w = np.linalg.eigvalsh(K.k0_matrix(m, B, K.bloch_matrix(M, nu, nd, B, omega)))
    ref = K.ring_free_k0_levels(M, nu, nd, omega=omega)
    assert w.shape == ref.shape
    assert np.max(np.abs(w - ref)) < 1e-12


@pytest.mark.parametrize("M,nu,nd,nnn,omega", [(6, 3, 2, False, 1), (6, 4, 2, False, 1), (5, 2, 2, False, 1),
                                               (6, 3, 3, True, 1), (7, 3, 2, True, 1), (6, 3, 2, False, -1),
                                               (6, 3, 3, True, -1)])
def test_projector_route(M, nu, nd, nnn, omega):
    """U = 4, eps = 0.3 (nearest- and next-nearest-neighbour rings): the spectrum of V^T H V
    equals that of H on the range of (1/M) sum_r omega^r T^r, computed from the dense
    Jordan-Wigner Hamiltonian and the brute-force translation matrix."""
    m = O.Model(M, ring(M, nnn), 1.0, 4.0, 0.3)
    B = O.basis(M, nu, nd)
    w = np.linalg.eigvalsh(K.k0_matrix(m, B, K.bloch_matrix(M, nu, nd, B, omega)))
    T = K.translation_matrix(M, nu, nd, B).toarray()
    P = sum(float(omega) ** r * np.linalg.matrix_power(T, r) for r in range(M)) / M
    ev, Q = np.linalg.eigh(P)
    Q = Q[:, ev > 0.5]
    w2 = np.linalg.eigvalsh(Q.T @ O.dense_fock(m, nu, nd) @ Q)
    assert np.max(np.abs(w - w2)) < 1e-12


@pytest.mark.parametrize("M,nu,nd", [(6, 3, 3), (6, 4, 2), (8, 4, 4)])
def test_t0_diagonal_double_occupancy(M, nu, nd):
    """t = 0: H in the k = 0 basis is diagonal, entry U times the doubly occupied sites of
    |r_up> T^n |r_dn> plus eps (N_up + N_dn), the quantity Algorithm V counts."""
    m = O.Model(M, ring(M), 0.0, 3.0, 0.25)
    B = O.basis(M, nu, nd)
    H0 = K.k0_matrix(m, B, K.bloch_matrix(M, nu, nd, B))
    cr = K.combined_reps(M, nu, nd)
    keep = ~cr["null"]
    dbl = np.array([bin(int(a) & int(b)).count("1") for a, b in zip(cr["up"][keep], cr["dn"][keep])])
    assert np.array_equal(H0, np.diag(np.diag(H0)))
    assert np.max(np.abs(np.diag(H0) - (3.0 * dbl + 0.25 * (nu + nd)))) < 1e-14


def test_row_form_is_an_isometry():
    """X[i, d] = sqrt(P_i) psi(R_i, d) keeps the norm of a translation-invariant psi and
    determines it: |X| = |psi| for psi = V phi."""
    M, nu, nd = 6, 4, 2
    B = O.basis(M, nu, nd)
    V = K.bloch_matrix(M, nu, nd, B)
    rng = np.random.default_rng(3)
    for _ in range(3):
        psi = V @ rng.standard_normal(V.shape[1])
        X, reps, per = K.row_form(M, nu, nd, B, psi)
        assert abs(np.linalg.norm(X) - np.linalg.norm(psi)) < 1e-13 * np.linalg.norm(psi)
        assert list(per) == [K.spin_tables(M, nu)["period"][int(np.flatnonzero(K.spin_strings(M, nu) == r)[0])]
                             for r in reps]


def test_k0_ground_state_M10_half_filling():
    """M = 10, (5, 5), U = 4: the lowest k = 0 eigenvalue equals the ground-state energy of
    the full sector (the ground state of a ring with an odd number of electrons per spin
    lies at k = 0)."""
    from scipy.sparse.linalg import LinearOperator, eigsh
    M = 10
    m = O.Model(M, ring(M), 1.0, 4.0)
    B = O.basis(M, 5, 5)
    V = K.bloch_matrix(M, 5, 5, B)
    op = LinearOperator((V.shape[1],) * 2, matvec=lambda v: K.k0_apply(m, B, V, np.ravel(v)), dtype=np.float64)
    w = eigsh(op, k=1, which="SA", tol=1e-13, v0=np.ones(V.shape[1]))[0]
    x0 = np.random.default_rng(0).standard_normal(B.shape[0])
    E0 = O.lanczos(m, B, x0, maxit=300, tol=1e-13)["E0"]
    assert abs(w[0] - E0) < 1e-10


def test_rep_columns_follow_table2():
    """Column order of Table I for one spin: each representative followed by its
    translations, with the phases of Table II (M = 4, N = 2: 0011, 1001(-), 1100, 0110,
    0101, 1010(-)); for other sizes a bijection onto all strings."""
    bits, sign = K.rep_columns(4, 2)
    rows = _rows("k0_table2_M4_N2.txt")
    assert [format(int(b), "04b") for b in bits] == [r[0] for r in rows]
    assert [int(x) for x in sign] == [int(r[4]) for r in rows]
    for M, N in [(6, 3), (8, 4), (9, 3), (6, 0), (5, 5), (10, 4)]:
        b, s = K.rep_columns(M, N)
        assert np.array_equal(np.sort(b), K.spin_strings(M, N))
        assert set(np.unique(s).tolist()) <= {-1.0, 1.0}


@pytest.mark.parametrize("M,nu,nd,omega", [(6, 4, 2, 1), (8, 4, 3, 1), (6, 3, 3, -1)])
def test_row_form_rep_is_an_isometry(M, nu, nd, omega):
    """X[i, (j, n)] = sqrt(P_i) <R_i (x) T^n R_j | psi> keeps the norm and the inner products
    of states of the sector."""
    B = O.basis(M, nu, nd)
    V = K.bloch_matrix(M, nu, nd, B, omega)
    rng = np.random.default_rng(7)
    a, b = (np.asarray(V @ rng.standard_normal(V.shape[1])) for _ in range(2))
    Xa, _, _ = K.row_form_rep(M, nu, nd, B, a)
    Xb, _, _ = K.row_form_rep(M, nu, nd, B, b)
    assert abs(float(np.sum(Xa * Xb)) - float(a @ b)) < 1e-12 * np.linalg.norm(a) * np.linalg.norm(b)


# ------------------------------------------------------------------ several translations (torus)

def torus_bonds(Lx, Ly):
    b = set()
    for y in range(Ly):
        for x in range(Lx):
            s = x + Lx * y
            for dx, dy in ((1, 0), (0, 1)):
                s2 = (x + dx) % Lx + Lx * ((y + dy) % Ly)
                b.add((min(s, s2), max(s, s2)))
    return sorted(b)


@pytest.mark.parametrize("M,nu,nd,omega", [(6, 3, 3, 1), (6, 4, 2, 1), (6, 3, 3, -1), (6, 4, 2, -1), (5, 2, 2, 1)])
def test_group_construction_equals_chain(M, nu, nd, omega):
    """One generator (the chain's T): the group construction spans the same space as the
    chain construction (equal projectors V V^T)."""
    B = O.basis(M, nu, nd)
    Vg = K.bloch_matrix_group(M, nu, nd, B, [[(i - 1) % M for i in range(M)]], [omega])
    V = K.bloch_matrix(M, nu, nd, B, omega)
    assert Vg.shape[1] == V.shape[1]
    assert abs((Vg @ Vg.T - V @ V.T)).max() < 1e-13


@pytest.mark.parametrize("Lx,Ly,nu,nd", [(3, 3, 2, 2), (3, 3, 3, 2), (4, 3, 2, 2), (4, 3, 3, 1)])
def test_torus_free_spectrum_and_dimension(Lx, Ly, nu, nd):
    """Torus translations, every real character: dimension = (1/|G|) sum_g chi(g) tr g by brute
    force, Bloch columns orthonormal and invariant (g V = chi(g) V), and at U = 0 the complete
    spectrum equals the sums of one-particle energies -2t (cos kx + cos ky) with total momentum
    of the character."""
    M = Lx * Ly
    gens = K.torus_translations(Lx, Ly)
    B = O.basis(M, nu, nd)
    m = O.Model(M, torus_bonds(Lx, Ly), 1.0, 0.0)
    for cx in ([1, -1] if Lx % 2 == 0 else [1]):
        for cy in ([1, -1] if Ly % 2 == 0 else [1]):
            V = K.bloch_matrix_group(M, nu, nd, B, gens, [cx, cy])
            assert V.shape[1] == K.character_dimension_group(M, nu, nd, B, gens, [cx, cy])
            assert abs((V.T @ V).toarray() - np.eye(V.shape[1])).max() < 1e-13
            for g, c in zip(gens, (cx, cy)):
                P = np.zeros((B.shape[0], B.shape[0]))
                idx = {int(v): k for k, v in enumerate(B.tolist())}
                for k, I in enumerate(B.tolist()):
                    I2, s = K._act_two_spin(M, I, nu, nd, g)
                    P[idx[I2], k] = s
                assert abs(P @ V.toarray() - c * V.toarray()).max() < 1e-13
            w = np.linalg.eigvalsh(K.k0_matrix(m, B, V))
            ref = K.torus_free_levels(Lx, Ly, nu, nd, cx < 0, cy < 0)
            assert w.shape == ref.shape and np.max(np.abs(w - ref)) < 1e-12


def test_group_character_must_be_consistent():
    """-1 on a generator of odd order is no character: refused."""
    with pytest.raises(ValueError):
        K.group_character(K.site_group([[(i - 1) % 5 for i in range(5)]]), [-1])


def test_group_columns_reduce_to_the_chain_and_cover_the_strings():
    """One generator: group_columns is the chain's column order with its signs; tori: every
    string once; row_form_group preserves inner products."""
    for M, N in [(4, 2), (6, 3), (8, 4), (6, 0)]:
        b1, s1 = K.rep_columns(M, N)
        b2, s2 = K.group_columns(M, N, [[(i - 1) % M for i in range(M)]])
        assert np.array_equal(b1, b2) and np.array_equal(s1, s2)
    for Lx, Ly, N in [(3, 3, 2), (4, 2, 3), (3, 3, 4)]:
        b, s = K.group_columns(Lx * Ly, N, K.torus_translations(Lx, Ly))
        assert np.array_equal(np.sort(b), K.spin_strings(Lx * Ly, N))
    M, nu, nd = 8, 3, 3
    gens = K.torus_translations(4, 2)
    B = O.basis(M, nu, nd)
    V = K.bloch_matrix_group(M, nu, nd, B, gens, [-1, 1])
    rng = np.random.default_rng(5)
    a, b = (np.asarray(V @ rng.standard_normal(V.shape[1])) for _ in range(2))
    Xa, _, _ = K.row_form_group(M, nu, nd, B, a, gens)
    Xb, _, _ = K.row_form_group(M, nu, nd, B, b, gens)
    assert abs(float(np.sum(Xa * Xb)) - float(a @ b)) < 1e-12 * np.linalg.norm(a) * np.linalg.norm(b)


@pytest.mark.parametrize("Lx,Ly,nu,nd,chars", [(3, 2, 3, 3, (1, 1)), (3, 2, 3, 2, (1, -1)), (2, 3, 2, 2, (-1, 1)),
                                               (2, 3, 3, 3, (-1, 1)), (2, 3, 3, 2, (1, 1))])
def test_group_projector_route_torus_6_sites(Lx, Ly, nu, nd, chars):
    """3 x 2 and 2 x 3 tori (a length-2 direction carries one bond per pair), U = 4,
    eps = 0.3: the spectrum of V^T H V for each real character equals that of H on the range
    of (1/|G|) sum_g chi(g) g, from the dense Jordan-Wigner Hamiltonian and brute-force g."""
    M = Lx * Ly
    gens = K.torus_translations(Lx, Ly)
    m = O.Model(M, torus_bonds(Lx, Ly), 1.0, 4.0, 0.3)
    B = O.basis(M, nu, nd)
    w = np.linalg.eigvalsh(K.k0_matrix(m, B, K.bloch_matrix_group(M, nu, nd, B, gens, list(chars))))
    els = K.site_group(gens)
    chi = K.group_character(els, list(chars))
    idx = {int(v): k for k, v in enumerate(B.tolist())}
    P = np.zeros((B.shape[0], B.shape[0]))
    for (p, _), c in zip(els, chi):
        for k, I in enumerate(B.tolist()):
            I2, s = K._act_two_spin(M, I, nu, nd, p)
            P[idx[I2], k] += c * s / len(els)
    ev, Q = np.linalg.eigh((P + P.T) / 2)
    Q = Q[:, ev > 0.5]
    w2 = np.linalg.eigvalsh(Q.T @ O.dense_fock(m, nu, nd) @ Q)
    assert w.shape == w2.shape and np.max(np.abs(w - w2)) < 1e-12
