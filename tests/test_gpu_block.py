"""Block Lanczos (hub_lanczos_block): low-lying levels with their multiplicities, against the
dense spectrum of the oracle's Hamiltonian (exact diagonalisation of tiny clusters), on the
fast path and the FP64 path."""
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


def _dense_from_rows(w):
    """Dense H from the oracle's two-spin rows and diagonal (any size the oracle handles)."""
    om = oracle_model(w)
    B = O.basis(w["M"], w["n_up"], w["n_dn"])
    D = B.shape[0]
    Hd = np.diag(O.diagonal(om, B))
    for n in range(D):
        cols, vals = O.row(om, B, n)
        Hd[n, cols] += vals
    return Hd


def _check_levels(ev, res, exact, k, scale):
    """Every converged Ritz value (residual < 1e-8) is an eigenvalue; the converged ones, from
    the bottom up to the first unconverged, are the lowest eigenvalues with multiplicity (for
    levels of multiplicity <= k)."""
    conv = [i for i in range(len(ev)) if res[i] < 1e-8 * scale]
    assert len(conv) >= 4
    for i in conv:
        assert np.min(np.abs(exact - ev[i])) < 1e-9 * scale, (i, ev[i])
    m = 0
    while m < len(ev) and res[m] < 1e-8 * scale:
        m += 1
    # the lowest m Ritz values are the lowest m eigenvalues, multiplicities included, except
    # that a level above multiplicity k can show at most k copies: compare level by level
    levels, counts = [], []
    for e in exact:
        if levels and abs(e - levels[-1]) < 1e-7 * scale:
            counts[-1] += 1
        else:
            levels.append(e)
            counts.append(1)
    got = ev[:m]
    pos = 0
    for lev, c in zip(levels, counts):
        if pos >= m:
            break
        n_here = int(np.sum(np.abs(got - lev) < 1e-7 * scale))
        assert n_here == min(c, k) or pos + n_here == m, (lev, c, n_here)
        pos += n_here
    return m


@pytest.mark.parametrize("case,k,steps", [("ring7_fast", 4, 100), ("ring6_fp64_eps", 3, 60), ("ring8_fast", 4, 120)])
def test_block_levels_match_dense(hub, case, k, steps):
    if case == "ring7_fast":
        w = dict(M=7, n_up=3, n_dn=3, bonds=W.ring_bonds(7), t=np.ones(7), U=np.full(7, 4.0), eps=np.zeros(7))
    elif case == "ring6_fp64_eps":
        w = dict(M=6, n_up=3, n_dn=2, bonds=W.ring_bonds(6), t=np.ones(6), U=np.full(6, 3.0),
                 eps=W.uniform(71, 6, -0.05, 0.05))
    else:
        w = dict(W.ring8())
    m = hub.Hubbard(w["M"], w["n_up"], w["n_dn"], w["bonds"], w["t"], w["U"], w["eps"])
    try:
        exact = np.linalg.eigvalsh(_dense_from_rows(w))
        scale = max(1.0, float(np.max(np.abs(exact))))
        ev, res = hub.hub_lanczos_block(m.h, k, None, steps, 3 * k)
        assert np.all(np.diff(ev) >= -1e-12 * scale)
        n_conv = _check_levels(ev, res, exact, k, scale)
        assert abs(ev[0] - exact[0]) < 1e-10 * scale
        print(f"{case}: {n_conv} converged Ritz values, lowest levels {np.round(ev[:n_conv], 8)}")
    finally:
        m.close()


def test_block_resolves_multiplicity_single_vector_does_not(hub):
    """On the 7-site ring (degenerate levels from momenta +-q) the single-vector spectrum lists
    a degenerate level once; the block form with k >= its multiplicity lists every copy."""
    w = dict(M=7, n_up=3, n_dn=3, bonds=W.ring_bonds(7), t=np.ones(7), U=np.full(7, 4.0), eps=np.zeros(7))
    m = hub.Hubbard(w["M"], w["n_up"], w["n_dn"], w["bonds"], w["t"], w["U"], w["eps"])
    try:
        exact = np.linalg.eigvalsh(_dense_from_rows(w))
        scale = max(1.0, float(np.max(np.abs(exact))))
        # the lowest level with multiplicity > 1
        i = 0
        while i + 1 < len(exact) and abs(exact[i + 1] - exact[i]) > 1e-7 * scale:
            i += 1
        g = int(np.sum(np.abs(exact - exact[i]) < 1e-7 * scale))
        assert g >= 2
        single, _ = hub.hub_lanczos_spectrum(m.h, None, 200, 12)
        assert int(np.sum(np.abs(single - exact[i]) < 1e-7 * scale)) == 1
        ev, res = hub.hub_lanczos_block(m.h, max(g, 2), None, 100, 12)
        assert int(np.sum(np.abs(ev - exact[i]) < 1e-7 * scale)) == g
    finally:
        m.close()


def test_block_of_one_is_lanczos_ground(hub):
    """k = 1 with the same start vector: the lowest Ritz value equals hub_lanczos_ground's E0."""
    w = W.ring8()
    m = hub.Hubbard(8, 4, 4, w["bonds"], w["t"], w["U"], w["eps"])
    try:
        x0 = torch.from_numpy(W.normal(3, m.D)).cuda()
        E0 = m.ground(x0, maxit=300, tol=1e-13)["E0"]
        ev, res = hub.hub_lanczos_block(m.h, 1, x0, 80, 1)
        assert abs(ev[0] - E0) < 1e-10 * abs(E0)
        assert res[0] < 1e-8
    finally:
        m.close()


def test_block_refusals(hub):
    w = W.ring8()
    m = hub.Hubbard(8, 4, 4, w["bonds"], w["t"], w["U"], w["eps"])
    try:
        for k, steps in ((9, 10), (0, 10), (4, 200), (2, 0)):
            with pytest.raises(hub.HubError) as e:
                hub.hub_lanczos_block(m.h, k, None, steps, 4)
            assert e.value.code == hub.HUB_ERR_ARG
        x = torch.from_numpy(W.normal(4, m.D)).cuda()
        X = torch.cat([x, x])                       # two equal start vectors: dependent
        with pytest.raises(hub.HubError) as e:
            hub.hub_lanczos_block(m.h, 2, X, 10, 4)
        assert e.value.code == hub.HUB_ERR_ARG
    finally:
        m.close()
