"""Batched persistent Lanczos (all sectors x parameter sets of an impurity star in one
launch) against the oracle and against one-at-a-time GPU Lanczos."""
import math

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


def _aim_params(n_sets):
    ps = [W.aim_star(k) for k in range(n_sets)]
    return ps[0]["bonds"], np.stack([p["t"] for p in ps]), np.stack([p["U"] for p in ps]), \
        np.stack([p["eps"] for p in ps])


def test_batch_all_sectors_vs_oracle(hub):
    """All 81 sectors of the 8-site impurity star for one parameter set: E0 within 1e-10
    (relative) of the oracle's plain Lanczos in the two-spin basis."""
    bonds, t, U, eps = _aim_params(2)
    jobs = [(a, b, 1) for a in range(9) for b in range(9)]
    jn, jd, jp = (np.array(c) for c in zip(*jobs))
    E0, it, st = hub.hub_batch_ground(8, bonds, t, U, eps, jn, jd, jp, maxit=400, tol=1e-13)
    assert np.all(np.isin(st, [0, 1]))
    om = O.Model(8, bonds, t[1], U[1], eps[1])
    for k, (a, b, _) in enumerate(jobs):
        B = O.basis(8, a, b)
        if B.shape[0] <= 200:
            ref = np.linalg.eigvalsh(np.column_stack([O.apply(om, B, e) for e in np.eye(B.shape[0])]))[0]
        else:
            ref = O.lanczos(om, B, W.normal(k, B.shape[0]), maxit=600, tol=1e-13)["E0"]
        assert abs(E0[k] - ref) <= 1e-10 * max(1.0, abs(ref)), (a, b, E0[k], ref)


def test_batch_matches_single_jobs(hub):
    """Jobs over several parameter sets equal hub_lanczos_ground run one job at a time."""
    bonds, t, U, eps = _aim_params(4)
    jobs = [(4, 4, 3), (3, 5, 0), (4, 3, 2), (0, 8, 1), (8, 8, 2), (2, 1, 3)]
    jn, jd, jp = (np.array(c) for c in zip(*jobs))
    E0, it, st = hub.hub_batch_ground(8, bonds, t, U, eps, jn, jd, jp, maxit=400, tol=1e-13)
    for k, (a, b, p) in enumerate(jobs):
        m = hub.Hubbard(8, a, b, bonds, t[p], U[p], eps[p])
        try:
            r = m.ground(torch.from_numpy(W.normal(k, m.D)).cuda(), maxit=400, tol=1e-13)
            assert abs(E0[k] - r["E0"]) <= 1e-10 * max(1.0, abs(r["E0"]))
        finally:
            m.close()


def test_batch_rejects_oversize_and_bad_jobs(hub):
    bonds = W.ring_bonds(12)
    t, U = np.ones((1, 12)), np.full((1, 12), 4.0)
    with pytest.raises(hub.HubError) as e:
        hub.hub_batch_ground(12, bonds, t, U, None, [6], [6], [0])          # 924^2 > 8192
    assert e.value.code == hub.HUB_ERR_ARG
    with pytest.raises(hub.HubError) as e:
        hub.hub_batch_ground(12, bonds, t, U, None, [1], [1], [1])          # parameter set out of range
    assert e.value.code == hub.HUB_ERR_ARG
