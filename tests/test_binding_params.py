"""Host logic of the binding (no GPU): the autograd Functions call Hubbard.ensure_params,
which rebuilds the hopping tables only when the parameters change."""
import numpy as np

from paper_1307_7542_gb300 import hub as H


def _stub(M=4, nb=4):
    """A Hubbard object without a library handle; set_params records its calls."""
    m = object.__new__(H.Hubbard)
    m.M, m.count_up, m.count_dn = M, 6, 6
    m.D = 36
    m.bonds = np.zeros((nb, 2), dtype=np.int32)
    m.calls = []

    def set_params(t, U, eps=None):
        m.calls.append((np.array(t), np.array(U), None if eps is None else np.array(eps)))
        m.t = np.asarray(t, dtype=np.float64).reshape(nb).copy()
        m.U = np.asarray(U, dtype=np.float64).reshape(M).copy()
        m.eps = np.zeros(M) if eps is None else np.asarray(eps, dtype=np.float64).reshape(M).copy()

    m.set_params = set_params
    return m


def test_ensure_params_skips_unchanged():
    m = _stub()
    t, U, e = np.ones(4), np.full(4, 4.0), np.zeros(4)
    assert m.ensure_params(t, U, e) is True           # first call: nothing set yet
    assert len(m.calls) == 1
    assert m.ensure_params(t.copy(), U.copy(), None) is False
    assert m.ensure_params(1.0, 4.0, e) is False      # scalars broadcast to the same arrays
    assert len(m.calls) == 1
    t2 = t.copy()
    t2[2] += 1e-12
    assert m.ensure_params(t2, U, e) is True
    assert len(m.calls) == 2


def test_ensure_params_leaves_a_momentum_sector():
    m = _stub()
    m.ensure_params(np.ones(4), np.full(4, 4.0), None)
    m.D = 10                                          # a momentum sector is active
    assert m.ensure_params(np.ones(4), np.full(4, 4.0), None) is True
    assert len(m.calls) == 2


def test_apply_host_dispatch(monkeypatch):
    """Hubbard.apply_host: a 1-D array goes to hub_apply_host, a 2-D array to
    hub_apply_host_many with the row count; y is allocated like x; bad shapes are refused."""
    import pytest
    calls = []
    monkeypatch.setattr(H, "hub_apply_host", lambda h, x, y, s=None: calls.append(("one", h, x.shape, y.shape)))
    monkeypatch.setattr(H, "hub_apply_host_many",
                        lambda h, n, x, y, s=None: calls.append(("many", h, n, x.shape, y.shape)))
    m = _stub()
    m.h = "handle"          # a marker only: cleared below so that close() frees nothing
    try:
        y = m.apply_host(np.zeros(36))
        assert y.shape == (36,) and calls[-1] == ("one", "handle", (36,), (36,))
        y = m.apply_host(np.zeros((3, 36)))
        assert y.shape == (3, 36) and calls[-1] == ("many", "handle", 3, (3, 36), (3, 36))
        out = np.empty((2, 36))
        assert m.apply_host(np.zeros((2, 36)), out) is out
        with pytest.raises(ValueError):
            m.apply_host(np.zeros((2, 36)), np.empty((3, 36)))
        with pytest.raises(ValueError):
            m.apply_host(np.zeros((2, 3, 6)))
        assert len(calls) == 3
    finally:
        m.h = None
