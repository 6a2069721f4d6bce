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
