"""The fast (double-float) product against the per-entry bound on inputs chosen to break it.

The bound is |y - y_ref|_n <= 1e-13 (|H||x|)_n for every entry (Eq. 11 products compared
with the oracle's two-spin rows).  The fast path holds x as FP32 pairs scaled so that
max |x| lies in [1, 2); vectors whose nonzero entries span more than 2^80, vectors whose
largest entry lies outside [2^-823, 2^877], and models with t, U or a site energy of
magnitude outside {0} and [2^-16, 2^16] are multiplied by the FP64 kernel instead.  These
cases sit on both sides of that window and maximise the rounding the hopping sums see: a
huge spike, blocks of tiny entries, and positive entries whose low parts are as large as
they can be (all of one sign), with partial sums that stay large.
"""
import numpy as np
import pytest

from helpers import abs_bound, assert_entrywise, oracle_model
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


def _model(hub, w):
    return hub.Hubbard(w["M"], w["n_up"], w["n_dn"], w["bonds"], w["t"], w["U"], w.get("eps"))


def _check(hub, w, x, rows=None):
    """hub_apply (AUTO: fast path or its FP64 route) against the oracle, entry by entry."""
    m = _model(hub, w)
    om = oracle_model(w)
    try:
        B = O.basis(w["M"], w["n_up"], w["n_dn"])
        y = m.apply(torch.from_numpy(x).cuda()).cpu().numpy()
        hub.hub_check(m.h)
        D = B.shape[0]
        spans = [(0, D)] if rows is None else rows
        worst = 0.0
        for r0, r1 in spans:
            ref = O.apply(om, B, x, rows=(r0, r1))
            bound = abs_bound(om, B, x, rows=(r0, r1))
            assert_entrywise(y[r0:r1], ref, bound)
            worst = max(worst, float(np.max(np.abs(y[r0:r1] - ref) / (bound + 1e-300))))
        return worst
    finally:
        m.close()


def _ring(M, n_up, n_dn, t=1.0, U=4.0, eps=False):
    return dict(M=M, n_up=n_up, n_dn=n_dn, bonds=W.ring_bonds(M), t=np.full(M, t), U=np.full(M, U),
                eps=W.uniform(31, M, -0.5, 0.5) if eps else np.zeros(M))


def _unit_entries(seed, n):
    """Entries of magnitude in [0.5, 1.5) with random signs (a known exponent range)."""
    return W.uniform(seed, n, 0.5, 1.5) * np.where(W.uniform(seed + 1, n) < 0.5, -1.0, 1.0)


@pytest.mark.parametrize("spike", [1e15, 1e30, -1e200])
def test_spike(hub, spike):
    """One entry far above the rest (1e15 is inside the window, 1e30 and 1e200 outside)."""
    w = _ring(10, 5, 5)
    D = 252 * 252
    x = _unit_entries(40, D)
    x[D // 3 + 5] = spike
    _check(hub, w, x)


@pytest.mark.parametrize("log2_rel", [-60, -78, -90, -130, -160, -1060])
def test_tiny_block(hub, log2_rel):
    """A block of rows whose entries sit 2^log2_rel below the largest entry (-60, -78:
    inside the window; -90, -130, -160: outside; -1060: FP64 subnormals).  Rows of the
    block whose neighbours are all tiny have a tiny (|H||x|)_n, so flushed or truncated
    low parts would show as large relative errors."""
    w = _ring(10, 5, 5)
    n = 252
    x = _unit_entries(41, n * n)
    x[40 * n:90 * n] *= 2.0 ** log2_rel
    _check(hub, w, x)


@pytest.mark.parametrize("scale_exp", [-820, 870, -830, 880])
def test_vector_scale_limits(hub, scale_exp):
    """Whole vectors scaled by 2^scale_exp: inside (-820, 870) and outside (-830, 880) the
    range of largest entries the fast path takes."""
    w = _ring(9, 4, 5)
    x = _unit_entries(42, 126 * 126) * 2.0 ** scale_exp
    _check(hub, w, x)


@pytest.mark.parametrize("t,U,eps", [(2.0 ** -15, 4.0, 0.0), (2.0 ** -17, 4.0, 0.0), (1.0, 1e-6, 0.0),
                                     (1.0, 4.0, 3e-6), (3e4, 2.0 ** 15, 0.0), (1.0, 7e4, 0.0)])
def test_parameter_range(hub, t, U, eps):
    """Models inside (t = 2^-15; t = 3e4 with U = 2^15) and outside (t = 2^-17, U = 1e-6, a
    site energy 3e-6, U = 7e4) the parameter range of the fast path, with entries that
    cover the whole window."""
    M = 10
    w = dict(M=M, n_up=5, n_dn=4, bonds=W.ring_bonds(M), t=np.full(M, t), U=np.full(M, U),
             eps=np.where(np.arange(M) % 3 == 0, eps, 0.0))
    D = 252 * 210
    x = _unit_entries(43, D) * 2.0 ** np.floor(W.uniform(44, D, -78, 0))
    _check(hub, w, x)


def _max_low_parts(seed, n, lo_exp=-10):
    """Positive entries 2^U[lo_exp, 0] (1 + m), m a random 23-bit fraction, plus 0.999 of
    the last place of the FP32 high part: each FP64 value splits into an FP32 high part and
    a low part of nearly one unit in its last place, all of one sign."""
    e = np.floor(W.uniform(seed, n, lo_exp, 1)).astype(np.int64)
    m = np.floor(W.uniform(seed + 1, n) * (1 << 23)) / (1 << 23)
    hi = np.ldexp(1.0 + m, e)
    return hi + np.ldexp(0.999, e - 23)


@pytest.mark.parametrize("case", ["ring14_t1", "ring14_t037_eps", "square4x4_66"])
def test_one_signed_low_parts(hub, case):
    """All entries positive with maximal, one-signed low parts and magnitudes over three
    decades, so the running sums of a row stay large while its terms add rounding errors:
    the worst case of the uncompensated double-float sum."""
    if case == "ring14_t1":
        w, rows = _ring(14, 7, 7), None
    elif case == "ring14_t037_eps":
        w, rows = _ring(14, 7, 7, t=0.37, U=3.3, eps=True), None
    else:
        w = dict(W.square4x4(4.0), n_up=6, n_dn=6)
        D = 8008 * 8008
        rows = [(0, 4000), (D // 2, D // 2 + 4000), (D - 4000, D)]
    D = O.basis(w["M"], w["n_up"], 0).shape[0] * O.basis(w["M"], 0, w["n_dn"]).shape[0]
    x = _max_low_parts(50, D)
    worst = _check(hub, w, x, rows)
    print(f"{case}: worst |dy| / (|H||x|) = {worst:.3e}")


@pytest.mark.parametrize("case", ["sign_mixed", "zeros"])
def test_bound_with_cancellation(hub, case):
    """Terms of both signs that cancel to near zero (y_n much smaller than (|H||x|)_n), and
    exact zeros mixed with maximal low parts."""
    w = _ring(12, 6, 6)
    D = 924 * 924
    x = _max_low_parts(60, D)
    if case == "sign_mixed":
        x *= np.where(W.uniform(61, D) < 0.5, -1.0, 1.0)
    else:
        x[W.uniform(62, D) < 0.4] = 0.0
    _check(hub, w, x)
