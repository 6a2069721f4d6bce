"""The benchmark lattice's ground-state energy against the oracle: 4x4 periodic Hubbard
lattice, half filling (8, 8), t = 1, D = 165,636,900.  The reference values in
tests/golden/square4x4_E0.txt were written by tests/golden/make_square4x4_E0.py with the CPU
oracle alone (two-spin basis, binary-search products, plain Lanczos from the seed-0 normal
start vector to |dE0| < 1e-12).  The GPU runs the same recurrence from the same start vector,
on the fast path and with HUB_MODE_FP64, and must agree within 1e-10 relative."""
import math
import os

import pytest

from conftest import ROOT, golden
from paper_1307_7542_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")


def _reference(U):
    """(E0, iterations) the oracle wrote for this U, or None."""
    if not os.path.exists(os.path.join(ROOT, "tests", "golden", "square4x4_E0.txt")):
        return None
    rows = {float(r[0]): (float(r[1]), int(r[2])) for r in golden("square4x4_E0.txt")}
    return rows.get(float(U))


@pytest.fixture(scope="module")
def hub(cuda_ok):
    import __graft_entry__
    __graft_entry__.build()
    from paper_1307_7542_gb300 import hub as H
    return H


@pytest.mark.parametrize("U", [2.0, 4.0, 8.0])
@pytest.mark.parametrize("mode", ["fast", "fp64"])
def test_square4x4_E0_matches_oracle(hub, U, mode):
    row = _reference(U)
    if row is None:
        pytest.skip(f"no oracle value for U = {U:g} in tests/golden/square4x4_E0.txt")
    ref, _ = row
    w = W.square4x4(U)
    m = hub.Hubbard(16, 8, 8, w["bonds"], w["t"], w["U"], w["eps"])
    try:
        if mode == "fp64":
            hub.hub_set_mode(m.h, hub.HUB_MODE_FP64)
        x0 = torch.from_numpy(W.normal(0, m.D)).cuda()
        r = m.ground(x0, maxit=400, tol=1e-12)
        assert r["status"] == 0, r
        assert abs(r["E0"] - ref) <= 1e-10 * abs(ref), (r["E0"], ref)
        assert math.isfinite(r["E0"])
    finally:
        m.close()
        torch.cuda.empty_cache()
