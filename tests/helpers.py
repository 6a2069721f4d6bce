"""Helpers shared by the parity tests: build both sides from one workload description."""
import numpy as np

from oracle import hub_oracle as O


def oracle_model(w):
    return O.Model(w["M"], w["bonds"], w["t"], w["U"], w.get("eps"))


def abs_bound(model, B, x, rows=None):
    """(|H| |x|)_n over rows (r0, r1): the scale of the per-entry tolerance."""
    return O.apply(model, B, x, rows=rows, absolute=True)


def assert_entrywise(y, ref, bound, rtol=1e-13):
    """|y - ref| <= rtol * (|H||x|) + 1e-300 for every entry (per-entry tolerance of the apply)."""
    err = np.abs(y - ref)
    bad = err > rtol * bound + 1e-300
    if bad.any():
        k = int(np.argmax(err / (bound + 1e-300)))
        raise AssertionError(f"{int(bad.sum())} entries exceed {rtol:g}*|H||x|; worst at {k}: "
                             f"got {y[k]!r}, want {ref[k]!r}, bound {bound[k]!r}")
