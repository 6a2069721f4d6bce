"""Host logic of the autotuner (no GPU): coordinate descent over the knobs with a stand-in
for the timed child process."""
import pytest

from paper_1307_7542_gb300 import autotune as A


def test_coordinate_descent_keeps_faster_settings_and_skips_repeats(monkeypatch):
    """A change is kept only when at least MARGIN faster; every setting is timed once."""
    cost = {("HUB_DN_BATCH", 1): 1.10, ("HUB_DN_BATCH", 2): 1.00, ("HUB_DN_BATCH", 3): 0.995,   # 0.5 %: kept out
            ("HUB_DN_MINB", 4): 1.05, ("HUB_DN_MINB", 5): 1.00, ("HUB_DN_MINB", 6): 0.90}
    timed = []

    def fake_measure(knobs, what, steps):
        timed.append(tuple(sorted(knobs.items())))
        t = 1.0
        for k, v in knobs.items():
            t *= cost.get((k, v), 1.0)
        return t

    monkeypatch.setattr(A, "measure", fake_measure)
    space = {"HUB_DN_BATCH": [1, 2, 3], "HUB_DN_MINB": [4, 5, 6]}
    log = []
    best, t = A.coordinate_descent(space, {"HUB_DN_BATCH": 2, "HUB_DN_MINB": 5}, "apply", 3, log)
    assert best == {"HUB_DN_BATCH": 2, "HUB_DN_MINB": 6}
    assert t == pytest.approx(0.90)
    assert len(timed) == len(set(timed)) == 1 + 2 + 2
    assert len(log) == len(timed)


def test_tags_are_distinct_and_filesystem_safe():
    a = A._tag({"HUB_BANK_CAP": -2, "HUB_DN_BATCH": 2})
    b = A._tag({"HUB_BANK_CAP": 2, "HUB_DN_BATCH": 2})
    assert a != b and "-" not in a and "/" not in a
