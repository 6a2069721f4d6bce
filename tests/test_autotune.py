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


def test_only_one_group_keeps_the_stored_others(monkeypatch, tmp_path):
    """--only small tunes the small-sector knobs and keeps the stored defines, timings and
    trials of the other groups in tuned.json."""
    import json
    tuned = tmp_path / "tuned.json"
    stored = {"gpu": "x", "defines": dict(A.DEFAULTS, HUB_DN_BATCH=4, HUB_BATCH_THREADS=512),
              "lanczos_step_ms_4x4": 4.9, "aim_batch_ms": 62.0,
              "trials": [{"what": "apply", "knobs": {}, "ms": 4.9}, {"what": "small", "knobs": {}, "ms": 9.0}]}
    tuned.write_text(json.dumps(stored))
    monkeypatch.setattr(A, "TUNED", str(tuned))
    monkeypatch.setattr(A, "measure", lambda knobs, what, steps: 1.0 if knobs["HUB_SMALL_THREADS"] != 128 else 0.5)
    assert A.main(["--only", "small", "--write", "--steps", "3"]) == 0
    out = json.loads(tuned.read_text())
    assert out["defines"]["HUB_SMALL_THREADS"] == 128
    assert out["defines"]["HUB_DN_BATCH"] == 4 and out["defines"]["HUB_BATCH_THREADS"] == 512
    assert out["lanczos_step_ms_4x4"] == 4.9 and out["aim_batch_ms"] == 62.0 and out["ring8_ground_ms"] == 0.5
    whats = [t["what"] for t in out["trials"]]
    assert whats[0] == "apply" and all(w == "small" for w in whats[1:]) and len(whats) > 2
