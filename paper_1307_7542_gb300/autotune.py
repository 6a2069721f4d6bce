"""Autotuner for the kernel shape knobs (run on the GPU it tunes for).

The fast apply (csrc/hub_fast.cu) and the batched solver (csrc/hub_batch.cu) take their launch
shapes from compile-time knobs:

* ``HUB_DN_LANE_COLS`` -- columns a pass-2 lane owns (2: 64-bit loads, 4: 128-bit loads);
* ``HUB_DN_BATCH``     -- strip rows whose loads pass 2 issues together (2 or 4);
* ``HUB_DN_MINB``      -- resident pass-2 CTAs per SM the register allocation aims for;
* ``HUB_BANK_CAP``     -- distinct columns per shared-memory bank and step in the pass-1
  schedule (k > 0 fixed, 0 adaptive, -k adaptive capped at k);
* ``HUB_FUSED_UPDATE`` -- 1: the Lanczos update r_j = w - c r_{j-1} is formed by pass 1 while
  it stages the rows; 0: a separate vector pass before pass 1;
* ``HUB_UPD_Q``        -- column quads per thread whose loads the fused update issues together;
* ``HUB_UP_THREADS``   -- threads of the pass-1 CTA (1024, 768 or 512; fewer leave more registers);
* ``HUB_BATCH_THREADS`` -- threads per CTA of the batched persistent solver.

For each candidate setting this module builds one copy of the library, times on the GPU what
the knob affects (one Lanczos step at 4x4 half filling for the apply knobs; the 5184-job
impurity batch of 81 sectors x 64 parameter sets for the batched knob), each in a fresh
process, and keeps the fastest by coordinate descent from the current setting (a change is
kept only if it is at least 1 % faster).  ``--write`` stores the result in tuned.json, which
``build()`` compiles in.

    python -m paper_1307_7542_gb300.autotune [--write] [--steps 20]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
TUNE_DIR = os.path.join(PKG, "_build", "tune")
TUNED = os.path.join(PKG, "tuned.json")

APPLY_SPACE = {
    "HUB_DN_LANE_COLS": [2, 4],
    "HUB_DN_BATCH": [2, 4],
    "HUB_DN_MINB": [3, 4, 5, 6],
    "HUB_BANK_CAP": [2, 3, 0, -2],
    "HUB_FUSED_UPDATE": [1, 0],
    "HUB_UPD_Q": [1, 2],
    "HUB_UP_THREADS": [1024, 768, 512],
}
BATCH_SPACE = {"HUB_BATCH_THREADS": [256, 512, 1024]}
DEFAULTS = {"HUB_DN_LANE_COLS": 4, "HUB_DN_BATCH": 2, "HUB_DN_MINB": 4, "HUB_BANK_CAP": 2,
            "HUB_FUSED_UPDATE": 0, "HUB_UPD_Q": 1, "HUB_UP_THREADS": 1024, "HUB_BATCH_THREADS": 256}
MARGIN = 0.01


def _tag(knobs: dict) -> str:
    return "_".join(f"{k.replace('HUB_', '').lower()}{v}".replace("-", "m") for k, v in sorted(knobs.items()))


def _child_apply(lib_path: str, steps: int) -> float:
    """ms per Lanczos step at 4x4 PBC (8,8), U = 4, with the library at lib_path."""
    import torch
    from paper_1307_7542_gb300 import hub, workloads as W
    hub.LIB_PATH = lib_path
    hub._lib = None
    w = W.square4x4(4.0)
    m = hub.Hubbard(16, 8, 8, w["bonds"], w["t"], w["U"], w["eps"])
    x0 = torch.from_numpy(W.normal(0, m.D)).cuda()
    m.ground(x0, maxit=3, tol=0.0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    r = m.ground(x0, maxit=steps, tol=0.0)
    e1.record()
    torch.cuda.synchronize()
    assert r["iters"] == steps
    m.close()
    return e0.elapsed_time(e1) / steps


def _child_batch(lib_path: str, steps: int) -> float:
    """ms for the AIM star batch (81 sectors x 64 parameter sets) with the library at lib_path."""
    import numpy as np
    import torch
    from paper_1307_7542_gb300 import hub, workloads as W
    hub.LIB_PATH = lib_path
    hub._lib = None
    ps = [W.aim_star(k) for k in range(64)]
    bonds = ps[0]["bonds"]
    t = np.stack([p["t"] for p in ps])
    U = np.stack([p["U"] for p in ps])
    eps = np.stack([p["eps"] for p in ps])
    jobs = [(a, b, p) for p in range(64) for a in range(9) for b in range(9)]
    jn, jd, jp = (np.array(c) for c in zip(*jobs))
    hub.hub_batch_ground(8, bonds, t, U, eps, jn[:81], jd[:81], jp[:81], maxit=400, tol=1e-12)
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(max(1, steps // 10)):
        t0 = time.perf_counter()
        hub.hub_batch_ground(8, bonds, t, U, eps, jn, jd, jp, maxit=400, tol=1e-12)
        best = min(best, 1000 * (time.perf_counter() - t0))
    return best


def measure(knobs: dict, what: str, steps: int) -> float:
    """Build the library with these knobs and time `what` ("apply" or "batch") in a child process."""
    from paper_1307_7542_gb300 import build
    os.makedirs(TUNE_DIR, exist_ok=True)
    lib_path = os.path.join(TUNE_DIR, f"lib_{_tag(knobs)}.so")
    if not os.path.exists(lib_path):
        build.build(out=lib_path, defines=[f"{k}={v}" for k, v in sorted(knobs.items())])
    cmd = [sys.executable, "-m", "paper_1307_7542_gb300.autotune", "--child", what, "--lib", lib_path,
           "--steps", str(steps)]
    r = subprocess.run(cmd, capture_output=True, text=True, cwd=ROOT)
    if r.returncode != 0:
        raise RuntimeError(f"measurement of {knobs} failed:\n{r.stdout}\n{r.stderr}")
    return float(json.loads(r.stdout.strip().splitlines()[-1])["ms"])


def coordinate_descent(space: dict, start: dict, what: str, steps: int, log: list) -> tuple:
    """One pass over the knobs of `space`: each alternative value is tried with the others
    fixed; a change is kept if it is at least MARGIN faster than the best so far."""
    best = dict(start)
    t_best = measure(best, what, steps)
    log.append({"what": what, "knobs": dict(best), "ms": t_best})
    seen = {_tag(best)}
    print(f"[{what}] start {best}: {t_best:.4f} ms", flush=True)
    for knob, values in space.items():
        for v in values:
            cand = dict(best, **{knob: v})
            if _tag(cand) in seen:
                continue
            seen.add(_tag(cand))
            t = measure(cand, what, steps)
            log.append({"what": what, "knobs": dict(cand), "ms": t})
            print(f"[{what}] {knob}={v}: {t:.4f} ms", flush=True)
            if t < t_best * (1.0 - MARGIN):
                best, t_best = cand, t
    return best, t_best


def main(argv=None) -> int:
    p = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    p.add_argument("--write", action="store_true", help="store the result in tuned.json")
    p.add_argument("--steps", type=int, default=20, help="Lanczos steps timed per candidate")
    p.add_argument("--child", choices=["apply", "batch"], help=argparse.SUPPRESS)
    p.add_argument("--lib", help=argparse.SUPPRESS)
    a = p.parse_args(argv)
    if a.child:
        fn = _child_apply if a.child == "apply" else _child_batch
        print(json.dumps({"ms": fn(a.lib, a.steps)}))
        return 0
    start = dict(DEFAULTS)
    if os.path.exists(TUNED):
        with open(TUNED) as f:
            start.update(json.load(f).get("defines", {}))
    log = []
    apply_start = {k: start[k] for k in APPLY_SPACE}
    best_apply, t_apply = coordinate_descent(APPLY_SPACE, apply_start, "apply", a.steps, log)
    batch_start = {k: start[k] for k in BATCH_SPACE}
    best_batch, t_batch = coordinate_descent(BATCH_SPACE, batch_start, "batch", a.steps, log)
    import torch
    result = {"gpu": torch.cuda.get_device_name(0), "defines": {**best_apply, **best_batch},
              "lanczos_step_ms_4x4": t_apply, "aim_batch_ms": t_batch, "trials": log}
    print(json.dumps({k: result[k] for k in ("gpu", "defines", "lanczos_step_ms_4x4", "aim_batch_ms")}))
    if a.write:
        with open(TUNED, "w") as f:
            json.dump(result, f, indent=1)
            f.write("\n")
    return 0


if __name__ == "__main__":
    sys.exit(main())
