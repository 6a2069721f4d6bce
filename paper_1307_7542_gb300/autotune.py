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
* ``HUB_UP_PAIRED``    -- 1: pass 1 adds the low parts of a column word's two entries together
  before accumulating them (two accumulators, as pass 2); 0: four accumulators of single terms;
* ``HUB_BATCH_THREADS`` -- threads per CTA of the batched persistent solver;
* ``HUB_BATCH_SPLIT``  -- jobs of at most this many states run in a second launch of the batched
  solver, its shared memory sized for them (0: one launch);
* ``HUB_SMALL_CLUSTER_MAX``, ``HUB_SMALL_THREADS``, ``HUB_SMALL_PER_THREAD``,
  ``HUB_SMALL_BATCH`` -- the largest sector the single-launch small-sector Lanczos
  (csrc/hub_small.cu) runs as one thread-block cluster (0: always the cooperative grid), its
  threads per CTA, states per thread the grid is sized for, and iterations per launch.

For each candidate setting this module builds one copy of the library, times on the GPU what
the knob affects (one Lanczos step at 4x4 half filling for the apply knobs; the 5184-job
impurity batch of 81 sectors x 64 parameter sets for the batched knob; the 8-site ring's ground
state to |dE0| < 1e-12 for the small-sector knobs), each in a fresh process, and keeps the
fastest by coordinate descent from the current setting (a change is kept only if it is at least
1 % faster).  ``--only`` tunes some of the three groups and keeps the others' stored values;
``--write`` stores the result in tuned.json, which ``build()`` compiles in.

    python -m paper_1307_7542_gb300.autotune [--write] [--steps 20] [--only apply,batch,small]
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
    "HUB_BANK_CAP": [2, 1, 3, 0, -2],
    "HUB_FUSED_UPDATE": [1, 0],
    "HUB_UPD_Q": [1, 2],
    "HUB_UP_THREADS": [1024, 768, 512],
    "HUB_UP_PAIRED": [1, 0],
}
BATCH_SPACE = {"HUB_BATCH_THREADS": [256, 512, 1024], "HUB_BATCH_SPLIT": [2048, 1024, 4096, 0]}
SMALL_SPACE = {"HUB_SMALL_CLUSTER_MAX": [8192, 12800, 0], "HUB_SMALL_THREADS": [128, 256, 320, 384, 512],
               "HUB_SMALL_PER_THREAD": [1, 2, 4], "HUB_SMALL_BATCH": [8, 4, 16]}
DEFAULTS = {"HUB_DN_LANE_COLS": 4, "HUB_DN_BATCH": 2, "HUB_DN_MINB": 4, "HUB_BANK_CAP": 2,
            "HUB_FUSED_UPDATE": 0, "HUB_UPD_Q": 1, "HUB_UP_THREADS": 1024, "HUB_UP_PAIRED": 1,
            "HUB_BATCH_THREADS": 256, "HUB_BATCH_SPLIT": 2048,
            "HUB_SMALL_CLUSTER_MAX": 8192, "HUB_SMALL_THREADS": 320, "HUB_SMALL_PER_THREAD": 1,
            "HUB_SMALL_BATCH": 8}
# tuned.json key of each group's timing
RESULT_KEYS = {"apply": "lanczos_step_ms_4x4", "batch": "aim_batch_ms", "small": "ring8_ground_ms"}
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


def _child_small(lib_path: str, steps: int) -> float:
    """ms for the 8-site ring's ground state (D = 4900) to |dE0| < 1e-12 from the seed-0 normal
    vector (best of `steps` // 2 runs), with the library at lib_path."""
    import torch
    from paper_1307_7542_gb300 import hub, workloads as W
    hub.LIB_PATH = lib_path
    hub._lib = None
    m = hub.Hubbard(8, 4, 4, W.ring_bonds(8), 1.0, 4.0)
    x0 = torch.from_numpy(W.normal(0, m.D)).cuda()
    m.ground(x0, maxit=300, tol=1e-12)
    best = float("inf")
    for _ in range(max(3, steps // 2)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m.ground(x0, maxit=300, tol=1e-12)
        torch.cuda.synchronize()
        best = min(best, 1000 * (time.perf_counter() - t0))
    m.close()
    return best


CHILDREN = {"apply": _child_apply, "batch": _child_batch, "small": _child_small}
SPACES = {"apply": APPLY_SPACE, "batch": BATCH_SPACE, "small": SMALL_SPACE}


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


def _gpu_name() -> str:
    try:
        import torch
        return torch.cuda.get_device_name(0)
    except Exception:
        return "unknown"


def main(argv=None) -> int:
    p = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    p.add_argument("--write", action="store_true", help="store the result in tuned.json")
    p.add_argument("--steps", type=int, default=20, help="Lanczos steps timed per candidate")
    p.add_argument("--only", default="apply,batch,small", help="groups to tune (comma-separated)")
    p.add_argument("--child", choices=sorted(CHILDREN), help=argparse.SUPPRESS)
    p.add_argument("--lib", help=argparse.SUPPRESS)
    a = p.parse_args(argv)
    if a.child:
        print(json.dumps({"ms": CHILDREN[a.child](a.lib, a.steps)}))
        return 0
    groups = [g for g in a.only.split(",") if g]
    if any(g not in SPACES for g in groups):
        p.error(f"--only takes groups from {sorted(SPACES)}")
    start = dict(DEFAULTS)
    stored = {}
    if os.path.exists(TUNED):
        with open(TUNED) as f:
            stored = json.load(f)
        start.update(stored.get("defines", {}))
    log = []
    defines = dict(start)
    timings = {RESULT_KEYS[g]: stored[RESULT_KEYS[g]] for g in SPACES if g not in groups and RESULT_KEYS[g] in stored}
    for g in groups:
        best, t = coordinate_descent(SPACES[g], {k: start[k] for k in SPACES[g]}, g, a.steps, log)
        defines.update(best)
        timings[RESULT_KEYS[g]] = t
    result = {"gpu": _gpu_name(), "defines": defines, **timings,
              "trials": [t for t in stored.get("trials", []) if t.get("what") not in groups] + log}
    print(json.dumps({k: v for k, v in result.items() if k != "trials"}))
    if a.write:
        with open(TUNED, "w") as f:
            json.dump(result, f, indent=1)
            f.write("\n")
    return 0


if __name__ == "__main__":
    sys.exit(main())
