#!/usr/bin/env python
"""Benchmark: H.x applies/s inside plain Lanczos on the 4x4 periodic Hubbard lattice.

Workload: 4x4 periodic square lattice, half filling (N_up = N_dn = 8), t = 1, U = 4,
D = 12870^2 = 165,636,900 (FP64 vectors of 1.33 GB, larger than L2), start vector
SplitMix64/Box-Muller normal with seed 0.  One step = one Lanczos iteration of the hot
path: the matrix-free apply w = H q plus the recurrence (two FP64 dot products, two
axpys, a normalisation and the alpha/beta read-back).  The spin bases and hopping
matrices are built once, before timing.

Prints ONE JSON line (rank 0).  --impl reference times the CPU oracle (two-spin basis,
binary search) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MEASURED = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
# FP64 issue rate of the GB300: the nominal 1.25 TFLOP/s dense FP64 counts an FMA as two
# flops, i.e. 152 SMs x 2 FP64 instructions/clock x 2.07 GHz = 0.629e12 instructions/s.
FP64_INSTR_PEAK = 152 * 2 * 2.07e9
SMEM_PEAK_TBS = 28.7          # shared-memory load bandwidth, conflict-free, all SMs (probe)
# FP32 pipe: 152 SMs x 128 lanes x 2.07 GHz (a packed f32x2 instruction occupies two lanes)
FP32_PEAK_TOPS = 152 * 128 * 2.07e9 / 1e12
FP32_OPS_PER_TERM = 14        # compensated double-float sum: TwoSum, TwoSum of its error, two adds
# DRAM bytes (read + write) per element of X from one ncu capture of each kernel on the 4x4
# (6,6) sector (profiles/k_up_4x4_sector66.md, profiles/k_dn_4x4_sector66.md); the
# per-element traffic does not depend on the sector, so a launch's traffic is this times D.
NCU_DRAM_BYTES_PER_ELEMENT = {"k_up": 0.98165581e9 / 64128064, "k_dn": 2.0847303e9 / 64128064}
STAGE_MAX_COLS = 14076        # rows up to this length are staged in shared memory by pass 1
# arithmetic of the timed fast path: vectors as pairs of FP32 numbers (48-bit significands),
# compensated sums; FP64 at the interface
DTYPE_FAST = "df32 (FP32 pairs, compensated sums; FP64 in/out)"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--U", type=float, default=4.0)
    p.add_argument("--e2e-steps", type=int, default=16)
    p.add_argument("--e2e-vectors", type=int, default=4)
    p.add_argument("--fp64-steps", type=int, default=10, help="Lanczos steps timed with HUB_MODE_FP64")
    p.add_argument("--lanczos-iters", type=int, default=200, help="iterations of the E0 wall-time run")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the batched, adjoint and 3x6 measurements reported beside the headline")
    p.add_argument("--workload", default="4x4", choices=sorted(WORKLOADS),
                   help="4x4: the benchmark case; the others are smaller cases for profiling")
    return p.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def peaks():
    try:
        with open(MEASURED) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        time.sleep(0.3)

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.15)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = max(float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit())
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, n in enumerate(names):
                if r[5 + k].strip().lower().startswith("active"):
                    reasons.add(n)
        sm_sorted = sorted(sm)
        med = sm_sorted[len(sm_sorted) // 2] if sm_sorted else None
        return {"sm_mhz": med, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(rows)}


def smi_index(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    ids = [v for v in vis.split(",") if v.strip()]
    if ids and ids[min(local_rank, len(ids) - 1)].strip().isdigit():
        return int(ids[min(local_rank, len(ids) - 1)])
    return local_rank


WORKLOADS = {
    "4x4": ("4x4 periodic square lattice, half filling (8,8), t=1", "4x4", 8, 8),
    "4x4-sector66": ("4x4 periodic square lattice, sector (6,6), t=1 (profiling case)", "4x4", 6, 6),
    # rows of C(18, 9) = 48620 spin-up states, too long to stage: pass 1 runs on the transposed
    # matrix (profiling case of the 3x6 (9,9) path at 1/60 of its size, vectors still > L2)
    "3x6-sector93": ("3x6 periodic square lattice, sector (9,3), t=1 (profiling case)", "3x6", 9, 3),
}


def workload(U, name="4x4"):
    from paper_1307_7542_gb300 import workloads as W
    label, lattice, nu, nd = WORKLOADS[name]
    w = W.square4x4(U) if lattice == "4x4" else W.square3x6(U)
    w["n_up"], w["n_dn"] = nu, nd
    w["label"] = label
    return w


def config_json(w, D, n_gpus):
    return {"workload": f"{w['label']}, U={w['U'][0]:g}",
            "M": w["M"], "n_up": w["n_up"], "n_dn": w["n_dn"], "dim": D,
            "step": "one Lanczos iteration (apply + recurrence)",
            "vector_bytes": 8 * D, "l2": f"inputs larger than L2 ({8 * D / 1e9:.2f} GB per FP64 vector); no flush needed",
            "parallelism": f"replicas x{n_gpus}" if n_gpus > 1 else "single GPU"}


# ----------------------------------------------------------------------------- CPU oracle

def oracle_sample(w, x, seconds, min_rows=20000):
    """Time the oracle's apply on the first R rows of the workload, R sized to take about
    `seconds`; returns (applies per second, rows, elapsed, threads)."""
    from oracle import hub_oracle as O
    om = O.Model(w["M"], w["bonds"], w["t"], w["U"], w["eps"])
    B = O.basis(w["M"], w["n_up"], w["n_dn"])
    D = B.shape[0]
    r = min_rows
    while True:                                   # grow the sample until it takes >= 1 s
        t0 = time.perf_counter()
        O.apply(om, B, x, rows=(0, r))
        dt = time.perf_counter() - t0
        if dt >= 1.0 or r >= D:
            break
        r = min(D, r * 4)
    R = int(min(D, max(r, r * seconds / max(dt, 1e-6))))
    t0 = time.perf_counter()
    O.apply(om, B, x, rows=(D // 3, min(D, D // 3 + R)))
    el = time.perf_counter() - t0
    return (R / D) / el, R, el, O.threads(), B, om


def run_reference(a):
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    import numpy as np
    from oracle import hub_oracle as O
    from paper_1307_7542_gb300 import workloads as W
    w = workload(a.U, a.workload)
    D = math.comb(16, w["n_up"]) * math.comb(16, w["n_dn"])
    x = W.normal(0, D)
    om = O.Model(w["M"], w["bonds"], w["t"], w["U"], w["eps"])
    B = O.basis(16, w["n_up"], w["n_dn"])
    # size one step (a bounded sample of rows) to about 2 s of CPU
    r = 20000
    while True:
        t0 = time.perf_counter()
        O.apply(om, B, x, rows=(0, r))
        dt = time.perf_counter() - t0
        if dt >= 0.5 or r >= D:
            break
        r = min(D, r * 4)
    # about 1 s per step, and at most ~150 s for the whole run however many steps are asked
    per_step = min(1.0, 150.0 / max(1, a.steps + a.warmup))
    R = int(min(D - 1, max(1000, r * per_step / max(dt, 1e-6))))
    for k in range(a.warmup):
        O.apply(om, B, x, rows=(0, R))
    t0 = time.perf_counter()
    for k in range(a.steps):
        r0 = (k * 7919 * R) % (D - R)
        O.apply(om, B, x, rows=(r0, r0 + R))
    el = time.perf_counter() - t0
    value = a.steps * (R / D) / el
    sample = f"{R} of {D} output rows per step ({R / D:.2e} of one apply), {O.threads()} threads"
    line = {"impl": "reference", "metric": "H.x applies/s (4x4 PBC half filling, U=4)",
            "value": value, "unit": "applies/s", "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1000 * el / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_json(w, D, 1),
            "cpu_baseline": {"value": value, "unit": "applies/s", "cores": O.threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "applies/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------------------- GPU arm

def combine_ranks(elapsed_ms, steps, world, device):
    """Whole-job timing over replicas: the slowest rank's time, and the steps all ranks did
    divided by it (each rank runs its own replica; no data-path collective)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(elapsed_ms)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    t_max = float(t.item())
    return t_max, world * steps / (t_max / 1000.0)


def extras(hub, W, torch):
    """Measurements beside the headline: batched vs one-at-a-time impurity solves, adjoint
    gradients vs finite differences, the 3x6 bandwidth-stress Lanczos step, the 4x4
    zero-temperature Green's function, the 8-site ring's E0 wall time, the momentum sectors
    of the 16- and 20-site rings and of the 4x4 torus."""
    import numpy as np
    out = {}
    # (1) AIM star M=8: 81 sectors x 64 parameter sets, one persistent launch
    ps = [W.aim_star(k) for k in range(64)]
    bonds = ps[0]["bonds"]
    t = np.stack([p["t"] for p in ps]); U = np.stack([p["U"] for p in ps]); eps = np.stack([p["eps"] for p in ps])
    jobs = [(a_, b_, p_) for p_ in range(64) for a_ in range(9) for b_ in range(9)]
    jn, jd, jp = (np.array(c) for c in zip(*jobs))
    hub.hub_batch_ground(8, bonds, t, U, eps, jn[:81], jd[:81], jp[:81], maxit=400, tol=1e-12)   # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    E0, it, st = hub.hub_batch_ground(8, bonds, t, U, eps, jn, jd, jp, maxit=400, tol=1e-12)
    t_batch = time.perf_counter() - t0
    # one at a time: the 81 sectors of parameter set 0 through hub_lanczos_ground
    t0 = time.perf_counter()
    maxdiff = 0.0
    for k in range(81):
        a_, b_, p_ = jobs[k]
        m = hub.Hubbard(8, a_, b_, bonds, t[p_], U[p_], eps[p_])
        r = m.ground(None, maxit=400, tol=1e-12)
        maxdiff = max(maxdiff, abs(r["E0"] - E0[k]) / max(1.0, abs(E0[k])))
        m.close()
    t_one = (time.perf_counter() - t0) / 81
    out["batched"] = {"workload": "AIM star M=8 (impurity + 7 bath sites), 81 sectors x 64 parameter sets",
                      "jobs": len(jobs), "batched_s": t_batch, "jobs_per_s": len(jobs) / t_batch,
                      "one_at_a_time_s_per_job": t_one, "one_at_a_time_total_s_extrapolated": t_one * len(jobs),
                      "speedup": t_one * len(jobs) / t_batch, "max_rel_dE0_vs_one_at_a_time": maxdiff,
                      "iterations_mean": float(np.mean(it)), "all_converged": bool(np.all(np.isin(st, [0, 1])))}
    # (2) disordered 3x4 open lattice: adjoint (one solve + hub_grad) vs central differences
    w = W.disordered3x4()
    m = hub.Hubbard(12, 6, 6, w["bonds"], w["t"], w["U"], w["eps"])
    x0 = torch.from_numpy(W.normal(0, m.D)).cuda()
    m.ground(x0, maxit=400, tol=1e-12)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = m.ground(x0, maxit=400, tol=1e-12, want_psi=True)
    dt, dU, de = m.grad(r["psi"])
    t_adj = time.perf_counter() - t0
    n_par = len(w["t"]) + 24
    h = 1e-4
    fd_err = 0.0
    t0 = time.perf_counter()
    sample = [0, 5, 11, 16]
    for k in sample:
        tp, tm = w["t"].copy(), w["t"].copy()
        tp[k] += h
        tm[k] -= h
        m.set_params(tp, w["U"], w["eps"]); Ep = m.ground(x0, maxit=400, tol=1e-12)["E0"]
        m.set_params(tm, w["U"], w["eps"]); Em = m.ground(x0, maxit=400, tol=1e-12)["E0"]
        fd_err = max(fd_err, abs((Ep - Em) / (2 * h) - dt[k]))
    t_fd_solve = (time.perf_counter() - t0) / (2 * len(sample))
    m.close()
    out["adjoint"] = {"workload": "3x4 open lattice (6,6), D=853776, 41 parameters (17 t_b, 12 U_i, 12 eps_i)",
                      "adjoint_s": t_adj, "fd_s_per_solve": t_fd_solve, "fd_total_s_extrapolated": t_fd_solve * 2 * n_par,
                      "speedup": t_fd_solve * 2 * n_par / t_adj, "max_abs_diff_vs_fd_h1e-4": fd_err,
                      "fd_params_timed": len(sample)}
    # (3) 3x6 periodic lattice, (9,9): D = 2,363,904,400 (18.9 GB per FP64 vector)
    w = W.square3x6(4.0)
    m = hub.Hubbard(18, 9, 9, w["bonds"], w["t"], w["U"], w["eps"])
    m.ground(None, maxit=2, tol=0.0)
    hub.hub_profile(m.h, True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = m.ground(None, maxit=4, tol=0.0)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    up_ms, n_up_l, _ = hub.hub_profile_read(m.h, hub.HUB_PROF_UP)
    dn_ms, n_dn_l, _ = hub.hub_profile_read(m.h, hub.HUB_PROF_DN)
    ap_ms, n_ap, _ = hub.hub_profile_read(m.h, hub.HUB_PROF_APPLY)
    D = m.D
    m.close()
    torch.cuda.empty_cache()
    out["square3x6"] = {"workload": "3x6 PBC (9,9), t=1, U=4", "dim": D, "lanczos_step_ms": 1000 * el / 4,
                        "apply_ms": ap_ms / max(n_ap, 1), "k_up_ms": up_ms / max(n_up_l, 1),
                        "k_dn_ms": dn_ms / max(n_dn_l, 1),
                        "apply_gbs_16B_per_element": 16 * D / (ap_ms / max(n_ap, 1) / 1000) / 1e9}
    # (4) zero-temperature Green's function (Sec. VII) at 4x4 PBC, half filling, site 0, spin up:
    # ground state of (8,8), c+ psi0 into (9,8) and c psi0 into (7,8), 100 continued-fraction
    # steps for each term, G on 400 frequencies
    w = W.square4x4(4.0)
    m0 = hub.Hubbard(16, 8, 8, w["bonds"], w["t"], w["U"], w["eps"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r0 = m0.ground(None, maxit=400, tol=1e-10, want_psi=True)
    torch.cuda.synchronize()
    t_gs = time.perf_counter() - t0
    omega = np.linspace(-12.0, 12.0, 400) + 0.1j
    G = np.zeros(omega.shape, dtype=np.complex128)
    stages, norms, k_steps = {}, [], 100
    for create, sign, nu in ((True, 1, 9), (False, -1, 7)):
        m1 = hub.Hubbard(16, nu, 8, w["bonds"], w["t"], w["U"], w["eps"])
        v = torch.empty(m1.D, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hub.hub_ladder(m0.h, m1.h, 0, 0, create, r0["psi"], v)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        a_, b_, n2 = hub.hub_green_coeffs(m1.h, v, k_steps)
        t2 = time.perf_counter()
        G += hub.hub_green_eval(a_, b_, n2, r0["E0"], sign, omega)
        t3 = time.perf_counter()
        norms.append(n2)
        key = "particle" if create else "hole"
        stages[key] = {"sector": [nu, 8], "dim": m1.D, "ladder_ms": 1000 * (t1 - t0),
                       "coeffs_s": t2 - t1, "steps": len(a_), "ms_per_step": 1000 * (t2 - t1) / max(len(a_), 1),
                       "eval_ms": 1000 * (t3 - t2)}
        m1.close()
        del v
    m0.close()
    torch.cuda.empty_cache()
    out["green_4x4"] = {"workload": "4x4 PBC (8,8), U=4: G_up(site 0, omega + 0.1i), 400 frequencies",
                        "ground_state_s": t_gs, "ground_state_iters": r0["iters"], "E0": r0["E0"],
                        "terms": stages, "sum_rule_norm2_total": sum(norms),
                        "total_s": t_gs + sum(v_["coeffs_s"] + v_["ladder_ms"] / 1000 for v_ in stages.values())}
    # (5) momentum sectors of the Hubbard ring (Sec. V), half filling, U = 4: at M = 16 the
    # full sector against its k = pi subspace, where the ground state lies, each to
    # |dE0| < 1e-12; at M = 20 the k = pi ground state and products (the full sector would
    # need 273 GB per vector).  Terms per element: the hops of both spins,
    # 2 * (2 M C(M-2, N-1) / C(M, N)), plus the diagonal.
    from paper_1307_7542_gb300 import ring as R
    full16 = R.run(16, 8, 8, "full", maxit=400, tol=1e-12, applies=5)
    kpi16 = R.run(16, 8, 8, "kpi", maxit=400, tol=1e-12, applies=20)
    kpi20 = R.run(20, 10, 10, "kpi", maxit=300, tol=1e-12, applies=3)
    for r in (kpi16, kpi20):
        M, N = r["M"], r["n_up"]
        terms = 2 * (2 * M * math.comb(M - 2, N - 1) / math.comb(M, N)) + 1
        r["terms_per_element"] = terms
        r["terms_per_s"] = terms * r["vector_len"] / (r["apply_ms"] / 1000)
        r["as_fp64_fma_frac_of_fp64_issue"] = r["terms_per_s"] / FP64_INSTR_PEAK
    # (6) the 8-site ring at half filling (D = 4900), E0 to |dE0| < 1e-12 from a seed-0 normal
    # start vector: latency-bound; through hub_lanczos_ground (the single-launch small-sector
    # solver: one thread-block-cluster launch per batch of eight iterations at this size; and,
    # with it turned off, the multi-kernel driver with its per-iteration launches and
    # read-backs) and as a single job of the persistent batched solver (one launch; it draws
    # its own start vector)
    bonds8 = np.array([(i, (i + 1) % 8) for i in range(8)], dtype=np.int32)
    m8 = hub.Hubbard(8, 4, 4, bonds8, 1.0, 4.0)
    x8 = torch.from_numpy(W.normal(0, m8.D)).cuda()

    def time_ground(reps=5):
        m8.ground(x8, maxit=300, tol=1e-12)
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r_ = m8.ground(x8, maxit=300, tol=1e-12)
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        return r_, ts
    r8, reps8 = time_ground()
    hub.hub_set_small_dim(m8.h, 0)
    r8m, reps8m = time_ground()
    m8.close()
    one = lambda a: np.asarray(a, dtype=np.float64).reshape(1, -1)
    hub.hub_batch_ground(8, bonds8, one(np.ones(8)), one(np.full(8, 4.0)), one(np.zeros(8)),
                         np.array([4]), np.array([4]), np.array([0]), maxit=300, tol=1e-12)
    reps_b = []
    for _ in range(5):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Eb, itb, _ = hub.hub_batch_ground(8, bonds8, one(np.ones(8)), one(np.full(8, 4.0)), one(np.zeros(8)),
                                          np.array([4]), np.array([4]), np.array([0]), maxit=300, tol=1e-12)
        reps_b.append(time.perf_counter() - t0)
    out["ring8"] = {"workload": "ring M=8, (4,4), D=4900, t=1, U=4, to |dE0| < 1e-12",
                    "E0": r8["E0"], "iterations": r8["iters"], "lanczos_ground_ms": 1000 * min(reps8),
                    "lanczos_ground_path": "single-launch small-sector solver (FP64, one 16-CTA cluster launch per 8 iterations)",
                    "multi_kernel_driver_E0": r8m["E0"], "multi_kernel_driver_iterations": r8m["iters"],
                    "multi_kernel_driver_ms": 1000 * min(reps8m),
                    "batched_single_job_E0": float(Eb[0]), "batched_single_job_iterations": int(itb[0]),
                    "batched_single_job_ms": 1000 * min(reps_b)}
    # (7b) block Lanczos at 4x4 (8,8): a block step applies H to k vectors with the same product
    # kernels (k products, FP64 in and out) plus the FP64 block Gram/QR work and the full
    # re-orthogonalisation; timed against k single Lanczos steps of hub_lanczos_ground on the
    # same handle, with the products inside the block step timed separately
    w = W.square4x4(4.0)
    mb = hub.Hubbard(16, 8, 8, w["bonds"], w["t"], w["U"], w["eps"])
    x0b = torch.from_numpy(W.normal(0, mb.D)).cuda()
    mb.ground(x0b, maxit=3, tol=0.0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mb.ground(x0b, maxit=6, tol=0.0)
    torch.cuda.synchronize()
    single_ms = 1000 * (time.perf_counter() - t0) / 6
    del x0b
    blk = {"workload": "4x4 PBC (8,8), U=4", "single_step_ms": single_ms}
    # one product alone (FP64 in and out, as the block solver calls it)
    xa = torch.from_numpy(W.normal(1, mb.D)).cuda()
    ya = torch.empty_like(xa)
    hub.hub_apply(mb.h, xa, ya)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(4):
        hub.hub_apply(mb.h, xa, ya)
    torch.cuda.synchronize()
    apply_ms = 1000 * (time.perf_counter() - t0) / 4
    del xa, ya
    blk["single_product_ms"] = apply_ms
    for kb in (2, 4):
        hub.hub_profile(mb.h, True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        evb, rsb = hub.hub_lanczos_block(mb.h, kb, None, 3, kb)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        pa_ms, pa_n, _ = hub.hub_profile_read(mb.h, hub.HUB_PROF_APPLY)
        hub.hub_profile(mb.h, False)
        blk[f"k={kb}"] = {"steps": 3, "ms_per_block_step": 1000 * el / 3,
                          "products_per_block_step": pa_n / 3, "product_ms_in_block": pa_ms / max(pa_n, 1),
                          "products_ms_per_block_step": pa_ms / 3,
                          "block_work_ms_per_block_step": 1000 * el / 3 - pa_ms / 3,
                          "vs_k_single_steps": (1000 * el / 3) / (kb * single_ms)}
    mb.close()
    torch.cuda.empty_cache()
    out["block_lanczos_4x4"] = blk
    # (7) the 4x4 torus (the benchmark lattice) in its four real-momentum sectors of the two
    # translations, U = 4, each to |dE0| < 1e-12; the lowest is the full sector's ground state
    tor = {}
    for kx, ky in (("0", "0"), ("pi", "0"), ("0", "pi"), ("pi", "pi")):
        tor[f"k=({kx},{ky})"] = R.run(16, 8, 8, "k", maxit=400, tol=1e-12, applies=10, torus=(4, 4), k=(kx, ky))
    low = min(tor.values(), key=lambda r: r["E0"])
    out["torus_4x4_momentum"] = {"workload": "4x4 PBC (8,8), t=1, U=4: sectors of the two translations",
                                 "sectors": tor, "lowest_sector": [k_ for k_, v_ in tor.items() if v_ is low][0],
                                 "lowest_E0": low["E0"],
                                 "all_sectors_lanczos_s": sum(v_["lanczos_s"] for v_ in tor.values())}
    out["ring_momentum"] = {"workload": "Hubbard ring, half filling, t=1, U=4; k = pi subspace of the "
                                        "translation (T eigenvalue -1) against the full sector",
                            "M16_full": full16, "M16_kpi": kpi16, "M20_kpi": kpi20,
                            "M16_E0_diff": abs(kpi16["E0"] - full16["E0"]),
                            "M16_speedup_time_to_tol": full16["lanczos_s"] / kpi16["lanczos_s"]}
    return out


def run_gpu(a):
    import numpy as np
    import torch
    import torch.distributed as dist

    rank, local, world = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    from paper_1307_7542_gb300 import hub
    from paper_1307_7542_gb300 import workloads as W

    w = workload(a.U, a.workload)
    t_setup = time.perf_counter()
    m = hub.Hubbard(w["M"], w["n_up"], w["n_dn"], w["bonds"], w["t"], w["U"], w["eps"])
    setup_s = time.perf_counter() - t_setup
    D = m.D
    x_host = W.normal(0, D)
    x0 = torch.from_numpy(x_host).cuda()
    stream = torch.cuda.current_stream()

    # warm-up steps
    m.ground(x0, maxit=max(a.warmup, 1), tol=0.0)
    torch.cuda.synchronize()

    clocks = Clocks(smi_index(local)) if rank == 0 else None
    if clocks:
        clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    hub.hub_profile(m.h, True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    r = m.ground(x0, maxit=a.steps, tol=0.0)
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    elapsed_ms = e0.elapsed_time(e1)
    apply_ms, n_apply, n_kern = hub.hub_profile_read(m.h, hub.HUB_PROF_APPLY)
    up_ms, n_up_l, _ = hub.hub_profile_read(m.h, hub.HUB_PROF_UP)
    dn_ms, n_dn_l, _ = hub.hub_profile_read(m.h, hub.HUB_PROF_DN)
    ud_ms, n_ud_l, _ = hub.hub_profile_read(m.h, hub.HUB_PROF_UPDATE)
    hub.hub_profile(m.h, False)
    clk = clocks.stop() if clocks else None
    assert r["iters"] == a.steps, r

    elapsed_ms, value = combine_ranks(elapsed_ms, a.steps, world, "cuda")

    # roofline of the product and of its dominant kernel
    apply_avg_ms = apply_ms / max(n_apply, 1)
    nnz_u, _ = hub.hub_csr_info(m.h, 0)
    nnz_d, _ = hub.hub_csr_info(m.h, 1)
    nnz_H = nnz_u * m.count_dn + nnz_d * m.count_up + D           # Sec. IV.A nnz formula
    hbm_gbs, peak_kind = peaks()
    peak_src = ("measured: MEASURED_PEAKS.json hbm_gbs" if peak_kind == "measured" else "fallback 6.8 TB/s")

    def gb(bytes_, ms):
        return bytes_ / (ms / 1000.0) / 1e9 if ms > 0 else 0.0

    apply = {"ms": apply_avg_ms, "launches": n_apply, "algorithmic_bytes": 16 * D,
             "gbs": gb(16 * D, apply_avg_ms), "hbm_frac": gb(16 * D, apply_avg_ms) / hbm_gbs,
             "fp64_equiv_rate_T": nnz_H / (apply_avg_ms / 1000.0) / 1e12,
             "fp64_alu_frac": nnz_H / (apply_avg_ms / 1000.0) / FP64_INSTR_PEAK}
    if n_up_l and n_dn_l:
        # fast path, each pass timed by its own event pair.  HBM bytes per element (double-float
        # vectors, 8 B): pass 1 reads X and writes Z (16 B); pass 2 (Lanczos epilogue) reads X by
        # strips, Z, r_j, r_{j-1} and writes w (40 B); the update reads w and r_{j-1} and writes
        # r_j (24 B).  FP32 pipe: each hopping term costs 14 FP32 operations in the compensated
        # double-float sum (both passes).
        up_avg, dn_avg = up_ms / n_up_l, dn_ms / n_dn_l
        terms = {"k_up": nnz_u * m.count_dn, "k_dn": nnz_d * m.count_up}
        passes = {"k_up": {"ms": up_avg, "algorithmic_bytes": 16 * D, "gbs": gb(16 * D, up_avg)},
                  "k_dn": {"ms": dn_avg, "algorithmic_bytes": 40 * D, "gbs": gb(40 * D, dn_avg)}}
        update = None
        if n_ud_l:
            ud_avg = ud_ms / n_ud_l
            update = {"kernel": "k_df_update", "ms": ud_avg, "launches": n_ud_l, "algorithmic_bytes": 24 * D,
                      "gbs": gb(24 * D, ud_avg), "hbm_frac": gb(24 * D, ud_avg) / hbm_gbs}
        for k_, v_ in passes.items():
            ops = FP32_OPS_PER_TERM * terms[k_]
            v_["hbm_frac"] = v_["gbs"] / hbm_gbs
            v_["fp32_ops"] = ops
            v_["fp32_tops"] = ops / (v_["ms"] / 1000.0) / 1e12
            v_["fp32_frac"] = v_["fp32_tops"] / FP32_PEAK_TOPS
        if m.count_up <= STAGE_MAX_COLS:
            # pass 1 gathers from shared memory: 8 B (high and low word) per spin-up hop and
            # for the diagonal's own element, per element of X
            smem_bytes = 8 * (nnz_u + m.count_up) * m.count_dn
            passes["k_up"]["shared_memory"] = {
                "algorithmic_bytes": smem_bytes, "tbs": gb(smem_bytes, up_avg) / 1000.0,
                "peak_tbs": SMEM_PEAK_TBS, "frac": gb(smem_bytes, up_avg) / 1000.0 / SMEM_PEAK_TBS,
                "peak_source": "probe: conflict-free 64-bit shared loads, all SMs (GB300)"}
        dom = max(passes, key=lambda k: passes[k]["ms"])
        staged_4x4 = a.workload.startswith("4x4") and m.count_up <= STAGE_MAX_COLS
        traffic = NCU_DRAM_BYTES_PER_ELEMENT[dom] * D if staged_4x4 and dom in NCU_DRAM_BYTES_PER_ELEMENT else None
        pd = passes[dom]
        if pd["fp32_frac"] >= pd["hbm_frac"]:
            roofline = {"bound": "alu", "kernel": dom, "achieved": pd["fp32_tops"], "peak": FP32_PEAK_TOPS,
                        "unit": "T FP32 op/s", "frac": pd["fp32_frac"],
                        "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2.07 GHz",
                        "hbm": {"achieved": pd["gbs"], "peak": hbm_gbs, "unit": "GB/s", "frac": pd["hbm_frac"],
                                "peak_source": peak_src}}
        else:
            roofline = {"bound": "hbm", "kernel": dom, "achieved": pd["gbs"], "peak": hbm_gbs, "unit": "GB/s",
                        "frac": pd["hbm_frac"], "peak_source": peak_src}
        roofline.update({"traffic": traffic,
                         "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum of the same kernel "
                                            "on the 4x4 (6,6) sector, scaled by elements" if traffic else None),
                         "passes": passes, "update": update, "apply": apply})
    else:
        # native FP64 kernel: bound by the FP64 pipe
        roofline = {"bound": "alu", "kernel": "k_apply_f64", "achieved": apply["fp64_equiv_rate_T"],
                    "peak": FP64_INSTR_PEAK / 1e12, "unit": "T FP64 instr/s",
                    "frac": apply["fp64_alu_frac"], "traffic": None,
                    "peak_source": "derived: 152 SMs x 2 FP64 instr/clk x 2.07 GHz (nominal 1.25 TFLOP/s)",
                    "apply": apply}

    # Lanczos E0 wall time: a full run of a.lanczos_iters iterations, energy only
    lanczos = None
    if a.lanczos_iters > 0:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rl = m.ground(x0, maxit=a.lanczos_iters, tol=0.0)
        torch.cuda.synchronize()
        lanczos = {"E0": rl["E0"], "iterations": rl["iters"], "wall_s": time.perf_counter() - t0}
        # time to |E0_j - E0_{j-1}| < 1e-12 for the three interaction strengths of the 4x4
        # configuration (same lattice and start vector)
        if a.workload == "4x4" and rank == 0:
            conv = {}
            for Uc in (2.0, 4.0, 8.0):
                wc = workload(Uc, a.workload)
                mc = hub.Hubbard(wc["M"], wc["n_up"], wc["n_dn"], wc["bonds"], wc["t"], wc["U"], wc["eps"])
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                rc_ = mc.ground(x0, maxit=1000, tol=1e-12)
                torch.cuda.synchronize()
                conv[f"U={Uc:g}"] = {"E0": rc_["E0"], "iterations": rc_["iters"],
                                     "wall_s": time.perf_counter() - t0, "converged": rc_["status"] == 0}
                mc.close()
            lanczos["to_tol_1e-12"] = conv

    # the same step with the native FP64 kernels (HUB_MODE_FP64): the path whose arithmetic is
    # FP64 throughout, bound by the FP64 pipe
    fp64_mode = None
    if a.fp64_steps > 0:
        hub.hub_set_mode(m.h, hub.HUB_MODE_FP64)
        m.ground(x0, maxit=2, tol=0.0)
        hub.hub_profile(m.h, True)
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        rf = m.ground(x0, maxit=a.fp64_steps, tol=0.0)
        f1.record(stream)
        torch.cuda.synchronize()
        f_ms = f0.elapsed_time(f1) / a.fp64_steps
        fa_ms, fa_n, _ = hub.hub_profile_read(m.h, hub.HUB_PROF_APPLY)
        hub.hub_profile(m.h, False)
        hub.hub_set_mode(m.h, hub.HUB_MODE_AUTO)
        fa = fa_ms / max(fa_n, 1)
        fp64_mode = {"dtype": "f64", "kernel": "k_apply_f64", "steps": a.fp64_steps, "ms_per_step": f_ms,
                     "applies_per_s": 1000.0 / f_ms, "apply_ms": fa,
                     "apply_hbm_frac_16B_per_element": gb(16 * D, fa) / hbm_gbs,
                     "fp64_instr_per_s_T": nnz_H / (fa / 1000.0) / 1e12,
                     "fp64_pipe_frac": nnz_H / (fa / 1000.0) / FP64_INSTR_PEAK,
                     "fp64_peak_source": "derived: 152 SMs x 2 FP64 instr/clk x 2.07 GHz (nominal 1.25 TFLOP/s)",
                     "E0_after_steps": rf["E0"]}

    # end-to-end through the C ABI with host buffers, host<->device copies inside the timed
    # region: hub_apply_host_many (several vectors per call, one vector's copies overlapping its
    # neighbours') gives `value`; the one-vector blocking call hub_apply_host is reported beside it
    e2e = None
    if a.e2e_steps > 0:
        def timed_calls(fn, n_calls, n_warm):
            """Host wall time and stream time (events recorded on the call's stream just before
            and after it: the copies and passes the call enqueues, as the GPU ran them) per call."""
            warm = []
            for _ in range(n_warm):
                t0 = time.perf_counter()
                fn()
                warm.append(time.perf_counter() - t0)
            torch.cuda.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(n_calls)]
            calls = []
            for k in range(n_calls):
                t0 = time.perf_counter()
                ev[k][0].record(stream)
                fn()
                ev[k][1].record(stream)
                calls.append(time.perf_counter() - t0)
            torch.cuda.synchronize()
            return calls, [e0_.elapsed_time(e1_) for e0_, e1_ in ev], warm

        def spread(calls):
            return [1000 * min(calls), 1000 * sorted(calls)[len(calls) // 2], 1000 * max(calls)]

        xh = torch.from_numpy(x_host).pin_memory()
        yh = torch.empty(D, dtype=torch.float64).pin_memory()
        calls, dev_calls, warm = timed_calls(lambda: hub.hub_apply_host(m.h, xh, yh), a.e2e_steps, 3)
        single_s = sum(calls)
        # what the call is made of: one copy each way alone, and the device product alone
        xd_ = torch.empty(D, dtype=torch.float64, device="cuda")
        yd_ = torch.empty(D, dtype=torch.float64, device="cuda")
        c0, c1, c2, c3 = (torch.cuda.Event(enable_timing=True) for _ in range(4))
        xd_.copy_(xh, non_blocking=True)
        torch.cuda.synchronize()
        c0.record(stream)
        xd_.copy_(xh, non_blocking=True)
        c1.record(stream)
        yh.copy_(yd_, non_blocking=True)
        c2.record(stream)
        hub.hub_apply(m.h, xd_, yd_)
        c3.record(stream)
        torch.cuda.synchronize()
        h2d_ms, d2h_ms, dev_ms = c0.elapsed_time(c1), c1.elapsed_time(c2), c2.elapsed_time(c3)
        single_ms = 1000 * single_s / a.e2e_steps
        single = {"value": world * a.e2e_steps / single_s, "unit": "applies/s",
                  "call": "hub_apply_host (one vector per call)", "ms_per_call": single_ms,
                  "h2d_gbs": gb(8 * D, h2d_ms), "d2h_gbs": gb(8 * D, d2h_ms), "hub_apply_device_ms": dev_ms,
                  "serial_ms": h2d_ms + dev_ms + d2h_ms,
                  "overlap_saved_ms": h2d_ms + dev_ms + d2h_ms - single_ms,
                  "call_ms_min_median_max": spread(calls), "call_ms": [1000 * c for c in calls],
                  "call_stream_ms": dev_calls, "warmup_call_ms": [1000 * c for c in warm]}
        del xh, yh, xd_, yd_
        # several vectors per call (the same input vector repeated: the contents do not change
        # the work)
        nv = max(1, a.e2e_vectors)
        n_calls = max(1, a.e2e_steps // nv)
        xs = torch.from_numpy(np.tile(x_host, nv)).pin_memory()
        ys = torch.empty(nv * D, dtype=torch.float64).pin_memory()
        calls, dev_calls, warm = timed_calls(lambda: hub.hub_apply_host_many(m.h, nv, xs, ys), n_calls, 1)
        e2e_s = sum(calls)
        e2e = {"value": world * nv * n_calls / e2e_s, "unit": "applies/s",
               "h2d_bytes_per_step": 8 * D, "d2h_bytes_per_step": 8 * D,
               "call": f"hub_apply_host_many ({nv} vectors per call, pinned host x in, host y out)",
               "vectors_per_call": nv, "calls": n_calls, "ms_per_apply": 1000 * e2e_s / (nv * n_calls),
               "call_ms_min_median_max": spread(calls), "call_ms": [1000 * c for c in calls],
               "call_stream_ms": dev_calls, "warmup_call_ms": [1000 * c for c in warm],
               "single_call": single}
        del xs, ys

    metric = ("H.x applies/s (4x4 PBC half filling, U=4)" if a.workload == "4x4"
              else f"H.x applies/s ({w['label']}, U={w['U'][0]:g})")
    line = {"metric": metric,
            "value": value, "unit": "applies/s", "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": elapsed_ms / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE_FAST if n_up_l else "f64", "data": "synthetic",
            "config": config_json(w, D, world), "roofline": roofline, "fp64_mode": fp64_mode,
            "lanczos_e0": lanczos, "setup_s": setup_s, "e2e": e2e, "gpu_launches": n_kern, "clocks": clk}

    if rank == 0 and world == 1 and not a.no_cpu_baseline and a.e2e_steps >= 0:
        aps, R, el, thr, _, _ = oracle_sample(w, x_host, a.cpu_seconds)
        line["cpu_baseline"] = {"value": aps, "unit": "applies/s", "cores": thr, "kind": "oracle",
                                "sample": f"oracle apply of {R} of {D} output rows ({el:.1f} s), scaled to "
                                          f"whole applies"}
    m.close()
    if world == 1 and not a.no_extras:
        torch.cuda.empty_cache()
        line["extras"] = extras(hub, W, torch)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    a = parse()
    if a.impl == "reference":
        return run_reference(a)
    return run_gpu(a)


if __name__ == "__main__":
    sys.exit(main())
