"""Periodic Hubbard ring in a momentum sector (Sec. V) from the command line.

    python -m paper_1307_7542_gb300.ring --M 16 [--n-up 8 --n-dn 8] --sector kpi
           [--U 4] [--t 1] [--maxit 300] [--tol 1e-12] [--applies 0]

--sector k0 / kpi / full selects the k = 0 or k = pi subspace of the translation
i -> i-1 mod M, or the whole (N_up, N_dn) sector.  Prints one JSON line: the sector's
dimensions, and, with --maxit > 0, E0, the iterations and the wall time of the Lanczos run
to |dE0| < tol; with --applies N > 0 the mean CUDA-event time of N products on a projected
random vector.  All work runs in the library's kernels.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

SECTORS = {"full": 0, "k0": 1, "kpi": 2}


def ring_bonds(M: int) -> np.ndarray:
    return np.array([(i, (i + 1) % M) for i in range(M)], dtype=np.int32)


def run(M: int, n_up: int, n_dn: int, sector: str = "k0", U: float = 4.0, t: float = 1.0,
        maxit: int = 300, tol: float = 1e-12, applies: int = 0) -> dict:
    import torch
    from . import hub
    t0 = time.perf_counter()
    m = hub.Hubbard(M, n_up, n_dn, ring_bonds(M), t, U)
    out = {"M": M, "n_up": n_up, "n_dn": n_dn, "sector": sector, "U": U, "t": t}
    try:
        if sector != "full":
            m.set_symmetry(SECTORS[sector])
            out.update(rows=m.k_rows, cols=m.k_cols, dim=m.k_dim)
        else:
            out.update(dim=m.D)
        out["vector_len"] = m.D
        out["setup_s"] = time.perf_counter() - t0
        if applies > 0:
            g = torch.Generator(device="cuda")
            g.manual_seed(0)
            x = torch.randn(m.D, dtype=torch.float64, device="cuda", generator=g)
            if sector != "full":
                x = m.k_project(x)
            y = torch.empty_like(x)
            m.apply(x, y)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(applies):
                m.apply(x, y)
            e1.record()
            torch.cuda.synchronize()
            out["apply_ms"] = e0.elapsed_time(e1) / applies
            del x, y
        if maxit > 0:
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            r = m.ground(None, maxit=maxit, tol=tol)
            torch.cuda.synchronize()
            out.update(E0=r["E0"], iters=r["iters"], status=r["status"], lanczos_s=time.perf_counter() - t1)
    finally:
        m.close()
        torch.cuda.empty_cache()
    return out


def main(argv=None) -> int:
    p = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    p.add_argument("--M", type=int, required=True)
    p.add_argument("--n-up", type=int, default=None, help="default M // 2")
    p.add_argument("--n-dn", type=int, default=None, help="default M // 2")
    p.add_argument("--sector", choices=sorted(SECTORS), default="k0")
    p.add_argument("--U", type=float, default=4.0)
    p.add_argument("--t", type=float, default=1.0)
    p.add_argument("--maxit", type=int, default=300)
    p.add_argument("--tol", type=float, default=1e-12)
    p.add_argument("--applies", type=int, default=0)
    a = p.parse_args(argv)
    nu = a.M // 2 if a.n_up is None else a.n_up
    nd = a.M // 2 if a.n_dn is None else a.n_dn
    print(json.dumps(run(a.M, nu, nd, a.sector, a.U, a.t, a.maxit, a.tol, a.applies)))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
