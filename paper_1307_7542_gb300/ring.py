"""Periodic Hubbard ring or torus in a momentum sector (Sec. V) from the command line.

    python -m paper_1307_7542_gb300.ring --M 16 [--n-up 8 --n-dn 8] --sector kpi
           [--U 4] [--t 1] [--maxit 300] [--tol 1e-12] [--applies 0]
    python -m paper_1307_7542_gb300.ring --torus 4x4 --k pi,pi [...]

Ring: --sector k0 / kpi / full selects the k = 0 or k = pi subspace of the translation
i -> i-1 mod M, or the whole (N_up, N_dn) sector.  Torus (sites x + Lx y, nearest-neighbour
bonds): --k kx,ky with each 0 or pi selects the sector of the two translations, or --sector
full.  Prints one JSON line: the sector's dimensions, and, with --maxit > 0, E0, the
iterations and the wall time of the Lanczos run to |dE0| < tol; with --applies N > 0 the mean
CUDA-event time of N products on a projected random vector.  All work runs in the library's
kernels.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

SECTORS = {"full": 0, "k0": 1, "kpi": 2}


def ring_bonds(M: int) -> np.ndarray:
    return np.array([(i, (i + 1) % M) for i in range(M)], dtype=np.int32)


def torus_bonds(Lx: int, Ly: int) -> np.ndarray:
    b = set()
    for y in range(Ly):
        for x in range(Lx):
            s = x + Lx * y
            for dx, dy in ((1, 0), (0, 1)):
                s2 = (x + dx) % Lx + Lx * ((y + dy) % Ly)
                b.add((min(s, s2), max(s, s2)))
    return np.array(sorted(b), dtype=np.int32)


def torus_translations(Lx: int, Ly: int) -> np.ndarray:
    """(x, y) -> (x - 1, y) and (x, y) -> (x, y - 1) as site permutations."""
    tx = [((x - 1) % Lx) + Lx * y for y in range(Ly) for x in range(Lx)]
    ty = [x + Lx * ((y - 1) % Ly) for y in range(Ly) for x in range(Lx)]
    return np.array([tx, ty], dtype=np.int32)


def run(M: int, n_up: int, n_dn: int, sector: str = "k0", U: float = 4.0, t: float = 1.0,
        maxit: int = 300, tol: float = 1e-12, applies: int = 0, torus=None, k=None) -> dict:
    """Ring of M sites, or with torus = (Lx, Ly) the torus (M = Lx Ly) in the sector k =
    (kx, ky), each 0 or pi (sector "full" for the whole (N_up, N_dn) sector)."""
    import torch
    from . import hub
    t0 = time.perf_counter()
    bonds = ring_bonds(M) if torus is None else torus_bonds(*torus)
    m = hub.Hubbard(M, n_up, n_dn, bonds, t, U)
    out = {"M": M, "n_up": n_up, "n_dn": n_dn, "sector": sector, "U": U, "t": t}
    if torus is not None:
        out.update(torus=list(torus), k=None if sector == "full" else list(k))
    try:
        if sector != "full":
            if torus is None:
                m.set_symmetry(SECTORS[sector])
            else:
                if any(kk not in ("0", "pi") for kk in k) or len(k) != 2:
                    raise ValueError("torus momentum components must be 0 or pi")
                m.set_translations(torus_translations(*torus), [1 if kk == "0" else -1 for kk in k])
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
    p.add_argument("--M", type=int, default=None, help="ring of M sites")
    p.add_argument("--torus", default=None, help="LxxLy torus, e.g. 4x4")
    p.add_argument("--k", default="0,0", help="torus sector: kx,ky with each 0 or pi")
    p.add_argument("--n-up", type=int, default=None, help="default M // 2")
    p.add_argument("--n-dn", type=int, default=None, help="default M // 2")
    p.add_argument("--sector", choices=sorted(SECTORS), default="k0", help="ring sector (torus: full or the --k sector)")
    p.add_argument("--U", type=float, default=4.0)
    p.add_argument("--t", type=float, default=1.0)
    p.add_argument("--maxit", type=int, default=300)
    p.add_argument("--tol", type=float, default=1e-12)
    p.add_argument("--applies", type=int, default=0)
    a = p.parse_args(argv)
    torus = None if a.torus is None else tuple(int(v) for v in a.torus.lower().split("x"))
    M = a.M if torus is None else torus[0] * torus[1]
    if M is None:
        p.error("give --M or --torus")
    nu = M // 2 if a.n_up is None else a.n_up
    nd = M // 2 if a.n_dn is None else a.n_dn
    k = [v.strip().lower() for v in a.k.split(",")]
    if torus is not None and a.sector not in ("full",):
        a.sector = "k"
    print(json.dumps(run(M, nu, nd, a.sector, a.U, a.t, a.maxit, a.tol, a.applies, torus, k)))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
