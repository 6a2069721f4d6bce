"""Write tests/golden/square4x4_E0.txt: the ground-state energy of the 4x4 periodic
Hubbard lattice at half filling, (N_up, N_dn) = (8, 8), t = 1, from the CPU oracle only.

The oracle's plain Lanczos (Sec. IV, Sec. V: no re-orthogonalisation, E0 the lowest
eigenvalue of the tridiagonal matrix) runs in the two-spin basis of dimension
12870^2 = 165,636,900 from the seed-0 normal start vector until |E0_j - E0_{j-1}| < 1e-12.
Nothing here touches the CUDA library.  One U takes two to four hours on eight cores
(45 to 90 s per oracle product there, 105 to 140 products).

    python tests/golden/make_square4x4_E0.py 4 2 8

Each finished U is appended as one line (U, E0 to 15 significant digits, iterations,
final |dE0|), so an interrupted run keeps what it finished.
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import hub_oracle as O  # noqa: E402
from paper_1307_7542_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(HERE, "square4x4_E0.txt")
HEADER = """# 4x4 periodic square lattice (bonds: workloads.square_bonds(4, 4)), N_up = N_dn = 8,
# t = 1, uniform U: ground-state energy from the CPU oracle's plain Lanczos (two-spin
# basis, binary-search products, Sec. IV-V) started from workloads.normal(0, D), stopped
# at |E0_j - E0_{j-1}| < 1e-12.  Written by tests/golden/make_square4x4_E0.py.
# Columns: U, E0, Lanczos iterations, last |dE0|.
"""


def run(U: float):
    w = W.square4x4(U)
    m = O.Model(w["M"], w["bonds"], w["t"], w["U"], w["eps"])
    B = O.basis(w["M"], w["n_up"], w["n_dn"])
    x0 = W.normal(0, B.shape[0])
    t0 = time.time()
    r = O.lanczos(m, B, x0, maxit=400, tol=1e-12)
    a, b = r["alpha"], r["beta"]
    k = len(a)
    dE = abs(r["E0"] - O.tridiag_lowest(a[: k - 1], b[: k - 1])) if k > 1 else float("nan")
    print(f"U={U:g} E0={r['E0']:.15g} iters={k} dE={dE:.2e} converged={r['converged']} "
          f"{time.time() - t0:.0f} s", flush=True)
    if not r["converged"]:
        raise SystemExit(f"U={U:g}: not converged in {k} iterations")
    return r["E0"], k, dE


def main(argv):
    Us = [float(a) for a in argv] or [4.0]
    if not os.path.exists(OUT):
        with open(OUT, "w") as f:
            f.write(HEADER)
    for U in Us:
        E0, k, dE = run(U)
        with open(OUT, "a") as f:
            f.write(f"{U:g} {E0:.15g} {k} {dE:.2e}\n")


if __name__ == "__main__":
    main(sys.argv[1:])
