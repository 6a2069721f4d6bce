"""Seeded synthetic inputs: lattices, parameter draws and start vectors.

This module holds no arithmetic of the method itself (no basis, no hopping, no
Hamiltonian).  It only produces the inputs that both the CUDA path and the CPU
oracle consume, so both sides see bit-identical bonds, parameters and vectors.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): state advances by the golden
gamma 0x9E3779B97F4A7C15 and each output is the state passed through the
finaliser (xor-shift 30, multiply 0xBF58476D1CE4E5B9, xor-shift 27, multiply
0x94D049BB133111EB, xor-shift 31).  A uniform double in [0, 1) is the top 53
bits times 2^-53; normals use the Box-Muller transform on pairs of uniforms.
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n consecutive SplitMix64 outputs for the given seed (counter-based: output k
    depends only on seed and k)."""
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed) + k * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, lo: float = 0.0, hi: float = 1.0, offset: int = 0) -> np.ndarray:
    """n uniform doubles in [lo, hi)."""
    u = (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return lo + (hi - lo) * u


def normal(seed: int, n: int, chunk: int = 1 << 24) -> np.ndarray:
    """n standard normal doubles (Box-Muller on consecutive uniform pairs), chunked so
    that large vectors need little temporary memory."""
    out = np.empty(n, dtype=np.float64)
    m = (n + 1) // 2
    for s in range(0, m, chunk):
        c = min(chunk, m - s)
        u = uniform(seed, 2 * c, offset=2 * s)
        u1 = 1.0 - u[0::2]                       # (0, 1]: log is finite
        u2 = u[1::2]
        r = np.sqrt(-2.0 * np.log(u1))
        z = np.empty(2 * c)
        z[0::2] = r * np.cos(2.0 * np.pi * u2)
        z[1::2] = r * np.sin(2.0 * np.pi * u2)
        lo = 2 * s
        out[lo:lo + min(2 * c, n - lo)] = z[: min(2 * c, n - lo)]
    return out


# ---------------------------------------------------------------------------------------
# Lattices.  Site s of an Lx x Ly lattice is s = x + Lx*y (x fastest); bond lists are
# undirected pairs (i, j), listed once.
# ---------------------------------------------------------------------------------------

def ring_bonds(M: int) -> np.ndarray:
    """1D ring of M sites with periodic boundary (for M = 2 the single bond (0, 1))."""
    if M == 2:
        return np.array([[0, 1]], dtype=np.int32)
    return np.array([[i, (i + 1) % M] for i in range(M)], dtype=np.int32)


def chain_bonds(M: int) -> np.ndarray:
    """1D open chain."""
    return np.array([[i, i + 1] for i in range(M - 1)], dtype=np.int32)


def square_bonds(Lx: int, Ly: int, periodic: bool = True) -> np.ndarray:
    """Lx x Ly square lattice: horizontal bonds first (row by row), then vertical ones."""
    bonds = []
    for y in range(Ly):
        for x in range(Lx):
            if x + 1 < Lx or (periodic and Lx > 2):
                bonds.append((x + Lx * y, (x + 1) % Lx + Lx * y))
    for y in range(Ly):
        for x in range(Lx):
            if y + 1 < Ly or (periodic and Ly > 2):
                bonds.append((x + Lx * y, x + Lx * ((y + 1) % Ly)))
    return np.array(bonds, dtype=np.int32)


def star_bonds(n_bath: int) -> np.ndarray:
    """Anderson impurity star: impurity site 0 coupled to bath sites 1..n_bath."""
    return np.array([[0, k] for k in range(1, n_bath + 1)], dtype=np.int32)


# ---------------------------------------------------------------------------------------
# Named workloads (the shapes of the benchmark cases).
# ---------------------------------------------------------------------------------------

def ring8():
    """1D periodic ring, M = 8, (4, 4), t = 1, U = 4."""
    return dict(name="ring M=8 (4,4) U=4", M=8, n_up=4, n_dn=4, bonds=ring_bonds(8),
                t=np.ones(8), U=np.full(8, 4.0), eps=np.zeros(8))


def square4x4(U: float = 4.0):
    """4x4 periodic square lattice, half filling (8, 8), t = 1."""
    b = square_bonds(4, 4, True)
    return dict(name=f"4x4 PBC (8,8) U={U:g}", M=16, n_up=8, n_dn=8, bonds=b,
                t=np.ones(len(b)), U=np.full(16, float(U)), eps=np.zeros(16))


def disordered3x4(seed: int = 0):
    """3x4 open lattice, (6, 6): t_b = 1 + U[-0.1, 0.1], U_i ~ U[2, 8], eps_i ~ U[-0.5, 0.5]."""
    b = square_bonds(3, 4, False)
    nb = len(b)
    t = 1.0 + uniform(seed, nb, -0.1, 0.1)
    U = uniform(seed + 1, 12, 2.0, 8.0)
    eps = uniform(seed + 2, 12, -0.5, 0.5)
    return dict(name="3x4 open (6,6) disordered", M=12, n_up=6, n_dn=6, bonds=b, t=t, U=U, eps=eps)


def square3x6(U: float = 4.0):
    """3x6 periodic lattice, (9, 9), t = 1."""
    b = square_bonds(3, 6, True)
    return dict(name=f"3x6 PBC (9,9) U={U:g}", M=18, n_up=9, n_dn=9, bonds=b,
                t=np.ones(len(b)), U=np.full(18, float(U)), eps=np.zeros(18))


def aim_star(param_set: int, n_bath: int = 7, U_imp: float = 4.0, seed: int = 0):
    """Anderson impurity star, impurity = site 0: bath levels eps_k ~ U[-2, 2],
    hybridisations V_k ~ U[0.2, 1] (entering as hopping t_k = V_k), U only on the
    impurity, impurity level -U_imp/2.  param_set selects an independent draw."""
    M = n_bath + 1
    s = seed * 1_000_003 + param_set * 2
    V = uniform(s, n_bath, 0.2, 1.0)
    eb = uniform(s + 1, n_bath, -2.0, 2.0)
    U = np.zeros(M)
    U[0] = U_imp
    eps = np.concatenate([[-U_imp / 2.0], eb])
    return dict(name=f"AIM star M={M} set {param_set}", M=M, bonds=star_bonds(n_bath), t=V, U=U, eps=eps)
