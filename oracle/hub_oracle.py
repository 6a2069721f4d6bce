"""Plain, slow CPU oracle for one-band Hubbard exact diagonalisation.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code with
the CUDA library and never imports it.

What it computes (all in FP64):

* ``basis``      -- the Lin-Gubernatis two-spin basis I = I_up + 2^M I_dn of a
                    sector, ascending (Sec. II, Eqs. 5-6, Eq. count2, Table I).
* ``apply``      -- y = H x, one output row at a time, hops applied to the full
                    two-spin state, target found by binary search (Sec. III.A,
                    Sec. V); written in ``hub_oracle.c``.
* ``lanczos``    -- the plain three-term Lanczos recurrence without
                    re-orthogonalisation (Sec. IV, Sec. V) with E0 the lowest
                    eigenvalue of the tridiagonal matrix.
* ``dense_fock`` -- an independent dense Hamiltonian built from Jordan-Wigner
                    creation/annihilation matrices for tiny clusters, for
                    brute-force checks (no hop rule, no sign rule).
* ``expectations`` -- <psi| dH/dtheta |psi> for every bond and site
                    (Hellmann-Feynman gradients), from the definition of H.
* ``ladder``, ``green_cf`` -- c+ / c of one site and spin between two-spin
                    sectors and the zero-temperature Green's function as the two
                    continued fractions of Sec. VII, Eq. count8; ``green_lehmann``
                    (dense eigenvectors) and ``free_green`` (U = 0, one-body
                    orbitals) are independent routes to the same function.

Every function states the passage it follows.  Where the paper is silent, the
reading taken is stated in the docstring.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from math import comb

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hub_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libhub_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C part of the oracle with gcc (OpenMP when available)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i64, i32, dp = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
        lib.hubo_basis.restype = i64
        lib.hubo_basis.argtypes = [i32, i32, i32, dp]
        lib.hubo_apply.restype = i32
        lib.hubo_apply.argtypes = [i32, i32, dp, dp, dp, dp, dp, i64, dp, dp, i64, i64, i32]
        lib.hubo_row.restype = i32
        lib.hubo_row.argtypes = [i32, i32, dp, dp, dp, i64, i64, dp, dp, i32]
        lib.hubo_expect.restype = i32
        lib.hubo_expect.argtypes = [i32, i32, dp, dp, i64, dp, dp, dp, dp]
        lib.hubo_threads.restype = i32
        _lib = lib
    return _lib


def threads() -> int:
    """OpenMP threads the C oracle uses (OMP_NUM_THREADS, else all cores)."""
    return int(_load().hubo_threads())


def _p(a: np.ndarray) -> ctypes.c_void_p:
    return ctypes.c_void_p(a.ctypes.data)


class Model:
    """Lattice and parameters: H = -sum_b t_b sum_s (c+_i c_j + h.c.) + sum_i U_i n_iu n_id
    + sum_i eps_i (n_iu + n_id)  (Sec. I, Eq. 1, with per-bond t and per-site U, eps)."""

    def __init__(self, M, bonds, t, U, eps=None):
        self.M = int(M)
        self.bonds = np.ascontiguousarray(np.asarray(bonds, dtype=np.int32).reshape(-1, 2))
        nb = self.bonds.shape[0]
        t = np.asarray(t, dtype=np.float64)
        self.t = np.ascontiguousarray(np.full(nb, float(t)) if t.ndim == 0 else t.reshape(nb))
        U = np.asarray(U, dtype=np.float64)
        self.U = np.ascontiguousarray(np.full(self.M, float(U)) if U.ndim == 0 else U.reshape(self.M))
        e = np.zeros(self.M) if eps is None else np.asarray(eps, dtype=np.float64)
        self.eps = np.ascontiguousarray(np.full(self.M, float(e)) if e.ndim == 0 else e.reshape(self.M))

    @property
    def n_bonds(self):
        return self.bonds.shape[0]


def basis(M: int, n_up: int, n_dn: int) -> np.ndarray:
    """Sorted two-spin basis of sector (n_up, n_dn) (Sec. II, Eqs. 5-6 and count2)."""
    lib = _load()
    D = lib.hubo_basis(M, n_up, n_dn, None)
    if D < 0:
        raise ValueError("bad sector")
    out = np.empty(D, dtype=np.uint64)
    if D:
        lib.hubo_basis(M, n_up, n_dn, _p(out))
    return out


def spin_parts(M: int, I: np.ndarray):
    """Split two-spin states into (I_up, I_dn) (Sec. II, Eq. 6)."""
    mask = np.uint64((1 << M) - 1)
    return I & mask, I >> np.uint64(M)


def apply(model: Model, B: np.ndarray, x: np.ndarray, rows=None, absolute: bool = False) -> np.ndarray:
    """(H x)_n for n in rows = (r0, r1) (default: all), matrix-free (Sec. IV, Sec. V).
    With absolute=True: (|H| |x|)_n, every matrix element and x entry by absolute value."""
    lib = _load()
    D = B.shape[0]
    r0, r1 = (0, D) if rows is None else rows
    x = np.ascontiguousarray(x, dtype=np.float64)
    assert x.shape == (D,)
    y = np.empty(r1 - r0, dtype=np.float64)
    rc = lib.hubo_apply(model.M, model.n_bonds, _p(model.bonds), _p(model.t), _p(model.U),
                        _p(model.eps), _p(B), D, _p(x), _p(y), r0, r1, 1 if absolute else 0)
    if rc != 0:
        raise RuntimeError(f"hubo_apply failed ({rc})")
    return y


def row(model: Model, B: np.ndarray, n: int):
    """Off-diagonal entries (cols, vals) of row n of H, sorted by column (Sec. III.A)."""
    lib = _load()
    cap = 2 * model.n_bonds
    cols = np.empty(max(cap, 1), dtype=np.int64)
    vals = np.empty(max(cap, 1), dtype=np.float64)
    k = lib.hubo_row(model.M, model.n_bonds, _p(model.bonds), _p(model.t), _p(B), B.shape[0], n,
                     _p(cols), _p(vals), cap)
    if k < 0:
        raise RuntimeError("hubo_row failed")
    order = np.argsort(cols[:k], kind="stable")
    return cols[:k][order], vals[:k][order]


def spin_csr(model: Model, n_up: int, n_dn: int, spin: str, B: np.ndarray | None = None):
    """The one-spin hopping matrix H_up or H_dn (Sec. IV.A, Eqs. 9-10), read off the
    two-spin Hamiltonian: by Eq. 11 the spin-up block of rows n = u (I_dn = first
    state) holds H_up, and the columns of rows n = d*count_up (I_up = first state)
    that keep I_up fixed hold H_dn.  Returns (basis_sigma, rowptr, cols, vals) with
    columns sorted ascending inside each row."""
    if B is None:
        B = basis(model.M, n_up, n_dn)
    n_u, n_d = comb(model.M, n_up), comb(model.M, n_dn)
    I_up, I_dn = spin_parts(model.M, B)
    if spin == "up":
        states = I_up[:n_u].astype(np.uint32)
        rows_n = [u for u in range(n_u)]
        keep = lambda c: (c // n_u) == 0          # same I_dn block
        to_idx = lambda c: c % n_u
    else:
        states = I_dn[::n_u][:n_d].astype(np.uint32)
        rows_n = [d * n_u for d in range(n_d)]
        keep = lambda c: (c % n_u) == 0           # same I_up
        to_idx = lambda c: c // n_u
    rowptr = [0]
    cols, vals = [], []
    for n in rows_n:
        c, v = row(model, B, n)
        sel = keep(c)
        cc, vv = to_idx(c[sel]), v[sel]
        o = np.argsort(cc, kind="stable")
        cols.extend(cc[o].tolist())
        vals.extend(vv[o].tolist())
        rowptr.append(len(cols))
    return (states, np.asarray(rowptr, dtype=np.int64), np.asarray(cols, dtype=np.int64),
            np.asarray(vals, dtype=np.float64))


def diagonal(model: Model, B: np.ndarray) -> np.ndarray:
    """Diagonal of H: sum_i U_i n_iu n_id + eps_i (n_iu + n_id) (Sec. III.B), per state."""
    M = model.M
    d = np.zeros(B.shape[0])
    for i in range(M):
        nu = ((B >> np.uint64(i)) & np.uint64(1)).astype(np.float64)
        nd = ((B >> np.uint64(M + i)) & np.uint64(1)).astype(np.float64)
        d += model.U[i] * nu * nd + model.eps[i] * (nu + nd)
    return d


def tridiag_lowest(alpha, beta) -> float:
    """Lowest eigenvalue of the symmetric tridiagonal matrix (diag alpha, offdiag beta)."""
    from scipy.linalg import eigvalsh_tridiagonal
    a = np.asarray(alpha, dtype=np.float64)
    if a.size == 1:
        return float(a[0])
    return float(eigvalsh_tridiagonal(a, np.asarray(beta[: a.size - 1], dtype=np.float64),
                                      select="i", select_range=(0, 0))[0])


def lanczos(model: Model, B: np.ndarray, x0: np.ndarray, maxit: int = 300, tol: float = 1e-12,
            want_psi: bool = False, fixed_iters: bool = False):
    """Plain Lanczos, no re-orthogonalisation (Sec. IV, Sec. V).

    q_1 = x0/|x0|; for j = 1..: w = H q_j; w -= beta_{j-1} q_{j-1}; alpha_j = <q_j, w>;
    w -= alpha_j q_j; beta_j = |w|; E0_j = lowest eigenvalue of T_j; stop when
    |E0_j - E0_{j-1}| < tol (reading: the paper names no criterion), when beta_j
    vanishes (invariant subspace), or at maxit.  With want_psi the recurrence is
    run a second time to form psi = sum_k v_k q_k from the lowest eigenvector v of
    T (the paper computes eigenvectors too, Table IV).
    Returns dict(E0, iters, alpha, beta, psi, converged).
    """
    D = B.shape[0]
    q = np.asarray(x0, dtype=np.float64) / np.linalg.norm(x0)
    q_prev = np.zeros(D)
    alpha, beta = [], []
    b_prev = 0.0
    E_prev = None
    converged = False
    for j in range(maxit):
        w = apply(model, B, q)
        w -= b_prev * q_prev
        a = float(np.dot(q, w))
        w -= a * q
        b = float(np.linalg.norm(w))
        alpha.append(a)
        beta.append(b)
        E = tridiag_lowest(alpha, beta)
        if not fixed_iters and E_prev is not None and abs(E - E_prev) < tol:
            converged = True
            break
        E_prev = E
        if b <= 1e-14 * max(1.0, abs(a)):
            converged = True
            break
        q_prev, q = q, w / b
        b_prev = b
    out = dict(E0=E, iters=len(alpha), alpha=np.array(alpha), beta=np.array(beta), psi=None,
               converged=converged)
    if want_psi:
        from scipy.linalg import eigh_tridiagonal
        k = len(alpha)
        if k == 1:
            v = np.ones(1)
        else:
            _, vecs = eigh_tridiagonal(out["alpha"], out["beta"][: k - 1], select="i", select_range=(0, 0))
            v = vecs[:, 0]
        q = np.asarray(x0, dtype=np.float64) / np.linalg.norm(x0)
        q_prev = np.zeros(D)
        psi = v[0] * q
        for j in range(k - 1):
            w = apply(model, B, q) - out["beta"][j - 1] * q_prev if j > 0 else apply(model, B, q)
            w -= out["alpha"][j] * q
            q_prev, q = q, w / out["beta"][j]
            psi += v[j + 1] * q
        out["psi"] = psi / np.linalg.norm(psi)
    return out


def quadratic_forms(model: Model, B: np.ndarray, v: np.ndarray):
    """Raw quadratic forms v^T (dH/dtheta) v for every bond and site (no normalisation)."""
    lib = _load()
    v = np.ascontiguousarray(v, dtype=np.float64)
    dt = np.empty(model.n_bonds)
    dU = np.empty(model.M)
    de = np.empty(model.M)
    rc = lib.hubo_expect(model.M, model.n_bonds, _p(model.bonds), _p(B), B.shape[0], _p(v),
                         _p(dt), _p(dU), _p(de))
    if rc != 0:
        raise RuntimeError("hubo_expect failed")
    return dt, dU, de


def bilinear_forms(model: Model, B: np.ndarray, a: np.ndarray, b: np.ndarray):
    """a^T (dH/dtheta) b by polarisation of the symmetric forms: (q(a+b) - q(a-b)) / 4."""
    p = quadratic_forms(model, B, a + b)
    m = quadratic_forms(model, B, a - b)
    return tuple((x - y) / 4.0 for x, y in zip(p, m))


def expectations(model: Model, B: np.ndarray, psi: np.ndarray):
    """(dE/dt_b, dE/dU_i, dE/deps_i) = <psi|dH/dtheta|psi>/<psi|psi> (Hellmann-Feynman),
    with dH/dt_b = -sum_s (c+_i c_j + h.c.), dH/dU_i = n_iu n_id, dH/deps_i = n_iu + n_id."""
    lib = _load()
    psi = np.ascontiguousarray(psi, dtype=np.float64)
    dt = np.empty(model.n_bonds)
    dU = np.empty(model.M)
    de = np.empty(model.M)
    rc = lib.hubo_expect(model.M, model.n_bonds, _p(model.bonds), _p(B), B.shape[0], _p(psi),
                         _p(dt), _p(dU), _p(de))
    if rc != 0:
        raise RuntimeError("hubo_expect failed")
    nrm = float(np.dot(psi, psi))
    return dt / nrm, dU / nrm, de / nrm


# --------------------------------------------------------------------------------------
# Independent dense construction for tiny clusters (no hop rule, no sign rule).
# --------------------------------------------------------------------------------------

def _annihilator(L: int, k: int):
    """c_k on the 2^L Fock space with modes ordered as in Sec. II, Eq. 7 (mode k <-> bit k;
    |I> = prod over set bits in ascending mode order of c+_k |0>).  Moving c_k to its
    creation partner passes the occupied modes below k, so
    <I - 2^k| c_k |I> = (-1)^(number of occupied modes below k)."""
    import scipy.sparse as sp
    dim = 1 << L
    I = np.arange(dim, dtype=np.int64)
    has = (I >> k) & 1 == 1
    src = I[has]
    below = src & ((1 << k) - 1)
    cnt = np.zeros_like(below)
    for m in range(k):
        cnt += (below >> m) & 1
    sign = np.where(cnt % 2 == 0, 1.0, -1.0)
    return sp.csr_matrix((sign, (src ^ (1 << k), src)), shape=(dim, dim))


def dense_fock(model: Model, n_up: int, n_dn: int) -> np.ndarray:
    """Dense H of sector (n_up, n_dn) from products of Jordan-Wigner operator matrices
    (Eq. 1), rows/columns in ascending two-spin order (Eq. 6).  Up site i is mode i,
    down site i is mode M+i (Sec. II, Eq. 5).  For 2M <= 14 only."""
    M = model.M
    L = 2 * M
    assert L <= 14, "dense Fock construction is for tiny clusters"
    c = [_annihilator(L, k) for k in range(L)]
    cd = [ck.T.tocsr() for ck in c]
    n = [cd[k] @ c[k] for k in range(L)]
    dim = 1 << L
    import scipy.sparse as sp
    H = sp.csr_matrix((dim, dim))
    for b, (i, j) in enumerate(model.bonds.tolist()):
        for off in (0, M):
            H = H - model.t[b] * (cd[off + i] @ c[off + j] + cd[off + j] @ c[off + i])
    for i in range(M):
        H = H + model.U[i] * (n[i] @ n[M + i]) + model.eps[i] * (n[i] + n[M + i])
    I = np.arange(dim)
    pu = np.array([bin(v & ((1 << M) - 1)).count("1") for v in I])
    pd = np.array([bin(v >> M).count("1") for v in I])
    sel = I[(pu == n_up) & (pd == n_dn)]
    return H[sel][:, sel].toarray()


def free_fermion_E0(model: Model, n_up: int, n_dn: int) -> float:
    """U = 0 ground energy: sum of the lowest n_up plus lowest n_dn eigenvalues of the
    one-body matrix h_ij = -t_ij (both directions), h_ii = eps_i."""
    M = model.M
    h = np.diag(model.eps.copy())
    for b, (i, j) in enumerate(model.bonds.tolist()):
        h[i, j] -= model.t[b]
        h[j, i] -= model.t[b]
    w = np.linalg.eigvalsh(h)
    return float(w[:n_up].sum() + w[:n_dn].sum())


def nnz_spin(M: int, n_sigma: int, n_bonds: int) -> int:
    """Nonzeros of H_sigma: F * C(M-2, N_sigma - 1) with F = 2 * (number of bonds)
    (Sec. IV.A, for M > 2 and 0 < N_sigma < M)."""
    return 2 * n_bonds * comb(M - 2, n_sigma - 1)


# --------------------------------------------------------------------------------------
# One-particle Green's function at zero temperature (Sec. VII, Eq. count8).
# --------------------------------------------------------------------------------------

def _popcount(a: np.ndarray, bits: int) -> np.ndarray:
    cnt = np.zeros(a.shape, dtype=np.int64)
    for m in range(bits):
        cnt += (a >> m) & 1
    return cnt


def ladder(M: int, B_from: np.ndarray, B_to: np.ndarray, site: int, spin: int, create: bool,
           x: np.ndarray) -> np.ndarray:
    """y = c+_{site,spin} x (create) or c_{site,spin} x, x in the sector with two-spin basis
    B_from, y in the sector with basis B_to (Sec. VII, the vecin construction).  The mode of
    (site, spin) is bit site + M*spin of the two-spin integer (Sec. II, Eq. 5), and the modes
    are ordered as in Eq. 7, so the operator passes the occupied modes below its own:
    c+_k |I> = (-1)^(set bits of I below k) |I + 2^k> and c_k |I> = (-1)^(...) |I - 2^k>.
    A target state comes from the source state with its bit flipped, if that exists."""
    bit = np.int64(1) << np.int64(site + M * spin)
    I_to = B_to.astype(np.int64)
    has = (I_to & bit) != 0
    ok = has if create else ~has
    I_src = I_to ^ bit
    sign = np.where(_popcount(I_src & (bit - 1), 2 * M) % 2 == 0, 1.0, -1.0)
    Bf = B_from.astype(np.int64)
    idx = np.searchsorted(Bf, I_src)
    idx_c = np.minimum(idx, Bf.size - 1) if Bf.size else idx
    found = ok & (idx < Bf.size) & (Bf[idx_c] == I_src) if Bf.size else np.zeros(I_to.shape, bool)
    y = np.zeros(B_to.size)
    y[found] = sign[found] * np.asarray(x, dtype=np.float64)[idx[found]]
    return y


def continued_fraction(alpha, beta, norm2: float, E0: float, sign: int, z) -> np.ndarray:
    """<v|(z - s (H - E0))^-1|v> from the Lanczos coefficients of v (Sec. VII): the (0, 0)
    element of the resolvent of the tridiagonal T, norm2 / (z - s(a_0 - E0) - b_0^2 /
    (z - s(a_1 - E0) - ...)), s = +1 particle term, -1 hole term of Eq. count8."""
    z = np.atleast_1d(np.asarray(z, dtype=np.complex128))
    k = len(alpha)
    if k == 0:
        return np.zeros(z.shape, dtype=np.complex128)
    f = z - sign * (alpha[k - 1] - E0)
    for j in range(k - 2, -1, -1):
        f = z - sign * (alpha[j] - E0) - beta[j] ** 2 / f
    return norm2 / f


def green_cf(model_plus: Model, B_plus: np.ndarray, v_plus: np.ndarray, model_minus: Model,
             B_minus: np.ndarray, v_minus: np.ndarray, E0: float, z, k: int = 400) -> np.ndarray:
    """Eq. count8 as the sum of the two continued fractions, each from up to k steps of the
    plain Lanczos recurrence (``lanczos``) started at v_plus = c+ psi0 (sector N + 1) and
    v_minus = c psi0 (sector N - 1); an empty or zero start vector contributes 0."""
    g = np.zeros(np.atleast_1d(z).shape, dtype=np.complex128)
    for model, B, v, s in ((model_plus, B_plus, v_plus, 1), (model_minus, B_minus, v_minus, -1)):
        if v is None or v.size == 0 or not np.any(v):
            continue
        r = lanczos(model, B, v, maxit=min(k, v.size), fixed_iters=True)
        g += continued_fraction(r["alpha"], r["beta"], float(np.dot(v, v)), E0, s, z)
    return g


def green_lehmann(model: Model, n_up: int, n_dn: int, site: int, spin: int, z) -> np.ndarray:
    """Eq. count8 from the Lehmann sum over dense eigenvectors (tiny clusters, 2M <= 14):
    sum_m |<m|c+|psi0>|^2 / (z - (E_m - E0)) + sum_m |<m|c|psi0>|^2 / (z + (E_m - E0)), with
    H from Jordan-Wigner operator matrices (``dense_fock``) and c from ``_annihilator``
    (no ladder rule).  The ground state of (n_up, n_dn) must be non-degenerate."""
    M = model.M
    L = 2 * M
    k = site + M * spin
    c = _annihilator(L, k).toarray()
    I = np.arange(1 << L)
    pu = np.array([bin(v & ((1 << M) - 1)).count("1") for v in I])
    pd = np.array([bin(v >> M).count("1") for v in I])

    def sector(nu, nd):
        return I[(pu == nu) & (pd == nd)]

    S0 = sector(n_up, n_dn)
    w0, V0 = np.linalg.eigh(dense_fock(model, n_up, n_dn))
    assert w0.size < 2 or w0[1] - w0[0] > 1e-8, "degenerate ground state"
    E0, psi = w0[0], V0[:, 0]
    z = np.atleast_1d(np.asarray(z, dtype=np.complex128))
    g = np.zeros(z.shape, dtype=np.complex128)
    for dn_, s, op in ((1, 1, c.T), (-1, -1, c)):
        nu, nd = (n_up + dn_, n_dn) if spin == 0 else (n_up, n_dn + dn_)
        if not (0 <= nu <= M and 0 <= nd <= M):
            continue
        S1 = sector(nu, nd)
        v = op[np.ix_(S1, S0)] @ psi
        w1, V1 = np.linalg.eigh(dense_fock(model, nu, nd))
        amp = V1.T @ v
        for a2, Em in zip(amp ** 2, w1):
            g += a2 / (z - s * (Em - E0))
    return g


def free_green(model: Model, n_sigma: int, site: int, z) -> np.ndarray:
    """U = 0: the Green's function of a non-interacting ground state (lowest n_sigma one-body
    orbitals phi_k of h_ij = -t_ij, h_ii = eps_i filled, gap above them) is
    sum_k |phi_k(site)|^2 / (z - e_k) over all orbitals: adding an electron to an empty
    orbital costs e_k, removing one from a filled orbital gives E_m - E0 = -e_k."""
    M = model.M
    h = np.diag(model.eps.copy())
    for b, (i, j) in enumerate(model.bonds.tolist()):
        h[i, j] -= model.t[b]
        h[j, i] -= model.t[b]
    e, phi = np.linalg.eigh(h)
    if 0 < n_sigma < M:
        assert e[n_sigma] - e[n_sigma - 1] > 1e-8, "open shell: degenerate ground state"
    z = np.atleast_1d(np.asarray(z, dtype=np.complex128))
    return np.sum(phi[site, :] ** 2 / (z[:, None] - e[None, :]), axis=1)


# --------------------------------------------------------------------------------------
# A few low-lying eigenvalues from plain Lanczos (Sec. IV).
# --------------------------------------------------------------------------------------

def lanczos_spectrum(model: Model, B: np.ndarray, x0: np.ndarray, maxit: int, n_eig: int, rtol: float = 1e-10):
    """The ground state and a few low-lying excited states (Sec. IV) from maxit steps of the
    plain recurrence (``lanczos``).  Without re-orthogonalisation the tridiagonal T acquires
    spurious copies of converged eigenvalues; reading: they are removed by the test of
    Cullum and Willoughby (Lanczos Algorithms for Large Symmetric Eigenvalue Computations,
    1985): a numerically multiple eigenvalue of T is kept once, a simple one is spurious if
    T without its first row and column has it too (tolerance rtol * max(1, |T|)).  Returns
    the lowest n_eig distinct kept values (ascending)."""
    from scipy.linalg import eigvalsh_tridiagonal
    r = lanczos(model, B, x0, maxit=maxit, fixed_iters=True)
    a, b = r["alpha"], r["beta"]
    k = a.size
    mu = eigvalsh_tridiagonal(a, b[: k - 1]) if k > 1 else a.copy()
    nu = eigvalsh_tridiagonal(a[1:], b[1: k - 1]) if k > 2 else (a[1:].copy() if k == 2 else np.zeros(0))
    tol = rtol * max(1.0, float(np.max(np.abs(mu))))
    good = []
    i = 0
    while i < k:
        j = i + 1
        while j < k and mu[j] - mu[j - 1] <= tol:
            j += 1
        if j - i > 1 or not np.any(np.abs(nu - mu[i]) <= tol):
            good.append(float(mu[i]))
        i = j
    return np.array(good[:n_eig])
