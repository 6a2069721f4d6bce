"""Translation-symmetric k = 0 sector of the periodic Hubbard chain (Sec. V).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  It shares no code with
the CUDA library and never imports it.

Everything here follows the definitions of Sec. V, written out plainly:

* ``translate``      -- one step of the translation T on one spin string, with its
                        fermion sign.  Direction: Table I writes T|0001> = |1000>
                        (site 1 -> site M) and Table II lists T|0011> = -|1001>, so
                        T c+_i T^-1 = c+_{i-1} (sites 1..M cyclic), and with creation
                        operators in ascending site order an electron leaving site 1 for
                        site M passes the other N - 1 of its spin: sign (-1)^(N-1).
* ``spin_periods``, ``spin_nstate`` -- the admissible periods of one spin string
                        (Eqs. count4, count5) and the number of representative states of
                        each period (Eq. count6, read as below).
* ``spin_tables``    -- per state: period, representative, translation and phase
                        (the per/rep/trans/esign arrays of Table II) and, per
                        representative, the phase after one full period (esignb).
* ``combined_reps``  -- the two-spin representative states |r_up> T^n |r_dn>,
                        n < hcf(P_up, P_dn) (Eq. count7), in the order of Table I.
* ``bloch_matrix``   -- V: column b is the k = 0 Bloch state P^-1/2 sum_{r<P} T^r |b>
                        of representative b in the full two-spin basis of Eq. 6.
* ``k0_apply``, ``k0_matrix`` -- H in the k = 0 basis as V^T H V, with H the full
                        two-spin apply of ``hub_oracle`` (the plain definition; the
                        paper's Algorithms III-V build the same matrix another way).

The paper implements k = 0 only.  Every function that depends on the momentum also takes
``omega`` = e^{ik} = -1 for k = pi, the other momentum with real Bloch states (M even):
a(k) = P^-1/2 sum_r e^{-ikr} T^r |a>, which vanishes unless e^{-ikP} times the closing
sign of the orbit is +1.

Several commuting translations (a torus): ``permute`` (a site permutation on one spin string
with its fermion sign), ``site_group`` (closure of the generators), ``group_character``,
``bloch_matrix_group`` (columns sum_g chi(g) g |r>, normalised), ``character_dimension_group``,
``torus_translations`` and ``torus_free_levels`` (U = 0 levels of a momentum sector), and the
test helpers ``group_orbit``, ``group_columns``, ``row_form_group`` that sample states of a
sector in the column order of Table I.

Readings taken where the paper is silent or its formula is garbled:

1. Eq. count6 subtracts, for a period z, the strings whose period is a proper divisor i
   of z.  As printed it subtracts C(i, y_i) for every such period i, which counts the
   strings of period i and those of the periods dividing i again (M = 8, N = 4 gives
   (70 - 6 - 2) / 8, not an integer).  Read: subtract the strings of exact period i,
   i * nstate(i).  The two agree whenever z has at most one smaller admissible period
   (Table II's case).
2. A combined representative whose orbit closes with a minus sign (T^P |b> = -|b>, P
   the orbit's length) has no k = 0 state: its Bloch sum vanishes.  The dimension sum
   of Sec. V counts such states too; they occur only when N_up != N_dn (for N_up =
   N_dn the two spins contribute the same sign).  They are dropped here, and
   ``combined_reps`` flags them.
3. Representatives within a period are taken in ascending order of their integer value,
   periods in the order Eqs. count4-count5 produce them scanning z from M down (Table
   II lists the period-4 cycle of M = 4, N = 2 before the period-2 one).
"""
from __future__ import annotations

from math import comb, gcd

import numpy as np

from . import hub_oracle as O


def translate(M: int, x, N: int):
    """One translation of spin strings x (N electrons each): returns (T x, sign) with
    T|x> = sign |T x> (Sec. V; direction and sign as in the module docstring)."""
    x = np.asarray(x, dtype=np.uint64)
    low = x & np.uint64(1)
    y = (x >> np.uint64(1)) | (low << np.uint64(M - 1))
    sign = np.where(low == 1, float((-1) ** (N - 1)) if N > 0 else 1.0, 1.0)
    return y, sign


def translate_pow(M: int, x, N: int, r: int):
    """T^r applied r times: (T^r x, sign)."""
    y = np.asarray(x, dtype=np.uint64).copy()
    s = np.ones(y.shape)
    for _ in range(r):
        y, si = translate(M, y, N)
        s = s * si
    return y, s


def spin_strings(M: int, N: int) -> np.ndarray:
    """All M-bit strings with N ones, ascending (the one-spin basis of Sec. II)."""
    return np.array(sorted(v for v in range(1 << M) if bin(v).count("1") == N), dtype=np.uint64)


def spin_periods(M: int, N: int) -> list:
    """Admissible periods z of one spin string: mod(M, z) = 0 (Eq. count4) and
    mod(N, M/z) = 0 (Eq. count5), scanning z = M, M-1, ..., 1."""
    return [z for z in range(M, 0, -1) if M % z == 0 and N % (M // z) == 0]


def spin_nstate(M: int, N: int) -> dict:
    """Number of representative states of each admissible period (Eq. count6, reading 1):
    nstate(z) = (C(z, y_z) - sum_i i * nstate(i)) / z over the admissible periods i < z
    dividing z, with y_b = N b / M."""
    out = {}
    for z in sorted(spin_periods(M, N)):
        sub = sum(i * out[i] for i in out if z % i == 0 and i < z)
        num = comb(z, N * z // M) - sub
        assert num % z == 0
        out[z] = num // z
    return out


def spin_nstate_printed(M: int, N: int) -> dict:
    """Eq. count6 exactly as printed: (C(z, y_z) - sum_i C(i, y_i)) / z, as a fraction."""
    per = spin_periods(M, N)
    out = {}
    for z in per:
        sub = sum(comb(i, N * i // M) for i in per if z % i == 0 and i < z)
        out[z] = (comb(z, N * z // M) - sub) / z
    return out


def spin_tables(M: int, N: int) -> dict:
    """Table II for every string of one spin (Sec. V), as arrays over the ascending strings:
    period P, representative rep (smallest integer of the cycle), trans t and esign s with
    T^t |rep> = s |state>, t the smallest such; per-index (position of P in spin_periods)
    and rep-index (position of rep among the representatives of period P, ascending).
    esignb: the phase of T^P |rep> = esignb |rep>."""
    S = spin_strings(M, N)
    n = S.shape[0]
    # the cycle of each string: T^k state for k = 0..M
    cyc = [S]
    cur = S
    for _ in range(M):
        cur, _s = translate(M, cur, N)
        cyc.append(cur)
    cyc = np.stack(cyc)                                  # [M+1, n]
    period = np.full(n, M, dtype=np.int64)
    for k in range(M, 0, -1):
        period = np.where(cyc[k] == S, k, period)
    rep = np.min(cyc[:M], axis=0)
    # translation and phase of each string with respect to its representative
    trans = np.full(n, -1, dtype=np.int64)
    esign = np.zeros(n)
    cur, sg = rep.copy(), np.ones(n)
    for t in range(M):
        hit = (cur == S) & (trans < 0)
        trans = np.where(hit, t, trans)
        esign = np.where(hit, sg, esign)
        cur, si = translate(M, cur, N)
        sg = sg * si
    assert np.all(trans >= 0)
    # phase after one period, per string's representative
    esignb = np.ones(n)
    cur, sg = rep.copy(), np.ones(n)
    for k in range(1, M + 1):
        cur, si = translate(M, cur, N)
        sg = sg * si
        esignb = np.where(k == period, sg, esignb)
    periods = spin_periods(M, N)
    per_index = np.array([periods.index(int(p)) for p in period], dtype=np.int64)
    rep_index = np.zeros(n, dtype=np.int64)
    for p in set(period.tolist()):
        reps_p = np.unique(rep[period == p])
        rep_index[period == p] = np.searchsorted(reps_p, rep[period == p])
    return {"state": S, "period": period, "rep": rep, "trans": trans, "esign": esign,
            "esignb": esignb, "per_index": per_index, "rep_index": rep_index}


def spin_reps(M: int, N: int):
    """Representatives of one spin in the order of Sec. V (period index, then ascending):
    returns (bits, period, esignb)."""
    tb = spin_tables(M, N)
    is_rep = tb["state"] == tb["rep"]
    bits, per, pidx, eb = tb["state"][is_rep], tb["period"][is_rep], tb["per_index"][is_rep], tb["esignb"][is_rep]
    order = np.lexsort((bits, pidx))
    return bits[order], per[order], eb[order]


def combined_reps(M: int, n_up: int, n_dn: int, omega: int = 1) -> dict:
    """Two-spin representatives |r_up> T^n |r_dn>, n = 0 .. hcf(P_up, P_dn) - 1 (Eq.
    count7), ordered as Table I: up representative, then down representative, then n.
    Per entry: up bits, down representative bits, n, down bits of T^n r_dn and the sign of
    T^n |r_dn> = sign |bits>, the orbit length P = lcm(P_up, P_dn) and `null` (reading 2):
    T^P of the signed two-spin state is minus itself (for k = 0; omega^P times that sign is
    -1 in general)."""
    ub, up_, _ = spin_reps(M, n_up)
    db, dp_, _ = spin_reps(M, n_dn)
    rows = []
    for a in range(ub.shape[0]):
        for b in range(db.shape[0]):
            for n in range(gcd(int(up_[a]), int(dp_[b]))):
                rows.append((a, b, n))
    if not rows:
        z = np.zeros(0, dtype=np.uint64)
        return {"up": z, "dn_rep": z, "n": z.astype(np.int64), "dn": z, "sign": np.zeros(0),
                "period": z.astype(np.int64), "null": np.zeros(0, dtype=bool)}
    a, b, n = (np.array(c, dtype=np.int64) for c in zip(*rows))
    up, dn_rep = ub[a], db[b]
    dn = dn_rep.copy()
    sign = np.ones(dn.shape[0])
    for k in range(int(n.max()) + 1):
        move = n > k
        t, s = translate(M, dn, n_dn)
        dn = np.where(move, t, dn)
        sign = np.where(move, sign * s, sign)
    period = np.array([up_[i] * dp_[j] // gcd(int(up_[i]), int(dp_[j])) for i, j in zip(a, b)], dtype=np.int64)
    # the sign T^P picks up on the signed state sign |up, dn>
    cu, cd, sg = up.copy(), dn.copy(), np.ones(dn.shape[0])
    closing = np.ones(dn.shape[0])
    for k in range(1, M + 1):
        cu, su = translate(M, cu, n_up)
        cd, sd = translate(M, cd, n_dn)
        sg = sg * su * sd
        closing = np.where(period == k, sg, closing)
    phase = np.where(period % 2 == 1, float(omega), 1.0)
    return {"up": up, "dn_rep": dn_rep, "n": n, "dn": dn, "sign": sign, "period": period,
            "null": closing * phase < 0}


def k0_dimension(M: int, n_up: int, n_dn: int, omega: int = 1) -> int:
    """Number of k = 0 (omega = -1: k = pi) states: combined representatives whose Bloch sum
    does not vanish."""
    return int(np.count_nonzero(~combined_reps(M, n_up, n_dn, omega)["null"]))


def _index(B: np.ndarray, I: np.ndarray) -> np.ndarray:
    idx = np.searchsorted(B, I)
    assert np.all(idx < B.shape[0]) and np.all(B[np.minimum(idx, B.shape[0] - 1)] == I)
    return idx


def bloch_matrix(M: int, n_up: int, n_dn: int, B: np.ndarray | None = None, omega: int = 1):
    """Sparse V (D x D0): column j = P^-1/2 sum_{r<P} omega^r T^r |b_j> for the j-th non-null
    combined representative b_j = sign |up, dn> (Sec. V; omega = 1 is k = 0, -1 is k = pi),
    rows in the two-spin basis B of Eq. 6 (I = I_up + 2^M I_dn ascending)."""
    import scipy.sparse as sp
    if B is None:
        B = O.basis(M, n_up, n_dn)
    cr = combined_reps(M, n_up, n_dn, omega)
    keep = ~cr["null"]
    up, dn, sg, P = cr["up"][keep], cr["dn"][keep], cr["sign"][keep], cr["period"][keep]
    D0 = up.shape[0]
    rows, cols, vals = [], [], []
    col = np.arange(D0)
    for r in range(M):
        live = r < P
        I = up + (dn << np.uint64(M))
        rows.append(_index(B, I[live]))
        cols.append(col[live])
        vals.append((sg / np.sqrt(P))[live])
        up, su = translate(M, up, n_up)
        dn, sd = translate(M, dn, n_dn)
        sg = sg * su * sd * float(omega)
    V = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(B.shape[0], D0))
    return V


def translation_matrix(M: int, n_up: int, n_dn: int, B: np.ndarray):
    """T on the full two-spin basis as a sparse signed permutation: T|I> = s |I'>."""
    import scipy.sparse as sp
    up, dn = O.spin_parts(M, B)
    tu, su = translate(M, up, n_up)
    td, sd = translate(M, dn, n_dn)
    dst = _index(B, tu + (td << np.uint64(M)))
    return sp.csr_matrix((su * sd, (dst, np.arange(B.shape[0]))), shape=(B.shape[0], B.shape[0]))


def character_dimension(M: int, n_up: int, n_dn: int, B: np.ndarray, omega: int = 1) -> int:
    """dim of the sector as the multiplicity of the eigenvalue omega of T:
    (1/M) sum_r omega^-r tr T^r, each trace the signed count of basis states that T^r maps to
    themselves."""
    up, dn = O.spin_parts(M, B)
    cu, cd, sg = up.copy(), dn.copy(), np.ones(B.shape[0])
    total = float(B.shape[0])                            # r = 0
    for r in range(1, M):
        cu, su = translate(M, cu, n_up)
        cd, sd = translate(M, cd, n_dn)
        sg = sg * su * sd
        total += float(omega) ** r * float(np.sum(sg[(cu == up) & (cd == dn)]))
    val = total / M
    assert abs(val - round(val)) < 1e-9
    return int(round(val))


def k0_apply(model: O.Model, B: np.ndarray, V, phi: np.ndarray) -> np.ndarray:
    """H in the k = 0 basis applied to phi: V^T (H (V phi)) with the full two-spin apply."""
    x = np.asarray(V @ phi, dtype=np.float64)
    return np.asarray(V.T @ O.apply(model, B, x))


def k0_matrix(model: O.Model, B: np.ndarray, V) -> np.ndarray:
    """Dense V^T H V (small sectors only)."""
    D0 = V.shape[1]
    HV = np.empty((B.shape[0], D0))
    for j in range(D0):
        HV[:, j] = O.apply(model, B, np.asarray(V[:, j].toarray()).ravel())
    return np.asarray(V.T @ HV)


def ring_free_k0_levels(M: int, n_up: int, n_dn: int, t: float = 1.0, omega: int = 1) -> np.ndarray:
    """U = 0 nearest-neighbour ring: every eigenvalue of the k = 0 (omega = -1: k = pi)
    sector, sorted.  One-particle states of momentum 2 pi m / M have energy
    -2 t cos(2 pi m / M); a product state lies in the sector when the momenta of all
    electrons add to 0 (pi) modulo 2 pi."""
    from itertools import combinations
    target = 0 if omega == 1 else M // 2
    e = -2.0 * t * np.cos(2.0 * np.pi * np.arange(M) / M)
    ups = [(sum(c) % M, sum(e[list(c)])) for c in combinations(range(M), n_up)]
    dns = [(sum(c) % M, sum(e[list(c)])) for c in combinations(range(M), n_dn)]
    out = [eu + ed for ku, eu in ups for kd, ed in dns if (ku + kd) % M == target]
    return np.sort(np.array(out))


def row_form(M: int, n_up: int, n_dn: int, B: np.ndarray, psi: np.ndarray):
    """Sample a translation-invariant two-spin vector psi on the rows of the up
    representatives: X[i, d] = sqrt(P_i) psi(R_i, d) for the up representatives R_i in
    ascending order (P_i their periods) and every down string d, ascending.  Returns
    (X, reps, periods)."""
    S_up = spin_strings(M, n_up)
    tb = spin_tables(M, n_up)
    reps = S_up[tb["state"] == tb["rep"]]
    per = tb["period"][tb["state"] == tb["rep"]]
    S_dn = spin_strings(M, n_dn)
    I = reps[:, None] + (S_dn[None, :] << np.uint64(M))
    X = psi[_index(B, I.ravel())].reshape(reps.shape[0], S_dn.shape[0]) * np.sqrt(per)[:, None]
    return X, reps, per


def rep_columns(M: int, N: int):
    """Column order of Table I for one spin: representatives R_j ascending, then the
    translations n = 0 .. P_j - 1; per column the string d = T^n R_j and the sign s with
    T^n |R_j> = s |d>.  Returns (d_bits, sign)."""
    tb = spin_tables(M, N)
    is_rep = tb["state"] == tb["rep"]
    reps, per = tb["state"][is_rep], tb["period"][is_rep]
    bits, sign = [], []
    for R, P in zip(reps.tolist(), per.tolist()):
        d, s = np.array([R], dtype=np.uint64), np.ones(1)
        for _ in range(P):
            bits.append(int(d[0]))
            sign.append(float(s[0]))
            d, si = translate(M, d, N)
            s = s * si
    return np.array(bits, dtype=np.uint64), np.array(sign)


def row_form_rep(M: int, n_up: int, n_dn: int, B: np.ndarray, psi: np.ndarray):
    """A translation-invariant two-spin vector psi on the rows of the up representatives
    with the columns of Table I's order: X[i, c] = sqrt(P_i) <R_i (x) T^n R_j | psi>
    = sqrt(P_i) s_c psi(R_i, d_c) for column c = (R_j, n) of ``rep_columns``.  Returns
    (X, reps, periods)."""
    tb = spin_tables(M, n_up)
    is_rep = tb["state"] == tb["rep"]
    reps, per = tb["state"][is_rep], tb["period"][is_rep]
    d_bits, sign = rep_columns(M, n_dn)
    I = reps[:, None] + (d_bits[None, :] << np.uint64(M))
    X = psi[_index(B, I.ravel())].reshape(reps.shape[0], d_bits.shape[0])
    return X * np.sqrt(per)[:, None] * sign[None, :], reps, per


# --------------------------------------------------------------------------------------
# Several commuting translations (a torus): the same construction for the abelian group G
# generated by site permutations, with a real character chi (chi(generator) = +-1).  Sec. V
# treats the chain (one generator, T); the definitions carry over unchanged: a state of the
# sector satisfies g Psi = chi(g) Psi for all g in G, and the Bloch state of a two-spin
# configuration r is sum_g chi(g) g |r>, normalised (zero when the sum cancels).
# --------------------------------------------------------------------------------------

def permute(x: int, N: int, perm) -> tuple:
    """g|x> = sign |x'> for the site permutation g: c+_i -> c+_perm[i], creation operators in
    ascending site order before and after: sign = parity of the reordering of the images."""
    sites = [i for i in range(len(perm)) if (x >> i) & 1]
    images = [perm[i] for i in sites]
    inv = sum(1 for a in range(len(images)) for b in range(a + 1, len(images)) if images[a] > images[b])
    y = 0
    for i in images:
        y |= 1 << i
    return y, (-1.0 if inv & 1 else 1.0)


def site_group(gens) -> list:
    """All elements of the group generated by the site permutations gens, as tuples, each with
    the exponents of the generators of one word reaching it (breadth-first from the identity)."""
    M = len(gens[0])
    ident = tuple(range(M))
    seen = {ident: (0,) * len(gens)}
    order = [ident]
    k = 0
    while k < len(order):
        p = order[k]
        k += 1
        for a, g in enumerate(gens):
            q = tuple(g[p[i]] for i in range(M))          # apply p, then g
            if q not in seen:
                e = list(seen[p])
                e[a] += 1
                seen[q] = tuple(e)
                order.append(q)
    return [(p, seen[p]) for p in order]


def group_character(elements, chars) -> list:
    """chi of every element from the generators' values (+-1), product over a word; raises if
    the values do not define a character (chi(p q) != chi(p) chi(q) for some pair)."""
    out = []
    for p, e in elements:
        c = 1.0
        for ch, n in zip(chars, e):
            c *= float(ch) ** n
        out.append(c)
    pos = {p: k for k, (p, _) in enumerate(elements)}
    for a, (p, _) in enumerate(elements):
        for b, (q, _) in enumerate(elements):
            pq = tuple(q[p[i]] for i in range(len(p)))
            if out[pos[pq]] != out[a] * out[b]:
                raise ValueError("the generator values do not define a character of the group")
    return out


def _act_two_spin(M, I, n_up, n_dn, perm):
    up, dn = int(I) & ((1 << M) - 1), int(I) >> M
    u2, su = permute(up, n_up, perm)
    d2, sd = permute(dn, n_dn, perm)
    return u2 + (d2 << M), su * sd


def bloch_matrix_group(M: int, n_up: int, n_dn: int, B: np.ndarray, gens, chars):
    """Sparse V: one column per orbit of two-spin configurations whose Bloch sum
    sum_g chi(g) g |r> (r the smallest configuration of the orbit) does not cancel, normalised;
    columns ordered by r.  Small sectors only (pure Python)."""
    import scipy.sparse as sp
    els = site_group(gens)
    chi = group_character(els, chars)
    index = {int(v): k for k, v in enumerate(B.tolist())}
    done = np.zeros(B.shape[0], dtype=bool)
    rows, cols, vals = [], [], []
    col = 0
    for k in range(B.shape[0]):
        if done[k]:
            continue
        acc = {}
        for (p, _), c in zip(els, chi):
            I2, s = _act_two_spin(M, B[k], n_up, n_dn, p)
            j = index[I2]
            done[j] = True
            acc[j] = acc.get(j, 0.0) + c * s
        nz = {j: v for j, v in acc.items() if abs(v) > 1e-12}
        if not nz:
            continue
        nrm = np.sqrt(sum(v * v for v in nz.values()))
        for j, v in sorted(nz.items()):
            rows.append(j)
            cols.append(col)
            vals.append(v / nrm)
        col += 1
    return sp.csr_matrix((vals, (rows, cols)), shape=(B.shape[0], col))


def character_dimension_group(M: int, n_up: int, n_dn: int, B: np.ndarray, gens, chars) -> int:
    """Multiplicity of the character chi: (1/|G|) sum_g chi(g) tr(g), each trace the signed
    count of configurations that g maps to themselves (brute force)."""
    els = site_group(gens)
    chi = group_character(els, chars)
    total = 0.0
    for (p, _), c in zip(els, chi):
        tr = 0.0
        for I in B.tolist():
            I2, s = _act_two_spin(M, I, n_up, n_dn, p)
            if I2 == I:
                tr += s
        total += c * tr
    val = total / len(els)
    assert abs(val - round(val)) < 1e-9
    return int(round(val))


def torus_translations(Lx: int, Ly: int):
    """The two translations of the Lx x Ly torus (site x + Lx y), each moving every electron
    one site down its axis: (x, y) -> (x - 1, y) and (x, y) -> (x, y - 1)."""
    tx = [((x - 1) % Lx) + Lx * y for y in range(Ly) for x in range(Lx)]
    ty = [x + Lx * ((y - 1) % Ly) for y in range(Ly) for x in range(Lx)]
    return [tx, ty]


def torus_free_levels(Lx: int, Ly: int, n_up: int, n_dn: int, kx_pi: bool, ky_pi: bool, t: float = 1.0):
    """U = 0 nearest-neighbour torus (Lx, Ly >= 3): every eigenvalue of the sector whose total
    momentum is (pi if kx_pi else 0, pi if ky_pi else 0), sorted.  One-particle states of
    momentum (2 pi mx / Lx, 2 pi my / Ly) have energy -2t (cos kx + cos ky)."""
    from itertools import combinations
    ks = [(mx, my) for my in range(Ly) for mx in range(Lx)]
    e = np.array([-2.0 * t * (np.cos(2 * np.pi * mx / Lx) + np.cos(2 * np.pi * my / Ly)) for mx, my in ks])
    tx, ty = (Lx // 2 if kx_pi else 0), (Ly // 2 if ky_pi else 0)
    ups = [(sum(ks[i][0] for i in c) % Lx, sum(ks[i][1] for i in c) % Ly, sum(e[list(c)])) for c in
           combinations(range(len(ks)), n_up)]
    dns = [(sum(ks[i][0] for i in c) % Lx, sum(ks[i][1] for i in c) % Ly, sum(e[list(c)])) for c in
           combinations(range(len(ks)), n_dn)]
    out = [eu + ed for ax, ay, eu in ups for bx, by, ed in dns if (ax + bx) % Lx == tx and (ay + by) % Ly == ty]
    return np.sort(np.array(out))


def group_orbit(M: int, N: int, x: int, gens):
    """(smallest image, stabiliser as [(element index, sign)]) of string x under the group
    generated by gens (elements in the breadth-first order of ``site_group``)."""
    els = site_group(gens)
    least, stab = x, []
    for k, (p, _) in enumerate(els):
        y, s = permute(x, N, p)
        least = min(least, y)
        if y == x:
            stab.append((k, s))
    return least, stab


def group_columns(M: int, N: int, gens):
    """Column order of Table I for a group: representatives ascending, each followed by the
    images c_k |R> for the coset representatives c_k of its stabiliser (smallest element index
    of each coset, in element order).  Returns (strings, signs)."""
    els = site_group(gens)
    g = len(els)
    pos = {p: k for k, (p, _) in enumerate(els)}
    bits, sign = [], []
    for x in spin_strings(M, N).tolist():
        least, stab = group_orbit(M, N, x, gens)
        if least != x:
            continue
        covered = [False] * g
        for e in range(g):
            if covered[e]:
                continue
            for h, _ in stab:
                pe, ph = els[e][0], els[h][0]
                covered[pos[tuple(ph[pe[i]] for i in range(M))]] = True
            y, s = permute(x, N, els[e][0])
            bits.append(y)
            sign.append(s)
    return np.array(bits, dtype=np.uint64), np.array(sign)


def row_form_group(M: int, n_up: int, n_dn: int, B: np.ndarray, psi: np.ndarray, gens):
    """X[i, c] = sqrt(P_i) s_c psi(R_i, d_c): rows the up representatives (ascending, P_i the
    orbit sizes), columns as ``group_columns``.  Returns (X, reps, orbit sizes)."""
    g = len(site_group(gens))
    reps, per = [], []
    for x in spin_strings(M, n_up).tolist():
        least, stab = group_orbit(M, n_up, x, gens)
        if least == x:
            reps.append(x)
            per.append(g // len(stab))
    d_bits, sign = group_columns(M, n_dn, gens)
    reps = np.array(reps, dtype=np.uint64)
    I = reps[:, None] + (d_bits[None, :] << np.uint64(M))
    X = psi[_index(B, I.ravel())].reshape(reps.shape[0], d_bits.shape[0])
    return X * np.sqrt(np.array(per, dtype=np.float64))[:, None] * sign[None, :], reps, np.array(per)
