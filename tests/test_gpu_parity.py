"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer work (spin bases, CSR structure) is compared bit for bit; FP64 results within
the stated tolerances: per apply entry |y - y_ref| <= 1e-13 (|H||x|)_n,
E0 within 1e-10 relative, gradients within the stated bounds.
"""
import math

import numpy as np
import pytest

from helpers import abs_bound, assert_entrywise, oracle_model
from oracle import hub_oracle as O
from paper_1307_7542_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def hub(cuda_ok):
    import __graft_entry__
    __graft_entry__.build()
    from paper_1307_7542_gb300 import hub as H
    return H


def _random_workload(M, nu, nd, seed, long_range=True, uniform=False):
    bonds = [tuple(b) for b in W.ring_bonds(M).tolist()]
    if long_range and M >= 4:
        r = W.uniform(seed + 99, 2 * M)
        for k in range(M):
            i, j = int(r[2 * k] * M), int(r[2 * k + 1] * M)
            if i != j and (i, j) not in bonds and (j, i) not in bonds:
                bonds.append((i, j))
    nb = len(bonds)
    if uniform:
        t, U, eps = np.ones(nb), np.full(M, 4.0), np.zeros(M)
    else:
        t = W.uniform(seed, nb, 0.3, 1.3) * np.where(W.uniform(seed + 1, nb) < 0.3, -1.0, 1.0)
        U = W.uniform(seed + 2, M, 0.0, 6.0)
        eps = W.uniform(seed + 3, M, -0.7, 0.7)
    return dict(M=M, n_up=nu, n_dn=nd, bonds=np.array(bonds, dtype=np.int32), t=t, U=U, eps=eps)


def _gpu_model(hub, w):
    return hub.Hubbard(w["M"], w["n_up"], w["n_dn"], w["bonds"], w["t"], w["U"], w.get("eps"))


# ------------------------------------------------------------------- basis and CSR (bit-exact)

@pytest.mark.parametrize("M,nu,nd", [(1, 0, 1), (1, 1, 1), (2, 1, 1), (3, 2, 1), (8, 4, 4), (8, 3, 5),
                                     (12, 6, 6), (16, 8, 8), (16, 0, 16), (18, 9, 9), (20, 3, 17)])
def test_basis_bitexact(hub, M, nu, nd):
    """Spin bases equal the oracle's per-spin lists (Sec. II, Table I order), bit for bit."""
    h = hub.hub_basis(M, nu, nd)
    try:
        n_u, n_d = hub.hub_dims(h)
        assert (n_u, n_d) == (math.comb(M, nu), math.comb(M, nd))
        up = hub.hub_get_basis(h, 0, n_u)
        dn = hub.hub_get_basis(h, 1, n_d)
        ref_up = O.spin_parts(M, O.basis(M, nu, 0))[0].astype(np.uint32)
        ref_dn = O.spin_parts(M, O.basis(M, 0, nd))[1].astype(np.uint32)
        assert np.array_equal(up, ref_up)
        assert np.array_equal(dn, ref_dn)
    finally:
        hub.hub_free(h)


def _csr_case(name):
    if name == "ring8":
        return W.ring8()
    if name == "random8":
        return _random_workload(8, 3, 5, 1)
    if name == "aim":
        p = W.aim_star(2)
        return dict(p, n_up=4, n_dn=5)
    if name == "open3x4":
        return dict(W.disordered3x4(), n_up=6, n_dn=6)
    if name == "square4x4":
        return W.square4x4(4.0)
    if name == "square3x6":
        return W.square3x6(4.0)
    raise KeyError(name)


@pytest.mark.parametrize("name", ["ring8", "random8", "aim", "open3x4", "square4x4", "square3x6"])
def test_csr_bitexact(hub, name):
    """H_up and H_dn (Sec. IV.A, Eqs. 9-10): row pointers, columns and values equal the
    oracle's, read off its two-spin Hamiltonian, bit for bit; nnz = 2B C(M-2, N-1)."""
    w = _csr_case(name)
    m = _gpu_model(hub, w)
    om = oracle_model(w)
    try:
        for spin, N in ((0, w["n_up"]), (1, w["n_dn"])):
            # the spin-sigma block of sector (N, 0) / (0, N) is H_sigma by Eq. 11
            sec = (N, 0) if spin == 0 else (0, N)
            B = O.basis(w["M"], *sec)
            _, rp, cols, vals = O.spin_csr(om, sec[0], sec[1], "up" if spin == 0 else "dn", B)
            grp, gcols, gvals = m.csr(spin)
            assert np.array_equal(grp.astype(np.int64), rp)
            assert np.array_equal(gcols.astype(np.int64), cols)
            assert np.array_equal(gvals, vals)
            assert rp[-1] == (O.nnz_spin(w["M"], N, len(w["bonds"])) if 0 < N < w["M"] else 0)
    finally:
        m.close()


def test_csr_from_full_sector_matches(hub):
    """The per-spin extraction from the full sector equals the one from (N, 0): the
    Kronecker structure of Eq. 11 checked in the oracle itself, used above."""
    w = _random_workload(7, 3, 2, 5)
    om = oracle_model(w)
    full_up = O.spin_csr(om, 3, 2, "up")
    only_up = O.spin_csr(om, 3, 0, "up")
    full_dn = O.spin_csr(om, 3, 2, "dn")
    only_dn = O.spin_csr(om, 0, 2, "dn")
    for a, b in zip(full_up[1:], only_up[1:]):
        assert np.array_equal(a, b)
    for a, b in zip(full_dn[1:], only_dn[1:]):
        assert np.array_equal(a, b)


# ------------------------------------------------------------------------- apply (FP64)

APPLY_CASES = [
    ("tiny", dict(M=3, n_up=2, n_dn=1, seed=0)),
    ("random8", dict(M=8, n_up=3, n_dn=5, seed=1)),
    ("random10", dict(M=10, n_up=5, n_dn=4, seed=2)),          # 252 x 210: ragged rows
    ("random11_uniform", dict(M=11, n_up=5, n_dn=6, seed=3, uniform=True)),
    ("full_up", dict(M=6, n_up=6, n_dn=2, seed=4)),
    ("empty_dn", dict(M=7, n_up=3, n_dn=0, seed=5)),
    ("one_state", dict(M=4, n_up=4, n_dn=0, seed=6)),
]


@pytest.mark.parametrize("name,kw", APPLY_CASES, ids=[c[0] for c in APPLY_CASES])
def test_apply_entrywise(hub, name, kw):
    w = _random_workload(kw["M"], kw["n_up"], kw["n_dn"], kw["seed"], uniform=kw.get("uniform", False))
    m = _gpu_model(hub, w)
    om = oracle_model(w)
    try:
        B = O.basis(w["M"], w["n_up"], w["n_dn"])
        x = W.normal(kw["seed"] + 7, B.shape[0])
        y = m.apply(torch.from_numpy(x).cuda()).cpu().numpy()
        assert_entrywise(y, O.apply(om, B, x), abs_bound(om, B, x))
    finally:
        m.close()


@pytest.mark.parametrize("name", ["ring8", "open3x4", "aim"])
def test_apply_workloads(hub, name):
    """The benchmark-shaped workloads (ring, disordered 3x4 at full size, AIM sector)."""
    w = _csr_case(name)
    m = _gpu_model(hub, w)
    om = oracle_model(w)
    try:
        B = O.basis(w["M"], w["n_up"], w["n_dn"])
        x = W.normal(3, B.shape[0])
        y = m.apply(torch.from_numpy(x).cuda()).cpu().numpy()
        assert_entrywise(y, O.apply(om, B, x), abs_bound(om, B, x))
    finally:
        m.close()


def test_apply_rows_larger_than_shared_memory(hub):
    """count_up = C(18, 9) = 48620: a row of X (389 KB) does not fit in shared memory."""
    w = dict(W.square3x6(4.0), n_up=9, n_dn=1)
    w["eps"] = W.uniform(4, 18, -0.5, 0.5)
    m = _gpu_model(hub, w)
    om = oracle_model(w)
    try:
        B = O.basis(18, 9, 1)
        x = W.normal(8, B.shape[0])
        y = m.apply(torch.from_numpy(x).cuda()).cpu().numpy()
        assert_entrywise(y, O.apply(om, B, x), abs_bound(om, B, x))
    finally:
        m.close()


@pytest.mark.slow
def test_apply_4x4_full_size_sampled(hub):
    """4x4 PBC, (8, 8), D = 165,636,900: the full-size apply, checked against the oracle's
    two-spin rows on sampled ranges (first, last and interior rows)."""
    w = W.square4x4(4.0)
    m = _gpu_model(hub, w)
    om = oracle_model(w)
    try:
        B = O.basis(16, 8, 8)
        x = W.normal(11, B.shape[0])
        y = m.apply(torch.from_numpy(x).cuda()).cpu().numpy()
        D = B.shape[0]
        for r0 in (0, D // 3 + 17, D // 2, D - 3000):
            rows = (r0, min(D, r0 + 3000))
            assert_entrywise(y[rows[0]:rows[1]], O.apply(om, B, x, rows=rows), abs_bound(om, B, x, rows=rows))
    finally:
        m.close()


@pytest.mark.slow
def test_apply_3x6_full_size_rank_one(hub):
    """3x6 PBC, (9, 9), D = 2,363,904,400 (flat indices beyond 2^31): for a product state
    x[d, u] = a[d] b[u], Eq. 11 gives y = a (H_up b)^T + (H_dn a) b^T + diag o x; H_up, H_dn
    and the diagonal come from the oracle's two-spin sectors (9, 0) and (0, 9)."""
    w = W.square3x6(4.0)
    n = math.comb(18, 9)
    m = _gpu_model(hub, w)
    om = oracle_model(w)
    try:
        a = W.normal(21, n)
        b = W.normal(22, n)
        ad = torch.from_numpy(a).cuda()
        bd = torch.from_numpy(b).cuda()
        x = torch.outer(ad, bd).reshape(-1)
        y = m.apply(x)
        del x
        Bu = O.basis(18, 9, 0)
        Hb = O.apply(O.Model(18, w["bonds"], w["t"], 0.0), Bu, b)      # H_up b (no diagonal: U, eps = 0)
        Ha = O.apply(O.Model(18, w["bonds"], w["t"], 0.0), Bu, a)      # H_dn = H_up for N_up = N_dn
        Hb_abs = O.apply(O.Model(18, w["bonds"], w["t"], 0.0), Bu, b, absolute=True)
        Ha_abs = O.apply(O.Model(18, w["bonds"], w["t"], 0.0), Bu, a, absolute=True)
        rng_d = np.unique(np.concatenate([[0, 1, n - 1, n // 2], (W.uniform(23, 40) * n).astype(np.int64)]))
        up_bits = O.spin_parts(18, Bu)[0]
        for d in rng_d:
            yrow = y[d * n:(d + 1) * n].cpu().numpy()
            pc = np.array([bin(int(v)).count("1") for v in (up_bits & up_bits[d])], dtype=np.float64)
            ref = a[d] * Hb + Ha[d] * b + 4.0 * pc * a[d] * b
            bound = np.abs(a[d]) * Hb_abs + Ha_abs[d] * np.abs(b) + 4.0 * pc * np.abs(a[d] * b)
            assert_entrywise(yrow, ref, bound)
    finally:
        m.close()
        torch.cuda.empty_cache()


def test_apply_hermitian(hub):
    """<a, H b> = <H a, b> on the GPU (a global property, any size)."""
    w = dict(W.disordered3x4(), n_up=5, n_dn=7)
    m = _gpu_model(hub, w)
    try:
        a = torch.from_numpy(W.normal(1, m.D)).cuda()
        b = torch.from_numpy(W.normal(2, m.D)).cuda()
        lhs = torch.dot(a, m.apply(b)).item()
        rhs = torch.dot(m.apply(a), b).item()
        assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    finally:
        m.close()


# ----------------------------------------------------------------------------- Lanczos

def test_lanczos_ring8(hub):
    """Ring M = 8, (4, 4), U = 4: GPU Lanczos E0 and psi against the oracle's, same x0."""
    w = W.ring8()
    m = _gpu_model(hub, w)
    om = oracle_model(w)
    try:
        B = O.basis(8, 4, 4)
        x0 = W.normal(0, B.shape[0])
        r = m.ground(torch.from_numpy(x0).cuda(), maxit=300, tol=1e-12, want_psi=True)
        ro = O.lanczos(om, B, x0, maxit=300, tol=1e-12, want_psi=True)
        assert r["status"] == 0 and ro["converged"]
        assert abs(r["E0"] - ro["E0"]) <= 1e-10 * abs(ro["E0"])
        psi = r["psi"].cpu().numpy()
        assert abs(np.linalg.norm(psi) - 1.0) < 1e-12
        assert 1.0 - abs(psi @ ro["psi"]) < 1e-9
        w0 = np.linalg.eigvalsh(np.column_stack([O.apply(om, B, e) for e in np.eye(B.shape[0])]))[0]
        assert abs(r["E0"] - w0) <= 1e-10 * abs(w0)
    finally:
        m.close()


@pytest.mark.parametrize("case", ["random9", "aim_sector", "dim1", "null_start"])
def test_lanczos_cases(hub, case):
    if case == "random9":
        w = _random_workload(9, 4, 3, 12)
    elif case == "aim_sector":
        w = dict(W.aim_star(5), n_up=3, n_dn=4)
    elif case == "dim1":
        w = _random_workload(5, 5, 0, 13)          # one state: breakdown at the first step
    else:
        w = _random_workload(8, 4, 3, 14)
    m = _gpu_model(hub, w)
    om = oracle_model(w)
    try:
        B = O.basis(w["M"], w["n_up"], w["n_dn"])
        Hd = np.column_stack([O.apply(om, B, e) for e in np.eye(B.shape[0])])
        w0 = np.linalg.eigvalsh(Hd)[0]
        x0 = None if case == "null_start" else torch.from_numpy(W.normal(9, B.shape[0])).cuda()
        r = m.ground(x0, maxit=600, tol=1e-13)
        assert r["status"] in (0, 1)
        assert abs(r["E0"] - w0) <= 1e-10 * max(1.0, abs(w0))
        if case == "dim1":
            assert r["status"] == 1 and r["iters"] == 1
    finally:
        m.close()


@pytest.mark.slow
@pytest.mark.parametrize("M", [14, 16])
def test_lanczos_table4(hub, M):
    """Table IV (Sec. V): 1D ring, U = 4, t = 1, half filling: E0(M=14) = -8.0883491038,
    E0(M=16) = -9.2144309716 (the paper's plain Lanczos; printed to 10 decimals)."""
    from conftest import golden
    ref = {int(r[0]): float(r[2]) for r in golden("table4_E0.txt")}[M]
    w = dict(M=M, n_up=M // 2, n_dn=M // 2, bonds=W.ring_bonds(M), t=np.ones(M), U=np.full(M, 4.0))
    m = _gpu_model(hub, w)
    try:
        r = m.ground(torch.from_numpy(W.normal(0, m.D)).cuda(), maxit=400, tol=1e-12)
        assert r["status"] == 0
        assert abs(r["E0"] - ref) < 5e-10
    finally:
        m.close()
        torch.cuda.empty_cache()


# --------------------------------------------------------------------- gradients and VJP

def test_grad_parity_open3x4(hub):
    """Hellmann-Feynman gradients at the disordered 3x4 open lattice (D = 853,776): the
    kernel's quadratic forms on the GPU ground state equal the oracle's on the same psi,
    and Euler's relation sum theta dE/dtheta = E0 holds."""
    w = dict(W.disordered3x4(), n_up=6, n_dn=6)
    m = _gpu_model(hub, w)
    om = oracle_model(w)
    try:
        r = m.ground(torch.from_numpy(W.normal(0, m.D)).cuda(), maxit=400, tol=1e-13, want_psi=True)
        psi = r["psi"]
        dt, dU, de = m.grad(psi)
        B = O.basis(12, 6, 6)
        rt, rU, re = O.quadratic_forms(om, B, psi.cpu().numpy())
        scale = 1.0
        np.testing.assert_allclose(dt, rt, rtol=0, atol=1e-12 * scale)
        np.testing.assert_allclose(dU, rU, rtol=0, atol=1e-12 * scale)
        np.testing.assert_allclose(de, re, rtol=0, atol=1e-12 * scale)
        assert abs(om.t @ dt + om.U @ dU + om.eps @ de - r["E0"]) < 1e-9
        assert abs(de.sum() - 12.0) < 1e-10
    finally:
        m.close()


def test_grad_vs_finite_differences(hub):
    """dE0/dtheta from hub_grad against central finite differences of GPU Lanczos energies
    (h = 1e-4) on a disordered cluster small enough for tight convergence."""
    w = _random_workload(8, 3, 4, 21, long_range=False)
    m = _gpu_model(hub, w)
    try:
        x0 = torch.from_numpy(W.normal(1, m.D)).cuda()
        r = m.ground(x0, maxit=800, tol=1e-14, want_psi=True)
        dt, dU, de = m.grad(r["psi"])
        h = 1e-4

        def E(t, U, eps):
            m.set_params(t, U, eps)
            return m.ground(x0, maxit=800, tol=1e-14)["E0"]

        for k in range(len(w["t"])):
            tp, tm = w["t"].copy(), w["t"].copy()
            tp[k] += h
            tm[k] -= h
            fd = (E(tp, w["U"], w["eps"]) - E(tm, w["U"], w["eps"])) / (2 * h)
            assert abs(fd - dt[k]) < 1e-6
        for i in (0, 3, 7):
            Up, Um = w["U"].copy(), w["U"].copy()
            Up[i] += h
            Um[i] -= h
            assert abs((E(w["t"], Up, w["eps"]) - E(w["t"], Um, w["eps"])) / (2 * h) - dU[i]) < 1e-6
            ep, em = w["eps"].copy(), w["eps"].copy()
            ep[i] += h
            em[i] -= h
            assert abs((E(w["t"], w["U"], ep) - E(w["t"], w["U"], em)) / (2 * h) - de[i]) < 1e-6
    finally:
        m.close()


@pytest.mark.parametrize("seed", [0, 1])
def test_vjp_parity(hub, seed):
    """xbar = H ybar and ybar^T (dH/dtheta) x against the oracle (bilinear forms by
    polarisation of the oracle's quadratic forms)."""
    w = _random_workload(9, 4, 5, 30 + seed)
    m = _gpu_model(hub, w)
    om = oracle_model(w)
    try:
        B = O.basis(9, 4, 5)
        x, yb = W.normal(40 + seed, m.D), W.normal(50 + seed, m.D)
        xbar, dt, dU, de = m.vjp(torch.from_numpy(yb).cuda(), torch.from_numpy(x).cuda())
        assert_entrywise(xbar.cpu().numpy(), O.apply(om, B, yb), abs_bound(om, B, yb))
        rt, rU, re = O.bilinear_forms(om, B, yb, x)
        tol = 1e-12 * np.sqrt(m.D)
        np.testing.assert_allclose(dt, rt, rtol=0, atol=tol)
        np.testing.assert_allclose(dU, rU, rtol=0, atol=tol)
        np.testing.assert_allclose(de, re, rtol=0, atol=tol)
    finally:
        m.close()


# ---------------------------------------------------------------------- error behaviour

def test_error_codes(hub):
    h = hub.hub_basis(6, 3, 3)
    try:
        x = torch.zeros(400, dtype=torch.float64, device="cuda")
        y = torch.zeros(400, dtype=torch.float64, device="cuda")
        with pytest.raises(hub.HubError) as e:
            hub.hub_apply(h, x, y)
        assert e.value.code == hub.HUB_ERR_STATE
        with pytest.raises(hub.HubError) as e:
            hub.hub_hopping(h, [[0, 1], [1, 0]], [1.0, 1.0])
        assert e.value.code == hub.HUB_ERR_ARG
        with pytest.raises(hub.HubError) as e:
            hub.hub_hopping(h, [[0, 6]], [1.0])
        assert e.value.code == hub.HUB_ERR_ARG
        with pytest.raises(hub.HubError) as e:
            hub.hub_hopping(h, [[2, 2]], [1.0])
        assert e.value.code == hub.HUB_ERR_ARG
        hub.hub_hopping(h, W.ring_bonds(6), np.ones(6))
        hub.hub_set_U(h, [4.0])
        with pytest.raises(hub.HubError) as e:
            hub.hub_apply(h, x, x)
        assert e.value.code == hub.HUB_ERR_ARG
        with pytest.raises(hub.HubError) as e:
            hub.hub_set_U(h, [1.0, 2.0])
        assert e.value.code == hub.HUB_ERR_ARG
    finally:
        hub.hub_free(h)
    for bad in [(0, 0, 0), (31, 1, 1), (4, 5, 0), (4, -1, 0)]:
        with pytest.raises(hub.HubError) as e:
            hub.hub_basis(*bad)
        assert e.value.code == hub.HUB_ERR_ARG


def test_apply_host_buffers(hub):
    w = W.ring8()
    m = _gpu_model(hub, w)
    try:
        x = W.normal(3, m.D)
        y = np.empty_like(x)
        hub.hub_apply_host(m.h, x, y)
        yd = m.apply(torch.from_numpy(x).cuda()).cpu().numpy()
        assert np.array_equal(y, yd)
    finally:
        m.close()


@pytest.mark.parametrize("case", ["max_in_first_chunk", "max_in_last_chunk", "odd_rows"])
def test_apply_host_pipelined(hub, case):
    """hub_apply_host on the fast path overlaps the copies with the passes in row chunks, with
    the conversion scale taken from the first chunk and redone when a later chunk holds a
    larger exponent: the result equals hub_apply bit for bit and the oracle within the
    per-entry bound (pinned host buffers)."""
    if case == "odd_rows":
        M, nu, nd = 11, 5, 3                       # count_dn = C(11, 3) = 165 rows: odd tail pair
    else:
        M, nu, nd = 12, 6, 6                       # 924 x 924
    bonds = W.ring_bonds(M)
    m = hub.Hubbard(M, nu, nd, bonds, 1.0, 4.0)
    om = O.Model(M, bonds, 1.0, 4.0)
    try:
        x = W.normal(17, m.D)
        n_up = m.count_up
        if case == "max_in_first_chunk":
            x[: 2 * n_up] *= 64.0
        elif case == "max_in_last_chunk":
            x[-2 * n_up:] *= 1e6
        xh = torch.from_numpy(x).pin_memory()
        yh = torch.empty_like(xh).pin_memory()
        hub.hub_apply_host(m.h, xh, yh)
        yd = m.apply(torch.from_numpy(x).cuda()).cpu().numpy()
        assert np.array_equal(yh.numpy(), yd)
        B = O.basis(M, nu, nd)
        assert_entrywise(yh.numpy(), O.apply(om, B, x), abs_bound(om, B, x))
    finally:
        m.close()


def _singles(hub, m, X):
    """One hub_apply_host call per row of X (pinned buffers)."""
    out = []
    for v in range(X.shape[0]):
        xh = torch.from_numpy(np.ascontiguousarray(X[v])).pin_memory()
        yh = torch.empty_like(xh).pin_memory()
        hub.hub_apply_host(m.h, xh, yh)
        out.append(yh.numpy().copy())
    return np.stack(out)


def test_apply_host_many_pipelined(hub):
    """hub_apply_host_many on the fast path, 12-site ring (6, 6), 924 rows: five vectors in one
    call (both buffer pairs used twice; one vector whose largest exponent is in its last row
    chunk, one outside the double-float window, routed to the FP64 kernel) equal one
    hub_apply_host call per vector bit for bit, also in place; the first equals the oracle
    within the per-entry bound."""
    M, nu, nd = 12, 6, 6
    bonds = W.ring_bonds(M)
    m = hub.Hubbard(M, nu, nd, bonds, 1.0, 4.0)
    om = O.Model(M, bonds, 1.0, 4.0)
    try:
        D, n_up = m.D, m.count_up
        X = np.stack([W.normal(30 + v, D) for v in range(5)])
        X[1, -2 * n_up:] *= 1e6                     # largest exponent in the last input chunk
        X[2, D // 3] = 1e280                        # above the window's largest |x|: FP64 kernel
        xh = torch.from_numpy(X).pin_memory()
        yh = torch.empty_like(xh).pin_memory()
        hub.hub_apply_host_many(m.h, 5, xh, yh)
        ref = _singles(hub, m, X)
        for v in range(5):
            assert np.array_equal(yh[v].numpy(), ref[v]), v
        B = O.basis(M, nu, nd)
        assert_entrywise(yh[0].numpy(), O.apply(om, B, X[0]), abs_bound(om, B, X[0]))
        # in place: the results overwrite the inputs
        zh = xh.clone().pin_memory()
        hub.hub_apply_host_many(m.h, 5, zh, zh)
        assert torch.equal(zh, yh)
        # two vectors, then three: buffers of an earlier call reused
        hub.hub_apply_host_many(m.h, 2, xh[3:], yh[3:])
        assert np.array_equal(yh[3:].numpy(), ref[3:])
    finally:
        m.close()


def test_apply_host_many_other_paths_and_arguments(hub):
    """Off the pipelined path (FP64 model; a sector with fewer than 16 rows) the call is one
    hub_apply_host per vector: the same results bit for bit.  n_vec = 0 leaves y untouched;
    a negative count, NULL arrays and partly overlapping arrays are refused."""
    w = _random_workload(9, 4, 3, 61)
    m = _gpu_model(hub, w)
    try:
        X = np.stack([W.normal(40 + v, m.D) for v in range(3)])
        Y = np.empty_like(X)
        hub.hub_apply_host_many(m.h, 3, X, Y)
        assert np.array_equal(Y, _singles(hub, m, X))
        Y0 = Y.copy()
        hub.hub_apply_host_many(m.h, 0, X, Y)
        assert np.array_equal(Y, Y0)
        for args in [(-1, X, Y), (2, None, Y), (2, X, None)]:
            with pytest.raises(hub.HubError) as e:
                hub.hub_apply_host_many(m.h, *args)
            assert e.value.code == hub.HUB_ERR_ARG
        flat = np.zeros(4 * m.D)
        with pytest.raises(hub.HubError) as e:
            hub.hub_apply_host_many(m.h, 2, flat[: 2 * m.D], flat[m.D:])
        assert e.value.code == hub.HUB_ERR_ARG
    finally:
        m.close()
    m = hub.Hubbard(5, 2, 2, W.ring_bonds(5), 1.0, 4.0)      # C(5, 2) = 10 rows: one piece
    try:
        X = np.stack([W.normal(50 + v, m.D) for v in range(3)])
        Y = np.empty_like(X)
        hub.hub_apply_host_many(m.h, 3, X, Y)
        assert np.array_equal(Y, _singles(hub, m, X))
    finally:
        m.close()


# --------------------------------------------------------------------------- autograd

def test_autograd_apply(hub):
    """ApplyFn backward (the library's VJP) against finite differences of <g, H(theta) x>."""
    w = _random_workload(7, 3, 3, 60)
    m = _gpu_model(hub, w)
    try:
        x = torch.from_numpy(W.normal(61, m.D)).cuda().requires_grad_(True)
        g = torch.from_numpy(W.normal(62, m.D)).cuda()
        t = torch.tensor(w["t"], requires_grad=True)
        U = torch.tensor(w["U"], requires_grad=True)
        e = torch.tensor(w["eps"], requires_grad=True)
        y = hub.apply_fn(m, x, t, U, e)
        (y * g).sum().backward()
        h = 1e-6
        for k in range(3):
            tp, tm = w["t"].copy(), w["t"].copy()
            tp[k] += h
            tm[k] -= h
            fp = (hub.apply_fn(m, x.detach(), torch.tensor(tp), U.detach(), e.detach()) * g).sum().item()
            fm = (hub.apply_fn(m, x.detach(), torch.tensor(tm), U.detach(), e.detach()) * g).sum().item()
            assert abs((fp - fm) / (2 * h) - t.grad[k].item()) < 1e-6 * max(1.0, abs(t.grad[k].item()))
        # x-gradient: H g
        m.set_params(w["t"], w["U"], w["eps"])
        assert torch.allclose(x.grad, m.apply(g), rtol=0, atol=1e-12)
    finally:
        m.close()


def test_autograd_ground_energy(hub):
    w = _random_workload(8, 4, 4, 70, long_range=False)
    m = _gpu_model(hub, w)
    try:
        t = torch.tensor(w["t"], requires_grad=True)
        U = torch.tensor(w["U"], requires_grad=True)
        e = torch.tensor(w["eps"], requires_grad=True)
        E = hub.ground_energy(m, t, U, e, x0=torch.from_numpy(W.normal(1, m.D)).cuda(), tol=1e-13)
        E.backward()
        total = (t.detach() * t.grad).sum() + (U.detach() * U.grad).sum() + (e.detach() * e.grad).sum()
        assert abs(total.item() - E.item()) < 1e-9
    finally:
        m.close()


# -------------------------------------------------------------------------- fast path

FAST_CASES = [
    ("ring8", dict(M=8, n_up=4, n_dn=4)),                     # shared CSR, even rows
    ("odd_rows", dict(M=7, n_up=3, n_dn=2)),                  # count_up = 35: padded rows
    ("unequal", dict(M=10, n_up=3, n_dn=6)),
    ("with_eps", dict(M=9, n_up=4, n_dn=5, eps=True)),
    ("t_not_one", dict(M=9, n_up=5, n_dn=4, t=0.37)),
]


@pytest.mark.parametrize("name,kw", FAST_CASES, ids=[c[0] for c in FAST_CASES])
def test_fast_and_fp64_modes(hub, name, kw):
    """Uniform t and U select the double-float two-pass apply; HUB_MODE_FP64 the FP64
    kernel.  Both agree with the oracle entry by entry (1e-13 |H||x|)."""
    M = kw["M"]
    bonds = W.ring_bonds(M) if name != "unequal" else np.concatenate([W.ring_bonds(M), [[0, 5], [2, 7]]])
    w = dict(M=M, n_up=kw["n_up"], n_dn=kw["n_dn"], bonds=bonds, t=np.full(len(bonds), kw.get("t", 1.0)),
             U=np.full(M, 3.0), eps=W.uniform(5, M, -0.5, 0.5) if kw.get("eps") else np.zeros(M))
    m = _gpu_model(hub, w)
    om = oracle_model(w)
    try:
        B = O.basis(M, w["n_up"], w["n_dn"])
        x = W.normal(17, B.shape[0])
        ref, bound = O.apply(om, B, x), abs_bound(om, B, x)
        xd = torch.from_numpy(x).cuda()
        y_fast = m.apply(xd).cpu().numpy()
        hub.hub_set_mode(m.h, hub.HUB_MODE_FP64)
        y_f64 = m.apply(xd).cpu().numpy()
        hub.hub_set_mode(m.h, hub.HUB_MODE_AUTO)
        assert_entrywise(y_fast, ref, bound)
        assert_entrywise(y_f64, ref, bound)
        hub.hub_check(m.h)
    finally:
        m.close()


def test_fast_wide_dynamic_range(hub):
    """Entries spanning 1e-18 .. 1e2 (and exact zeros): the per-entry bound still holds."""
    w = W.ring8()
    m = _gpu_model(hub, w)
    om = oracle_model(w)
    try:
        B = O.basis(8, 4, 4)
        x = W.normal(3, B.shape[0]) * 10.0 ** W.uniform(4, B.shape[0], -18, 2)
        x[::17] = 0.0
        y = m.apply(torch.from_numpy(x).cuda()).cpu().numpy()
        assert_entrywise(y, O.apply(om, B, x), abs_bound(om, B, x))
        for scale in (1e-200, 1e250):
            ys = m.apply(torch.from_numpy(x * scale).cuda()).cpu().numpy()
            assert_entrywise(ys, O.apply(om, B, x * scale), abs_bound(om, B, x * scale))
    finally:
        m.close()


def test_fast_lanczos_matches_fp64_lanczos(hub):
    """The double-float Lanczos and the FP64 Lanczos reach the same E0 (1e-10 relative)
    and the same psi, on a sector with unequal spins."""
    w = dict(M=10, n_up=4, n_dn=5, bonds=W.ring_bonds(10), t=np.ones(10), U=np.full(10, 4.0), eps=np.zeros(10))
    m = _gpu_model(hub, w)
    hub.hub_set_small_dim(m.h, 0)          # the multi-kernel drivers, not the small-sector solver
    try:
        x0 = torch.from_numpy(W.normal(2, m.D)).cuda()
        r1 = m.ground(x0, maxit=400, tol=1e-13, want_psi=True)
        hub.hub_set_mode(m.h, hub.HUB_MODE_FP64)
        r2 = m.ground(x0, maxit=400, tol=1e-13, want_psi=True)
        assert abs(r1["E0"] - r2["E0"]) <= 1e-10 * abs(r2["E0"])
        assert 1.0 - abs(torch.dot(r1["psi"], r2["psi"]).item()) < 1e-9
    finally:
        m.close()


# -------------------------------------------- Sec. IX complement and Sec. X shared tables

@pytest.mark.parametrize("M,nu", [(8, 3), (10, 4), (9, 5), (16, 7)])
def test_half_filling_complement(hub, M, nu):
    """Sec. IX: in a half-filled sector (N_up + N_dn = M) the basis of one spin is the other's
    bitwise complement in reversed order; the GPU bases satisfy it bit for bit."""
    m = hub.Hubbard(M, nu, M - nu, W.ring_bonds(M), 1.0, 4.0)
    up, dn = m.basis(0).astype(np.int64), m.basis(1).astype(np.int64)
    assert np.array_equal(dn, (~up[::-1]) & ((1 << M) - 1))
    m.close()


@pytest.mark.parametrize("M,n", [(8, 4), (12, 6), (9, 3)])
def test_equal_spin_counts_share_tables(hub, M, n):
    """Sec. X: for N_up = N_dn the spin-up and spin-down hopping matrices are identical (the
    library keeps one copy); both spins' CSR read back equal."""
    m = hub.Hubbard(M, n, n, W.ring_bonds(M), 1.0, 4.0)
    a, b = m.csr(0), m.csr(1)
    for x, y in zip(a, b):
        assert np.array_equal(np.asarray(x), np.asarray(y))
    m.close()


# ---------------------------------------- 32-bit column tables (a spin count above 65536)

@pytest.mark.parametrize("nu,nd", [pytest.param(2, 10, marks=pytest.mark.slow), (10, 1)])
def test_apply_wide_sectors(hub, nu, nd):
    """M = 20 with C(20, 10) = 184,756 states of one spin, more than 16-bit column indices
    hold: (2, 10) runs pass 1 on staged rows of 190 columns with 32-bit schedule words and
    pass 2 with 32-bit strip rows; (10, 1) runs pass 1 on the transposed matrix (rows of
    184,756 columns do not fit in shared memory).  Sampled rows against the oracle (whose
    two-spin basis scan makes the first case slow)."""
    M = 20
    bonds = np.array([tuple(b) for b in W.ring_bonds(M).tolist()] + [(0, 10), (3, 17), (5, 12)], dtype=np.int32)
    m = hub.Hubbard(M, nu, nd, bonds, 1.0, 3.0)
    om = O.Model(M, bonds, 1.0, 3.0)
    try:
        B = O.basis(M, nu, nd)
        x = W.normal(23, B.shape[0])
        y = m.apply(torch.from_numpy(x).cuda()).cpu().numpy()
        D = B.shape[0]
        for r0 in (0, D // 2 + 5, D - 2000):
            rows = (r0, min(D, r0 + 2000))
            assert_entrywise(y[rows[0]:rows[1]], O.apply(om, B, x, rows=rows), abs_bound(om, B, x, rows=rows))
        if D < 5_000_000:
            # and a short Lanczos run agrees with the oracle's on the same start vector
            r = m.ground(torch.from_numpy(x).cuda(), maxit=12, tol=0.0)
            ro = O.lanczos(om, B, x, maxit=12, fixed_iters=True)
            assert abs(r["E0"] - ro["E0"]) < 1e-10 * abs(ro["E0"])
    finally:
        m.close()


def test_lanczos_graph_replay_matches_direct_launches(hub):
    """The fast Lanczos replays each iteration as a captured CUDA graph unless profiling is on;
    both give bit-identical alpha and beta, the cached graphs are reused for a second run and
    recaptured after new parameters (U), matching a fresh handle with those parameters."""
    M = 8
    bonds = W.ring_bonds(M)
    m = hub.Hubbard(M, 4, 4, bonds, 1.0, 4.0)
    hub.hub_set_small_dim(m.h, 0)          # the multi-kernel driver, not the small-sector solver
    x0 = torch.from_numpy(W.normal(0, m.D)).cuda()
    runs = []
    for prof in (False, False, True):
        hub.hub_profile(m.h, prof)
        r = m.ground(x0, maxit=40, tol=0.0)
        runs.append((r["E0"],) + tuple(np.array(c) for c in hub.hub_lanczos_coeffs(m.h)))
    hub.hub_profile(m.h, False)
    for k in (1, 2):
        assert runs[k][0] == runs[0][0]
        assert np.array_equal(runs[k][1], runs[0][1]) and np.array_equal(runs[k][2], runs[0][2])
    m.set_params(1.0, 6.0)
    e6 = m.ground(x0, maxit=40, tol=0.0)["E0"]
    a6 = hub.hub_lanczos_coeffs(m.h)[0]
    m.close()
    fresh = hub.Hubbard(M, 4, 4, bonds, 1.0, 6.0)
    hub.hub_set_small_dim(fresh.h, 0)
    hub.hub_profile(fresh.h, True)
    ef = fresh.ground(x0, maxit=40, tol=0.0)["E0"]
    af = hub.hub_lanczos_coeffs(fresh.h)[0]
    fresh.close()
    assert e6 == ef and np.array_equal(a6, af)
