"""Thin Python binding of the C ABI in ``include/hub.h`` (argument marshalling only).

Every function named ``hub_*`` here calls the C entry point of the same name in
``_build/libhub.so``; all arithmetic runs in the CUDA kernels of that library.  There
is no CPU fallback: if the library cannot be loaded, every call raises.

``Hubbard`` wraps one handle (a sector of a lattice model) and takes torch tensors on
the GPU for vectors.  ``ApplyFn`` and ``GroundEnergyFn`` are torch.autograd.Functions
whose backward passes are the library's adjoint kernels (``hub_apply_vjp``, ``hub_grad``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libhub.so")

HUB_OK = 0
HUB_CONVERGED_BREAKDOWN = 1
HUB_ERR_ARG = -1
HUB_ERR_OOM = -2
HUB_ERR_CUDA = -3
HUB_ERR_NOCONV = -4
HUB_ERR_STATE = -5
HUB_ERR_TIMEOUT = -6
HUB_SYM_NONE = 0
HUB_SYM_K0 = 1
HUB_SYM_KPI = 2
HUB_SPIN_UP = 0
HUB_SPIN_DN = 1

# (name, restype, argtypes) of every exported entry point.
_i, _i64, _d, _p = ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
SIGNATURES = {
    "hub_last_error": (ctypes.c_char_p, []),
    "hub_basis": (_i, [_i, _i, _i, ctypes.POINTER(_p)]),
    "hub_dims": (_i, [_p, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "hub_get_basis": (_i, [_p, _i, _p]),
    "hub_hopping": (_i, [_p, _i, _p, _p, _p]),
    "hub_set_U": (_i, [_p, _i, _p]),
    "hub_csr_info": (_i, [_p, _i, ctypes.POINTER(_i64), ctypes.POINTER(ctypes.c_int32)]),
    "hub_get_csr": (_i, [_p, _i, _p, _p, _p]),
    "hub_apply": (_i, [_p, _p, _p, _p]),
    "hub_apply_host": (_i, [_p, _p, _p, _p]),
    "hub_apply_host_many": (_i, [_p, _i64, _p, _p, _p]),
    "hub_lanczos_ground": (_i, [_p, _p, _i, _d, ctypes.POINTER(_d), _p, ctypes.POINTER(_i), _p]),
    "hub_lanczos_coeffs": (_i, [_p, _p, _p, _i, ctypes.POINTER(_i)]),
    "hub_lanczos_spectrum": (_i, [_p, _p, _i, _i, _p, _p, ctypes.POINTER(_i), _p]),
    "hub_lanczos_ritz": (_i, [_p, _p, _i, _d, _p, ctypes.POINTER(_d), _p]),
    "hub_lanczos_block": (_i, [_p, _i, _p, _i, _i, _p, _p, ctypes.POINTER(_i), _p]),
    "hub_ladder": (_i, [_p, _p, _i, _i, _i, _p, _p, _p]),
    "hub_green_coeffs": (_i, [_p, _p, _i, _p, _p, ctypes.POINTER(_d), ctypes.POINTER(_i), _p]),
    "hub_green_eval": (_i, [_i, _p, _p, _d, _d, _i, _i, _p, _p, _p, _p]),
    "hub_grad": (_i, [_p, _p, _p, _p, _p, _p]),
    "hub_apply_vjp": (_i, [_p, _p, _p, _p, _p, _p, _p, _p]),
    "hub_grad_noalloc": (_i, [_p, _p, _p, _p, _p, _p]),
    "hub_batch_ground": (_i, [_i, _i, _p, _i, _p, _p, _p, _i, _p, _p, _p, _i, _d, _p, _p, _p, _p]),
    "hub_set_symmetry": (_i, [_p, _i]),
    "hub_set_translations": (_i, [_p, _i, _p, _p]),
    "hub_k_dims": (_i, [_p, ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "hub_k_reps": (_i, [_p, _p, _p]),
    "hub_k_columns": (_i, [_p, _p, _p]),
    "hub_k_project": (_i, [_p, _p, _p, _p]),
    "hub_set_mode": (_i, [_p, _i]),
    "hub_check": (_i, [_p]),
    "hub_test_fail_waits": (_i, [_p, _i]),
    "hub_profile": (_i, [_p, _i]),
    "hub_profile_read": (_i, [_p, _i, ctypes.POINTER(_d), ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "hub_free": (None, [_p]),
    "hub_set_small_dim": (_i, [_p, _i64]),
}

_lib = None


class HubError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


def lib():
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                               "(run __graft_entry__.build() or python -m paper_1307_7542_gb300.build)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc, ok=(HUB_OK,)):
    if rc not in ok:
        raise HubError(rc, lib().hub_last_error().decode())
    return rc


def _ptr(t):
    """Device or host address of a contiguous torch tensor / numpy array (None -> NULL)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        assert t.flags["C_CONTIGUOUS"]
        return ctypes.c_void_p(t.ctypes.data)
    assert t.is_contiguous()
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


# ------------------------------------------------------------------------ raw C ABI calls

def hub_basis(M, n_up, n_dn):
    h = ctypes.c_void_p()
    _check(lib().hub_basis(M, n_up, n_dn, ctypes.byref(h)))
    return h


def hub_dims(h):
    a, b = _i64(), _i64()
    _check(lib().hub_dims(h, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def hub_get_basis(h, spin, n):
    out = np.empty(n, dtype=np.uint32)
    _check(lib().hub_get_basis(h, spin, _ptr(out)))
    return out


def hub_hopping(h, bonds, t, eps=None):
    bonds = np.ascontiguousarray(np.asarray(bonds, dtype=np.int32).reshape(-1, 2))
    t = np.ascontiguousarray(np.asarray(t, dtype=np.float64).reshape(-1))
    e = None if eps is None else np.ascontiguousarray(np.asarray(eps, dtype=np.float64).reshape(-1))
    _check(lib().hub_hopping(h, bonds.shape[0], _ptr(bonds), _ptr(t), _ptr(e)))


def hub_set_U(h, U):
    U = np.ascontiguousarray(np.atleast_1d(np.asarray(U, dtype=np.float64)))
    _check(lib().hub_set_U(h, U.shape[0], _ptr(U)))


def hub_csr_info(h, spin):
    nnz, mx = _i64(), ctypes.c_int32()
    _check(lib().hub_csr_info(h, spin, ctypes.byref(nnz), ctypes.byref(mx)))
    return nnz.value, mx.value


def hub_get_csr(h, spin, n_rows):
    nnz, _ = hub_csr_info(h, spin)
    rp = np.empty(n_rows + 1, dtype=np.int32)
    cols = np.empty(max(nnz, 1), dtype=np.int32)
    vals = np.empty(max(nnz, 1), dtype=np.float64)
    _check(lib().hub_get_csr(h, spin, _ptr(rp), _ptr(cols), _ptr(vals)))
    return rp, cols[:nnz], vals[:nnz]


def hub_apply(h, x, y, stream=None):
    _check(lib().hub_apply(h, _ptr(x), _ptr(y), _stream(stream)))


def hub_apply_host(h, x, y, stream=None):
    _check(lib().hub_apply_host(h, _ptr(x), _ptr(y), _stream(stream)))


def hub_apply_host_many(h, n_vec, x, y, stream=None):
    """x, y: host arrays holding n_vec vectors one after another (e.g. shape (n_vec, D))."""
    _check(lib().hub_apply_host_many(h, n_vec, _ptr(x), _ptr(y), _stream(stream)))


def hub_lanczos_ground(h, x0, maxit, tol, psi=None, stream=None):
    E0, it = _d(), _i()
    rc = lib().hub_lanczos_ground(h, _ptr(x0), maxit, tol, ctypes.byref(E0), _ptr(psi),
                                  ctypes.byref(it), _stream(stream))
    _check(rc, ok=(HUB_OK, HUB_CONVERGED_BREAKDOWN, HUB_ERR_NOCONV))
    return E0.value, it.value, rc


def hub_lanczos_coeffs(h, cap=100000):
    a, b = np.empty(cap), np.empty(cap)
    n = _i()
    _check(lib().hub_lanczos_coeffs(h, _ptr(a), _ptr(b), cap, ctypes.byref(n)))
    return a[: n.value], b[: n.value]


def hub_grad(h, psi, n_bonds, M, stream=None):
    dt, dU, de = np.empty(n_bonds), np.empty(M), np.empty(M)
    _check(lib().hub_grad(h, _ptr(psi), _ptr(dt), _ptr(dU), _ptr(de), _stream(stream)))
    return dt, dU, de


def hub_lanczos_spectrum(h, x0, maxit, n_eig, stream=None):
    """Lowest n_eig distinct Ritz values (Cullum-Willoughby filtered) and their residual estimates."""
    e, r = np.empty(n_eig), np.empty(n_eig)
    n = _i()
    _check(lib().hub_lanczos_spectrum(h, _ptr(x0), maxit, n_eig, _ptr(e), _ptr(r), ctypes.byref(n),
                                      _stream(stream)))
    return e[: n.value], r[: n.value]


def hub_lanczos_block(h, k, X0, steps, n_eig, stream=None):
    """Lowest n_eig eigenvalues with multiplicity (block Lanczos, block size k) and the
    residual norms of their Ritz vectors."""
    e, r = np.empty(n_eig), np.empty(n_eig)
    n = _i()
    _check(lib().hub_lanczos_block(h, k, _ptr(X0), steps, n_eig, _ptr(e), _ptr(r), ctypes.byref(n),
                                   _stream(stream)))
    return e[: n.value], r[: n.value]


def hub_lanczos_ritz(h, x0, maxit, target, psi, stream=None):
    """Normalised Ritz vector (into psi) for the eigenvalue of T nearest target; returns that value."""
    v = _d()
    _check(lib().hub_lanczos_ritz(h, _ptr(x0), maxit, target, _ptr(psi), ctypes.byref(v), _stream(stream)))
    return v.value


def hub_ladder(h_from, h_to, site, spin, create, x, y, stream=None):
    """y = c+_{site,spin} x (create) or c_{site,spin} x, from the sector of h_from to that of h_to."""
    _check(lib().hub_ladder(h_from, h_to, site, spin, 1 if create else 0, _ptr(x), _ptr(y), _stream(stream)))


def hub_green_coeffs(h, v, k, stream=None):
    """k Lanczos steps from v: (alpha, beta, |v|^2) of the continued fraction."""
    a, b = np.empty(k), np.empty(k)
    n2, n = _d(), _i()
    _check(lib().hub_green_coeffs(h, _ptr(v), k, _ptr(a), _ptr(b), ctypes.byref(n2), ctypes.byref(n),
                                  _stream(stream)))
    return a[: n.value], b[: n.value], n2.value


def hub_green_eval(alpha, beta, norm2, E0, sign, z):
    """Continued fraction of the particle (sign +1) or hole (sign -1) term at complex points z."""
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    b = np.ascontiguousarray(beta, dtype=np.float64)
    z = np.atleast_1d(np.asarray(z, dtype=np.complex128))
    zr, zi = np.ascontiguousarray(z.real), np.ascontiguousarray(z.imag)
    gr, gi = np.empty(z.size), np.empty(z.size)
    _check(lib().hub_green_eval(a.size, _ptr(a), _ptr(b), norm2, E0, sign, z.size, _ptr(zr), _ptr(zi),
                                _ptr(gr), _ptr(gi)))
    return gr + 1j * gi


def hub_batch_ground(M, bonds, t, U, eps, job_nup, job_ndn, job_param, maxit=300, tol=1e-12, stream=None):
    """Ground-state energies of many (sector, parameter set) jobs in one persistent launch.
    t: [n_params, n_bonds]; U, eps: [n_params, M] (eps may be None).  Returns (E0, iters, status)."""
    bonds = np.ascontiguousarray(np.asarray(bonds, dtype=np.int32).reshape(-1, 2))
    t = np.ascontiguousarray(np.asarray(t, dtype=np.float64).reshape(-1, bonds.shape[0]))
    U = np.ascontiguousarray(np.asarray(U, dtype=np.float64).reshape(t.shape[0], M))
    e = None if eps is None else np.ascontiguousarray(np.asarray(eps, dtype=np.float64).reshape(t.shape[0], M))
    jn = np.ascontiguousarray(np.asarray(job_nup, dtype=np.int32))
    jd = np.ascontiguousarray(np.asarray(job_ndn, dtype=np.int32))
    jp = np.ascontiguousarray(np.asarray(job_param, dtype=np.int32))
    n = jn.shape[0]
    E0, it, st = np.empty(n), np.empty(n, dtype=np.int32), np.empty(n, dtype=np.int32)
    rc = lib().hub_batch_ground(M, bonds.shape[0], _ptr(bonds), t.shape[0], _ptr(t), _ptr(U), _ptr(e), n,
                                _ptr(jn), _ptr(jd), _ptr(jp), maxit, tol, _ptr(E0), _ptr(it), _ptr(st),
                                _stream(stream))
    _check(rc, ok=(HUB_OK, HUB_ERR_NOCONV))
    return E0, it, st


def hub_grad_noalloc(h, psi, n_bonds, M, stream=None):
    """hub_grad with its scratch in a fixed device array (no allocation at call time)."""
    dt, dU, de = np.empty(n_bonds), np.empty(M), np.empty(M)
    _check(lib().hub_grad_noalloc(h, _ptr(psi), _ptr(dt), _ptr(dU), _ptr(de), _stream(stream)))
    return dt, dU, de


def hub_apply_vjp(h, ybar, x, xbar, n_bonds, M, want_params=True, stream=None):
    dt = np.empty(n_bonds) if want_params else None
    dU = np.empty(M) if want_params else None
    de = np.empty(M) if want_params else None
    _check(lib().hub_apply_vjp(h, _ptr(ybar), _ptr(x), _ptr(xbar), _ptr(dt), _ptr(dU), _ptr(de),
                               _stream(stream)))
    return dt, dU, de


def hub_profile(h, enable):
    _check(lib().hub_profile(h, 1 if enable else 0))


HUB_MODE_AUTO, HUB_MODE_FP64 = 0, 1
HUB_PROF_APPLY, HUB_PROF_UP, HUB_PROF_DN, HUB_PROF_UPDATE = 0, 1, 2, 3


def hub_profile_read(h, kind=HUB_PROF_APPLY):
    """(summed milliseconds, launches) of one kind, and all kernel launches, since hub_profile(h, 1)."""
    ms, na, nk = _d(), _i64(), _i64()
    _check(lib().hub_profile_read(h, kind, ctypes.byref(ms), ctypes.byref(na), ctypes.byref(nk)))
    return ms.value, na.value, nk.value


def hub_set_symmetry(h, sym):
    _check(lib().hub_set_symmetry(h, sym))


def hub_set_translations(h, perms, chars):
    perms = np.ascontiguousarray(np.asarray(perms, dtype=np.int32))
    chars = np.ascontiguousarray(np.asarray(chars, dtype=np.int32).reshape(-1))
    assert perms.ndim == 2 and perms.shape[0] == chars.shape[0]
    _check(lib().hub_set_translations(h, perms.shape[0], _ptr(perms), _ptr(chars)))


def hub_k_dims(h):
    r, c, d = _i64(), _i64(), _i64()
    _check(lib().hub_k_dims(h, ctypes.byref(r), ctypes.byref(c), ctypes.byref(d)))
    return r.value, c.value, d.value


def hub_k_reps(h, rows):
    reps = np.empty(rows, dtype=np.uint32)
    per = np.empty(rows, dtype=np.int32)
    _check(lib().hub_k_reps(h, reps.ctypes.data, per.ctypes.data))
    return reps, per


def hub_k_columns(h, cols):
    bits = np.empty(cols, dtype=np.uint32)
    sign = np.empty(cols, dtype=np.int32)
    _check(lib().hub_k_columns(h, bits.ctypes.data, sign.ctypes.data))
    return bits, sign


def hub_k_project(h, x, y, stream=None):
    _check(lib().hub_k_project(h, _ptr(x), _ptr(y), _stream(stream)))


def hub_set_mode(h, mode):
    _check(lib().hub_set_mode(h, mode))


def hub_check(h):
    _check(lib().hub_check(h))


def hub_set_small_dim(h, max_dim):
    """Largest sector hub_lanczos_ground runs as the single-launch small-sector solver (0: off)."""
    _check(lib().hub_set_small_dim(h, int(max_dim)))


def hub_test_fail_waits(h, enable):
    """Test hook: pass 1 takes its given-up-wait exit (see include/hub.h)."""
    _check(lib().hub_test_fail_waits(h, 1 if enable else 0))


def hub_free(h):
    if h:
        lib().hub_free(h)


# ------------------------------------------------------------------------- object wrapper

class Hubbard:
    """One sector (N_up, N_dn) of a lattice model on the GPU.

    Parameters follow Eq. 1: bonds (pairs of 0-based sites), per-bond t, per-site (or
    uniform) U, optional per-site eps.
    """

    def __init__(self, M, n_up, n_dn, bonds, t, U, eps=None):
        self.M, self.n_up, self.n_dn = int(M), int(n_up), int(n_dn)
        self.bonds = np.ascontiguousarray(np.asarray(bonds, dtype=np.int32).reshape(-1, 2))
        self.h = hub_basis(self.M, self.n_up, self.n_dn)
        self.count_up, self.count_dn = hub_dims(self.h)
        self.D = self.count_up * self.count_dn
        self.set_params(t, U, eps)

    def set_params(self, t, U, eps=None):
        nb = self.bonds.shape[0]
        t = np.asarray(t, dtype=np.float64)
        self.t = np.full(nb, float(t)) if t.ndim == 0 else t.reshape(nb).copy()
        U = np.asarray(U, dtype=np.float64)
        self.U = np.full(self.M, float(U)) if U.ndim == 0 else U.reshape(self.M).copy()
        self.eps = np.zeros(self.M) if eps is None else np.asarray(eps, dtype=np.float64).reshape(self.M).copy()
        hub_hopping(self.h, self.bonds, self.t, self.eps if np.any(self.eps) else None)
        hub_set_U(self.h, self.U if np.any(self.U != self.U[0]) else self.U[:1])
        self.D = self.count_up * self.count_dn      # new parameters leave the k = 0 sector

    def ensure_params(self, t, U, eps=None):
        """set_params unless (t, U, eps) equal the current parameters and the model is in its
        full sector: the hopping tables (and the captured Lanczos iterations that depend on
        them) are then kept."""
        nb = self.bonds.shape[0]
        t = np.asarray(t, dtype=np.float64)
        t = np.full(nb, float(t)) if t.ndim == 0 else t.reshape(nb)
        U = np.asarray(U, dtype=np.float64)
        U = np.full(self.M, float(U)) if U.ndim == 0 else U.reshape(self.M)
        e = np.zeros(self.M) if eps is None else np.asarray(eps, dtype=np.float64).reshape(self.M)
        same = (hasattr(self, "t") and np.array_equal(t, self.t) and np.array_equal(U, self.U)
                and np.array_equal(e, self.eps) and self.D == self.count_up * self.count_dn)
        if not same:
            self.set_params(t, U, e)
        return not same

    def set_symmetry(self, sym):
        """HUB_SYM_K0 / HUB_SYM_KPI: work in the k = 0 / k = pi sector of the translation
        i -> i-1 mod M (Sec. V); vectors are then k_rows x k_cols arrays in row form.
        HUB_SYM_NONE: the full sector."""
        hub_set_symmetry(self.h, sym)
        if sym in (HUB_SYM_K0, HUB_SYM_KPI):
            self.k_rows, self.k_cols, self.k_dim = hub_k_dims(self.h)
            self.D = self.k_rows * self.k_cols
        else:
            self.D = self.count_up * self.count_dn

    def set_translations(self, perms, chars):
        """The sector g Psi = chi(g) Psi of the group generated by the site permutations
        perms (chi = +-1 on each); vectors then in row form, k_rows x k_cols."""
        hub_set_translations(self.h, perms, chars)
        self.k_rows, self.k_cols, self.k_dim = hub_k_dims(self.h)
        self.D = self.k_rows * self.k_cols

    def k_reps(self):
        return hub_k_reps(self.h, self.k_rows)

    def k_columns(self):
        return hub_k_columns(self.h, self.k_cols)

    def k_project(self, x, y=None, stream=None):
        import torch
        if y is None:
            y = torch.empty_like(x)
        hub_k_project(self.h, x, y, stream)
        return y

    @property
    def n_bonds(self):
        return self.bonds.shape[0]

    def basis(self, spin):
        return hub_get_basis(self.h, spin, self.count_up if spin == 0 else self.count_dn)

    def csr(self, spin):
        return hub_get_csr(self.h, spin, self.count_up if spin == 0 else self.count_dn)

    def apply(self, x, y=None, stream=None):
        import torch
        if y is None:
            y = torch.empty_like(x)
        hub_apply(self.h, x, y, stream)
        return y

    def apply_host(self, x, y=None, stream=None):
        """y = H x on host arrays (numpy arrays or CPU tensors; page-locked memory copies
        fastest): one vector of shape (D,) through hub_apply_host, or n vectors of shape
        (n, D) in one hub_apply_host_many call.  y defaults to a new array like x."""
        if y is None:
            y = x.new_empty(tuple(x.shape)) if hasattr(x, "new_empty") else np.empty_like(x)
        if tuple(y.shape) != tuple(x.shape):
            raise ValueError(f"apply_host: x has shape {tuple(x.shape)}, y {tuple(y.shape)}")
        if len(x.shape) == 1:
            hub_apply_host(self.h, x, y, stream)
        elif len(x.shape) == 2:
            hub_apply_host_many(self.h, int(x.shape[0]), x, y, stream)
        else:
            raise ValueError("apply_host: x must have one or two dimensions")
        return y

    def ground(self, x0=None, maxit=300, tol=1e-12, want_psi=False, stream=None):
        import torch
        psi = torch.empty(self.D, dtype=torch.float64, device="cuda") if want_psi else None
        E0, iters, rc = hub_lanczos_ground(self.h, x0, maxit, tol, psi, stream)
        return dict(E0=E0, iters=iters, status=rc, psi=psi)

    def grad(self, psi, stream=None):
        return hub_grad(self.h, psi, self.n_bonds, self.M, stream)

    def vjp(self, ybar, x, want_params=True, stream=None):
        import torch
        xbar = torch.empty_like(ybar)
        dt, dU, de = hub_apply_vjp(self.h, ybar, x, xbar, self.n_bonds, self.M, want_params, stream)
        return xbar, dt, dU, de

    def close(self):
        if self.h:
            hub_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------------- autograd

def _autograd():
    import torch

    class ApplyFn(torch.autograd.Function):
        """y = H(t, U, eps) x.  Backward: xbar = H ybar (H symmetric); parameter
        cotangents ybar^T (dH/dtheta) x from the library's bilinear-form kernel."""

        @staticmethod
        def forward(ctx, model, x, t, U, eps):
            model.ensure_params(t.detach().cpu().numpy(), U.detach().cpu().numpy(), eps.detach().cpu().numpy())
            y = model.apply(x.detach().contiguous())
            ctx.model = model
            ctx.param_devices = (t.device, U.device, eps.device)
            ctx.save_for_backward(x)
            return y

        @staticmethod
        def backward(ctx, ybar):
            (x,) = ctx.saved_tensors
            m = ctx.model
            xbar, dt, dU, de = m.vjp(ybar.contiguous(), x.contiguous(), want_params=any(ctx.needs_input_grad[2:]))
            devs = ctx.param_devices
            cvt = (lambda a, dev: None if a is None else torch.as_tensor(a, dtype=torch.float64, device=dev))
            return None, xbar, cvt(dt, devs[0]), cvt(dU, devs[1]), cvt(de, devs[2])

    class GroundEnergyFn(torch.autograd.Function):
        """E0(t, U, eps) by Lanczos; backward by Hellmann-Feynman (hub_grad on psi)."""

        @staticmethod
        def forward(ctx, model, t, U, eps, x0, maxit, tol):
            model.ensure_params(t.detach().cpu().numpy(), U.detach().cpu().numpy(), eps.detach().cpu().numpy())
            r = model.ground(x0, maxit=maxit, tol=tol, want_psi=True)
            ctx.model = model
            ctx.psi = r["psi"]
            return torch.tensor(r["E0"], dtype=torch.float64)

        @staticmethod
        def backward(ctx, gE):
            dt, dU, de = ctx.model.grad(ctx.psi)
            g = float(gE)
            cvt = (lambda a: torch.as_tensor(a * g, dtype=torch.float64))
            return None, cvt(dt), cvt(dU), cvt(de), None, None, None

    return ApplyFn, GroundEnergyFn


def apply_fn(model, x, t, U, eps):
    """Differentiable y = H x (see ApplyFn)."""
    return _autograd()[0].apply(model, x, t, U, eps)


def ground_energy(model, t, U, eps, x0=None, maxit=300, tol=1e-12):
    """Differentiable ground-state energy (see GroundEnergyFn)."""
    return _autograd()[1].apply(model, t, U, eps, x0, maxit, tol)
