"""The C-ABI library builds, loads and exports every entry point include/hub.h declares
(no compute calls: these run without a GPU)."""
import os
import re
import subprocess

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "hub.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hub_[A-Za-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1307_7542_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared()
    for must in ("hub_basis", "hub_hopping", "hub_apply", "hub_lanczos_ground", "hub_grad", "hub_apply_vjp",
                 "hub_free"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s+(hub_\w+)", out))
    missing = [n for n in declared() if n not in exported]
    assert not missing, f"declared but not exported: {missing}"


def test_binding_covers_every_symbol(libpath):
    from paper_1307_7542_gb300 import hub
    assert sorted(hub.SIGNATURES) == declared()
    L = hub.lib()
    for n in declared():
        assert hasattr(L, n)
    assert L.hub_last_error() is not None


def test_header_compiles_as_c():
    """include/hub.h is plain C (no CUDA or torch types in the signatures)."""
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-fsyntax-only", "-x", "c", HEADER],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_no_gpu_returns_error_code(libpath):
    """Without a device, set-up fails with a negative code and a message, never a crash."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1307_7542_gb300 import hub
    with pytest.raises(hub.HubError) as e:
        hub.hub_basis(4, 2, 2)
    assert e.value.code < 0


def test_null_handles_are_refused(libpath):
    """Every entry point that takes a handle refuses NULL with HUB_ERR_ARG and a message,
    before any device work (host logic, no GPU needed)."""
    from paper_1307_7542_gb300 import hub
    import ctypes
    L = hub.lib()
    i64 = ctypes.c_int64()
    d = ctypes.c_double()
    n = ctypes.c_int()
    buf = (ctypes.c_int32 * 8)()
    calls = {
        "hub_dims": lambda: L.hub_dims(None, ctypes.byref(i64), ctypes.byref(i64)),
        "hub_hopping": lambda: L.hub_hopping(None, 0, None, None, None),
        "hub_set_U": lambda: L.hub_set_U(None, 1, None),
        "hub_apply": lambda: L.hub_apply(None, None, None, None),
        "hub_apply_host": lambda: L.hub_apply_host(None, None, None, None),
        "hub_apply_host_many": lambda: L.hub_apply_host_many(None, 2, None, None, None),
        "hub_lanczos_ground": lambda: L.hub_lanczos_ground(None, None, 10, 0.0, ctypes.byref(d), None,
                                                           ctypes.byref(n), None),
        "hub_lanczos_coeffs": lambda: L.hub_lanczos_coeffs(None, None, None, 0, ctypes.byref(n)),
        "hub_lanczos_spectrum": lambda: L.hub_lanczos_spectrum(None, None, 10, 1, None, None, ctypes.byref(n), None),
        "hub_lanczos_ritz": lambda: L.hub_lanczos_ritz(None, None, 10, 0.0, None, ctypes.byref(d), None),
        "hub_lanczos_block": lambda: L.hub_lanczos_block(None, 2, None, 10, 1, buf, None, ctypes.byref(n), None),
        "hub_green_coeffs": lambda: L.hub_green_coeffs(None, None, 1, None, None, ctypes.byref(d), ctypes.byref(n), None),
        "hub_ladder": lambda: L.hub_ladder(None, None, 0, 0, 1, None, None, None),
        "hub_grad": lambda: L.hub_grad(None, None, None, None, None, None),
        "hub_grad_noalloc": lambda: L.hub_grad_noalloc(None, None, None, None, None, None),
        "hub_apply_vjp": lambda: L.hub_apply_vjp(None, None, None, None, None, None, None, None),
        "hub_set_symmetry": lambda: L.hub_set_symmetry(None, 1),
        "hub_set_translations": lambda: L.hub_set_translations(None, 1, buf, buf),
        "hub_k_dims": lambda: L.hub_k_dims(None, None, None, None),
        "hub_k_reps": lambda: L.hub_k_reps(None, None, None),
        "hub_k_columns": lambda: L.hub_k_columns(None, None, None),
        "hub_k_project": lambda: L.hub_k_project(None, None, None, None),
        "hub_set_mode": lambda: L.hub_set_mode(None, 0),
        "hub_check": lambda: L.hub_check(None),
        "hub_test_fail_waits": lambda: L.hub_test_fail_waits(None, 1),
        "hub_set_small_dim": lambda: L.hub_set_small_dim(None, 0),
        "hub_profile": lambda: L.hub_profile(None, 1),
        "hub_profile_read": lambda: L.hub_profile_read(None, 0, None, None, None),
        "hub_csr_info": lambda: L.hub_csr_info(None, 0, None, None),
        "hub_get_csr": lambda: L.hub_get_csr(None, 0, None, None, None),
        "hub_get_basis": lambda: L.hub_get_basis(None, 0, None),
    }
    for name, call in calls.items():
        assert call() == hub.HUB_ERR_ARG, name
        assert L.hub_last_error(), name
    L.hub_free(None)


def test_green_eval_is_the_continued_fraction(libpath):
    """hub_green_eval (host code) equals the oracle's continued fraction on random coefficients,
    particle and hole terms, at points on and off the real axis; k = 0 gives 0; bad arguments
    are refused."""
    import numpy as np
    from oracle import hub_oracle as O
    from paper_1307_7542_gb300 import hub
    rng = np.random.default_rng(11)
    for k in (1, 2, 7, 40):
        a = rng.uniform(-3, 3, k)
        b = rng.uniform(0.1, 2.0, k)
        z = rng.uniform(-8, 8, 25) + 1j * rng.uniform(0.01, 1.0, 25)
        for sign in (1, -1):
            g = hub.hub_green_eval(a, b, 0.7, -1.3, sign, z)
            ref = O.continued_fraction(a, b, 0.7, -1.3, sign, z)
            assert np.max(np.abs(g - ref) / np.abs(ref)) < 1e-13
    assert np.all(hub.hub_green_eval(np.zeros(0), np.zeros(0), 1.0, 0.0, 1, np.array([1.0 + 1j])) == 0)
    with pytest.raises(hub.HubError):
        hub.hub_green_eval(np.ones(3), np.ones(3), 1.0, 0.0, 2, np.array([1.0 + 1j]))


def test_binding_constants_match_the_header():
    """Every #define HUB_* of include/hub.h exists in the binding with the same value."""
    from paper_1307_7542_gb300 import hub
    src = open(HEADER).read()
    defs = dict(re.findall(r"#define\s+(HUB_[A-Z0-9_]+)\s+\(?(-?\d+)\)?", src))
    assert len(defs) >= 15
    for name, val in defs.items():
        assert hasattr(hub, name), name
        assert getattr(hub, name) == int(val), name


def test_plain_c_caller(libpath, tmp_path):
    """tests/c_abi_check.c, compiled with gcc against include/hub.h and the library, runs the
    device-free calls and checks them (refusals, the continued fraction by hand)."""
    exe = str(tmp_path / "c_abi_check")
    libdir = os.path.dirname(libpath)
    lib = os.path.basename(libpath)[3:-3]
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", os.path.join(ROOT, "tests", "c_abi_check.c"),
                        "-I", os.path.join(ROOT, "include"), "-L", libdir, f"-l{lib}",
                        f"-Wl,-rpath,{libdir}", "-lm", "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr


def test_group_construction_host_checks(tmp_path):
    """tests/cpp_group_check.cpp (g++, csrc/hub_group.h): the momentum-sector group closure and
    refusals, the action on spin strings as a representation with fermion signs, orbits and
    stabilisers, and every move-table entry against the action."""
    exe = str(tmp_path / "cpp_group_check")
    r = subprocess.run(["g++", "-std=c++17", "-O1", "-Wall", "-Werror", "-I",
                        os.path.join(ROOT, "paper_1307_7542_gb300", "csrc"),
                        os.path.join(ROOT, "tests", "cpp_group_check.cpp"), "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
