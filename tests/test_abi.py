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
