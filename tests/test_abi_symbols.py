"""The C-ABI library builds for sm_103a, loads, and exports every function of include/magnus.h.

CPU only: no compute call is made (there is no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "magnus.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(mg_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_path():
    names = declared_functions()
    for required in ["mg_ctx_create", "mg_plan_create", "mg_set_controls", "mg_evolve", "mg_expm",
                     "mg_cgemm", "mg_build_omega", "mg_coefficients", "mg_propagate", "mg_strerror"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2411_09982_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_header():
    from paper_2411_09982_gb300 import magnus
    assert set(declared_functions()) <= set(magnus.SIGNATURES), set(declared_functions()) - set(magnus.SIGNATURES)


def test_strerror_is_host_only():
    from paper_2411_09982_gb300 import magnus
    lib = magnus.load()
    assert lib.mg_strerror(0) == b"ok"
    assert lib.mg_strerror(magnus.MG_ETIMEOUT).startswith(b"device-side wait")


def test_ctx_create_fails_loudly_without_gpu():
    """No CPU fallback: on a machine without an sm_103a GPU the context cannot be created."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2411_09982_gb300 import magnus
    with pytest.raises(magnus.MagnusError):
        magnus.Context(0)
