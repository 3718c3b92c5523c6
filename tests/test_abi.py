"""The C-ABI library loads and exports every function include/lt.h declares.

CPU-only: the library is built here if needed (nvcc cross-compiles for
sm_103a) and loaded with ctypes; no compute call is made.
"""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lt.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(lt_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1902_03252_gb300 import _build
    try:
        return _build.build()
    except RuntimeError as e:
        pytest.skip(f"cannot build the CUDA library here: {e}")


def test_header_declares_the_boundary():
    names = declared()
    for must in ("lt_model_create", "lt_model_set_params", "lt_deflect_grid", "lt_find_images",
                 "lt_chi2", "lt_chi2_grad", "lt_model_destroy", "lt_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(lt_\w+)$", out, flags=re.M))
    missing = [n for n in declared() if n not in exported]
    assert not missing, missing
    L = C.CDLL(lib_path)
    for n in declared():
        getattr(L, n)
    L.lt_version.restype = C.c_char_p
    assert b"sm_103a" in L.lt_version()


def test_binding_fails_loudly_without_gpu():
    """No CPU fallback: on a machine without a GPU the binding raises."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1902_03252_gb300 import lt
    with pytest.raises(RuntimeError):
        lt.Model(4, 1)
