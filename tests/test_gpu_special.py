"""The FP32 special functions of the deflection kernel, on the GPU, at every
float argument the kernel can give them.

* The hardware approximations (PTX rsqrt / sqrt / rcp / lg2, flush-to-zero
  forms): the largest relative error over every float of a range that covers
  all the kernel's arguments, against double precision.
* The library's atan(t)/t and atanh(t)/t of u = t^2 (polynomial plus range
  reduction, as the kernels evaluate them): the same, over every float u the
  kernel can produce with a finite error bound (atan: [0, 2^14], since the
  difference-form argument is below 1/q and the bound is finite only for
  q >= 0.01; atanh: [0, 1/4] for its polynomial and, weighted by 1 - u,
  [1/4, 0.99999988] for its logarithm, up to its clamp).

The error bound of the FP32 deflection is built on the constants kEps* of
the kernel header (units of the FP32 unit roundoff u = 2^-24), which these
tests read as their budgets; each test fails if the hardware or the code
exceeds its budget.  lg2 enters the bound only through atanh(t)/t, whose
budget covers it.
"""
import ctypes as C
import os
import re
import subprocess

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(os.path.dirname(HERE), "paper_1902_03252_gb300", "csrc", "lt_internal.cuh")
U = 2.0 ** -24


def budget(name):
    m = re.search(rf"constexpr double {name} = ([0-9.eE+-]+);", open(HEADER).read())
    assert m, name
    return float(m.group(1))


# (which, name, lo, hi, budget in u)
CASES = [
    (0, "rsqrt.approx.ftz", 2.0 ** -120, 2.0 ** 120, budget("kEpsRsqrt")),
    (1, "sqrt.approx.ftz", 2.0 ** -120, 2.0 ** 120, budget("kEpsSqrt")),
    (2, "rcp.approx.ftz", 2.0 ** -120, 2.0 ** 120, budget("kEpsRcp")),
    (3, "lg2.approx.ftz on [2.99, 2^26]", 2.99, 2.0 ** 26, 8.0),
    (4, "atan(t)/t of u on [0, 2^14]", 0.0, 16384.0, budget("kEpsAtanc")),
    (5, "atanh(t)/t of u on [0, 1/4]", 0.0, 0.25, budget("kEpsAtanhc")),
    (6, "(1 - u) x atanh(t)/t of u on [1/4, 0.99999988]", 0.25, 0.99999988,
     budget("kEpsAtanhcLog")),
]


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1902_03252_gb300 import _build
    out = tmp_path_factory.mktemp("special") / "libspecial.so"
    subprocess.check_call([_build.nvcc(), *_build.ARCH, "-O3", "-std=c++17", "-ftz=true",
                           "-Xcompiler", "-fPIC", "-shared",
                           os.path.join(HERE, "gpu_special_check.cu"), "-o", str(out)])
    L = C.CDLL(str(out))
    L.special_max_err.argtypes = [C.c_int, C.c_float, C.c_float, C.POINTER(C.c_double),
                                  C.POINTER(C.c_float)]
    L.special_max_err.restype = C.c_int
    return L


@pytest.mark.parametrize("which,name,lo,hi,budget", CASES, ids=[c[1] for c in CASES])
def test_max_relative_error(lib, which, name, lo, hi, budget):
    err = C.c_double(0.0)
    worst = C.c_float(0.0)
    rc = lib.special_max_err(which, lo, hi, C.byref(err), C.byref(worst))
    assert rc == 0, rc
    ulp = err.value / U
    print(f"{name}: max relative error {ulp:.3f} u at x = {worst.value!r}")
    assert ulp <= budget, (name, ulp, worst.value)
