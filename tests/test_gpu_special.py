"""The FP32 special functions of the deflection kernel, on the GPU, at every
float argument the kernel can give them.

* The hardware approximations (PTX rsqrt / sqrt / rcp / lg2, flush-to-zero
  forms): the largest relative error over every float of a range that covers
  all the kernel's arguments, against double precision.
* The library's atan(t)/t and atanh(t)/t of u = t^2 (polynomial plus range
  reduction, as the kernels evaluate them): the same, over every float u the
  kernel can produce (atan: [0, 128], since the difference-form argument is
  below 1/q <= 10 for the ellipticities the library accepts with a finite
  bound; atanh: [0, 0.99999988], its clamp).

The error bound of the FP32 deflection is built on the budgets below (units
of the FP32 unit roundoff u = 2^-24); each test fails if the hardware or the
code exceeds its budget.
"""
import ctypes as C
import os
import subprocess

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
U = 2.0 ** -24

# (which, name, lo, hi, budget in u)
CASES = [
    (0, "rsqrt.approx.ftz", 2.0 ** -120, 2.0 ** 120, 2.0),
    (1, "sqrt.approx.ftz", 2.0 ** -120, 2.0 ** 120, 2.0),
    (2, "rcp.approx.ftz", 2.0 ** -120, 2.0 ** 120, 2.0),
    (3, "lg2.approx.ftz on [2.99, 2^26]", 2.99, 2.0 ** 26, 4.0),
    (4, "atan(t)/t of u on [0, 128]", 0.0, 128.0, 16.0),
    (5, "atanh(t)/t of u on [0, 0.99999988]", 0.0, 0.99999988, 16.0),
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
