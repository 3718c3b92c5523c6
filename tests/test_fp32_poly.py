"""The FP32 polynomials of the deflection kernel (atan(t)/t on u = t^2 in
[0, 1], atanh(t)/t on [0, 1/4]), evaluated exactly as the kernel evaluates
them (Horner's rule with fused multiply-adds rounded once to float,
flush-to-zero inputs), checked against the exact functions at every float u
of their intervals.  The coefficients are read from the kernel header, so the
check covers the literals the kernel is built with.

The measured maxima are the polynomial errors the FP32 error bound is built
on (13.5 and 7.7 ulp); the test fails if the coefficients change in a way that
raises them.
"""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(os.path.dirname(HERE), "paper_1902_03252_gb300", "csrc", "lt_internal.cuh")
U = 2.0 ** -24
# the bound's budget for the two polynomials (relative error in units of U);
# the atan interval reaches just above 1 because the reduced argument 1/t^2
# is formed as rsqrt(t^2)^2 and may round a few units above 1
BUDGET = {"atanc_poly32": (0.0, 1.0 + 8 * U, 13.6), "atanhc_poly32": (0.0, 0.25, 7.8)}


def coefficients(name):
    src = open(HEADER).read()
    body = src[src.index(f"float {name}(float u)"):]
    body = body[:body.index("\n}")]
    return [float(np.float32(v)) for v in re.findall(r"([-+]?\d\.\d+e[-+]\d+)f", body)]


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    out = tmp_path_factory.mktemp("poly") / "libpolycheck.so"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                           os.path.join(HERE, "fp32_poly_check.c"), "-o", str(out), "-lm"])
    L = C.CDLL(str(out))
    L.poly_max_rel_err.argtypes = [C.c_int, C.POINTER(C.c_float), C.c_int, C.c_float, C.c_float,
                                   C.c_int, C.POINTER(C.c_float)]
    L.poly_max_rel_err.restype = C.c_double
    return L


def run(lib, which, name, lo, hi):
    c = coefficients(name)
    arr = (C.c_float * len(c))(*c)
    worst = C.c_float(0.0)
    e = lib.poly_max_rel_err(which, arr, len(c), lo, hi, os.cpu_count() or 4, C.byref(worst))
    return e / U, worst.value, c


def test_coefficients_parsed():
    assert len(coefficients("atanc_poly32")) == 7
    assert len(coefficients("atanhc_poly32")) == 5


@pytest.mark.parametrize("which,name", [(0, "atanc_poly32"), (1, "atanhc_poly32")])
def test_polynomial_exhaustive(lib, which, name):
    lo, hi, budget = BUDGET[name]
    err, worst, c = run(lib, which, name, lo, hi)
    print(f"{name}: max relative error {err:.3f} ulp at u = {worst!r} over every float in "
          f"[{lo}, {hi}]")
    assert err <= budget, (err, worst)


def test_check_sees_a_wrong_coefficient(lib):
    """A coefficient changed in its last place raises the measured error,
    and a dropped term raises it far beyond the budget."""
    c = coefficients("atanhc_poly32")
    arr = (C.c_float * 5)(*c)
    base = lib.poly_max_rel_err(1, arr, 5, 0.0, 0.25, os.cpu_count() or 4, None) / U
    bad = list(c)
    bad[-1] = float(np.nextafter(np.float32(bad[-1]), np.float32(2)))
    bad = lib.poly_max_rel_err(1, (C.c_float * 5)(*bad), 5, 0.0, 0.25, os.cpu_count() or 4,
                               None) / U
    assert bad != base
    drop = lib.poly_max_rel_err(1, (C.c_float * 4)(*c[1:]), 4, 0.0, 0.25, os.cpu_count() or 4,
                                None) / U
    assert drop > 100 * base
