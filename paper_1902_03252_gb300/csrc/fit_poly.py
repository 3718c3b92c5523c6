"""Coefficients of the FP32 special functions of the deflection kernel.

atanc(u) = atan(sqrt u)/sqrt u on [0, 1] and atanhc(u) = atanh(sqrt u)/sqrt u
on [0, U_H] are approximated by polynomials in u, fitted by least squares in
the relative sense at Chebyshev nodes of the interval (near-minimax; see
Trefethen, "Approximation Theory and Approximation Practice", ch. 16), in
float64.  Prints, for each degree, the maximum relative error of the float64
polynomial and of its float32 Horner evaluation (float32 coefficients)
against the float64 function, and the coefficients of the degrees the kernel
uses (highest degree first, for Horner).

The kernel uses degree 6 for atanc and 4 for atanhc.  Each degree less saves
one FP32 operation per node and potential in the deflection, and the larger
approximation error (13.5 and 7.7 ulp, against 1.5 and 1.7 ulp at degrees 8
and 5) is added to the error bound's coefficients errGx and errGy, which
are about 80 and 100 ulp: the bound grows by several per cent.

Usage: python fit_poly.py
"""
import numpy as np

U_H = 0.25  # atanhc polynomial interval; above it the kernel uses a logarithm


def fit(f, a, b, deg, n=4000):
    k = np.arange(n)
    x = (a + b) / 2 + (b - a) / 2 * np.cos(np.pi * (k + 0.5) / n)
    y = f(x)
    V = np.vander(x, deg + 1)
    c, *_ = np.linalg.lstsq(V / y[:, None], np.ones_like(y), rcond=None)
    return c


def check(f, c, a, b):
    x = np.linspace(a, b, 200001)
    y = f(x)
    p64 = np.polyval(c, x)
    xf = x.astype(np.float32)
    acc = np.float32(c[0])
    for ci in c[1:]:
        acc = (acc * xf + np.float32(ci)).astype(np.float32)
    return np.max(np.abs(p64 / y - 1)), np.max(np.abs(acc.astype(np.float64) / y - 1))


def atanc(u):
    s = np.sqrt(u)
    return np.where(u > 0, np.arctan(s) / np.where(s > 0, s, 1), 1.0)


def atanhc(u):
    s = np.sqrt(u)
    return np.where(u > 0, np.arctanh(s) / np.where(s > 0, s, 1), 1.0)


USED = {"atanc": 6, "atanhc": 4}  # degrees in the kernel

if __name__ == "__main__":
    for name, f, a, b in (("atanc", atanc, 0.0, 1.0), ("atanhc", atanhc, 0.0, U_H)):
        for deg in range(3, 10):
            c = np.array([float(np.float32(v)) for v in fit(f, a, b, deg)])
            e64, e32 = check(f, c, a, b)
            print(f"{name} deg {deg}: rel err f64 {e64:.2e}  f32 Horner {e32:.2e} "
                  f"({e32 / 2.0**-24:.1f} ulp)")
            if deg == USED[name]:
                print("  coefficients:", ", ".join(f"{v:.9e}f" for v in c))

