"""Pins of the oracle's deflections against mathematics the paper fixes.

None of these retypes the oracle's formula: the SIS is checked against its
closed-form magnitude (Sect. 2.1), the PIEMD against an independent
quadrature of the homoeoidal integrals of its convergence, Poisson's
equation, curl-freeness and its circular/SIS limits, and the SIE of
Algorithm 1 against central differences of its pseudo-elliptical potential.
"""
import math

import numpy as np
import pytest
from scipy import integrate

C_KMS = 299792.458
ARCSEC = 206264.80625


def b0(sv):
    return 4 * math.pi * (sv / C_KMS) ** 2 * ARCSEC


def one(kind, x=0.0, y=0.0, e=0.0, phi=0.0, rc=0.0, rcut=0.0, sv=500.0):
    return np.array([[kind], [x], [y], [e], [phi], [rc], [rcut], [sv]], dtype=float)


def test_sis_constant_magnitude(oracle):
    """|alpha| = theta_E everywhere but the centre (Sect. 2.1, Eq. 10)."""
    rng = np.random.default_rng(1)
    p = one(0, 3.0, -2.0, sv=812.0)
    x, y = rng.uniform(-80, 80, (2, 500))
    ax, ay, _ = oracle.alpha_points(p, x, y)
    np.testing.assert_allclose(np.hypot(ax, ay), b0(812.0), rtol=2e-15)
    # points radially away from the centre
    d = np.hypot(x - 3.0, y + 2.0)
    np.testing.assert_allclose(ax * (x - 3.0) + ay * (y + 2.0), b0(812.0) * d, rtol=1e-13)


def test_sis_centre_is_zero(oracle):
    ax, ay, _ = oracle.alpha_points(one(0, 1.5, 2.5), [1.5], [2.5])
    assert ax[0] == 0.0 and ay[0] == 0.0


def piemd_kappa(x, y, q, a, s, B):
    """Convergence of the dPIE reading in its own (unrotated) frame."""
    pa = math.sqrt(q * q * (a * a + x * x) + y * y)
    ps = math.sqrt(q * q * (s * s + x * x) + y * y)
    return 0.5 * B * s / (s - a) * (1 / pa - 1 / ps)


def quad_alpha_cored(x, y, q, w):
    """Deflection of kappa = 1/(2 sqrt(q^2 (w^2 + x^2) + y^2)) by the
    homoeoidal integrals alpha_x = q x J0, alpha_y = q y J1 with
    J_n = int_0^1 kappa(xi^2(u)) / (1 - (1-q^2) u)^(n + 1/2) du,
    xi^2(u) = u (x^2 + y^2 / (1 - (1-q^2) u)) (Schramm 1990), integrated
    numerically (u = t^2 removes the endpoint behaviour)."""
    k2 = 1 - q * q

    def J(n):
        def f(t):
            u = t * t
            m = 1 - k2 * u
            xi2 = u * (x * x + y * y / m)
            return t / (q * math.sqrt(w * w + xi2)) / m ** (n + 0.5)
        return integrate.quad(f, 0, 1, epsabs=0, epsrel=1e-13, limit=400)[0]
    return q * x * J(0), q * y * J(1)


def test_piemd_matches_quadrature(oracle):
    rng = np.random.default_rng(2)
    for _ in range(40):
        e = rng.uniform(0.0, 0.9)
        q = 1 - e
        a = 10 ** rng.uniform(-2, 0.5)
        s = a + 10 ** rng.uniform(0, 2.5)
        phi = rng.uniform(0, math.pi)
        cx, cy = rng.uniform(-50, 50, 2)
        sv = rng.uniform(50, 1200)
        p = one(1, cx, cy, e, phi, a, s, sv)
        x, y = cx + rng.uniform(-60, 60) * rng.choice([1e-2, 0.3, 1]), cy + rng.uniform(-60, 60)
        ax, ay, _ = oracle.alpha_points(p, [x], [y])
        # into the lens frame, quadrature of both cored terms, back out
        c, sn = math.cos(phi), math.sin(phi)
        xp, yp = (x - cx) * c + (y - cy) * sn, (y - cy) * c - (x - cx) * sn
        fa = quad_alpha_cored(xp, yp, q, a)
        fs = quad_alpha_cored(xp, yp, q, s)
        B = b0(sv) * s / (s - a)
        gx, gy = B * (fa[0] - fs[0]), B * (fa[1] - fs[1])
        ex, ey = gx * c - gy * sn, gy * c + gx * sn
        scale = max(abs(ex), abs(ey), 1e-3 * B)
        assert abs(ax[0] - ex) < 1e-10 * scale and abs(ay[0] - ey) < 1e-10 * scale, (ax, ex, ay, ey)


@pytest.mark.parametrize("e", [0.0, 0.2, 0.5, 0.85])
def test_piemd_poisson_and_curl(oracle, e):
    """div alpha = 2 kappa and curl alpha = 0 by central differences."""
    rng = np.random.default_rng(3)
    a, s, sv, phi = 0.4, 120.0, 700.0, 0.7
    p = one(1, 1.0, -2.0, e, phi, a, s, sv)
    h = 1e-4
    for _ in range(20):
        x, y = rng.uniform(-30, 30, 2)
        X = np.array([x + h, x - h, x, x])
        Y = np.array([y, y, y + h, y - h])
        ax, ay, _ = oracle.alpha_points(p, X, Y)
        div = (ax[0] - ax[1] + ay[2] - ay[3]) / (2 * h)
        curl = (ay[0] - ay[1] - (ax[2] - ax[3])) / (2 * h)
        c, sn = math.cos(phi), math.sin(phi)
        xp, yp = (x - 1.0) * c + (y + 2.0) * sn, (y + 2.0) * c - (x - 1.0) * sn
        kap = piemd_kappa(xp, yp, 1 - e, a, s, b0(sv))
        assert abs(div - 2 * kap) < 1e-6 * max(1.0, 2 * kap), (div, 2 * kap)
        assert abs(curl) < 1e-6 * max(1.0, 2 * kap)


def test_piemd_circular_limit(oracle):
    """e = 0: Gauss's law, alpha(R) = M(<R)/(pi R) with
    M(<R)/pi = B [(sqrt(a^2+R^2) - a) - (sqrt(s^2+R^2) - s)]."""
    rng = np.random.default_rng(4)
    a, s, sv = 0.7, 80.0, 900.0
    p = one(1, -3.0, 4.0, 0.0, 1.1, a, s, sv)
    B = b0(sv) * s / (s - a)
    x, y = rng.uniform(-100, 100, (2, 300))
    ax, ay, _ = oracle.alpha_points(p, x, y)
    R = np.hypot(x + 3.0, y - 4.0)
    mag = B * ((np.sqrt(a * a + R * R) - a) - (np.sqrt(s * s + R * R) - s)) / R
    np.testing.assert_allclose(np.hypot(ax, ay), mag, rtol=1e-12)


def test_piemd_sis_limit(oracle):
    """Vanishing core, infinite cut, e = 0 reduces to the paper's SIS."""
    rng = np.random.default_rng(5)
    p = one(1, 0.0, 0.0, 0.0, 0.3, 1e-9, 1e12, 1000.0)
    x, y = rng.uniform(-100, 100, (2, 100))
    ax, ay, _ = oracle.alpha_points(p, x, y)
    bx, by, _ = oracle.alpha_points(one(0, sv=1000.0), x, y)
    np.testing.assert_allclose(ax, bx, rtol=1e-7, atol=1e-7)
    np.testing.assert_allclose(ay, by, rtol=1e-7, atol=1e-7)


def test_sie_is_gradient_of_pseudo_elliptical_potential(oracle):
    """Algorithm 1 returns grad of Psi_eps = b0 R(x', y') (Sect. 2.2.2,
    pseudo-elliptical SIS), checked by central differences of the potential."""
    rng = np.random.default_rng(6)
    for _ in range(30):
        eps, phi = rng.uniform(0, 0.3), rng.uniform(0, math.pi)
        cx, cy, sv = *rng.uniform(-20, 20, 2), rng.uniform(10, 1000)
        p = one(2, cx, cy, eps, phi, sv=sv)
        c, sn = math.cos(phi), math.sin(phi)

        def pot(x, y):
            xp, yp = (x - cx) * c + (y - cy) * sn, (y - cy) * c - (x - cx) * sn
            return b0(sv) * math.sqrt(xp * xp * (1 - eps) + yp * yp * (1 + eps))
        x, y = rng.uniform(-40, 40, 2)
        h = 1e-5
        gx = (pot(x + h, y) - pot(x - h, y)) / (2 * h)
        gy = (pot(x, y + h) - pot(x, y - h)) / (2 * h)
        ax, ay, _ = oracle.alpha_points(p, [x], [y])
        assert abs(ax[0] - gx) < 1e-7 * b0(sv) and abs(ay[0] - gy) < 1e-7 * b0(sv)


def test_sie_reduces_to_sis(oracle):
    """eps = 0: the SIE equations reduce to the SIS (Sect. 2.2.2)."""
    rng = np.random.default_rng(7)
    x, y = rng.uniform(-50, 50, (2, 200))
    ax, ay, _ = oracle.alpha_points(one(2, 2.0, 1.0, 0.0, 0.9, sv=640.0), x, y)
    bx, by, _ = oracle.alpha_points(one(0, 2.0, 1.0, sv=640.0), x, y)
    np.testing.assert_allclose(ax, bx, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(ay, by, rtol=1e-13, atol=1e-13)


def test_superposition(oracle):
    """alpha of a sum of potentials is the sum of their alphas (Sect. 2.2.2)."""
    rng = np.random.default_rng(8)
    ps = [one(1, *rng.uniform(-30, 30, 2), 0.3, 0.4, 0.5, 90.0, 800.0),
          one(0, *rng.uniform(-30, 30, 2), sv=300.0),
          one(2, *rng.uniform(-30, 30, 2), 0.1, 2.0, sv=200.0)]
    x, y = rng.uniform(-40, 40, (2, 50))
    tot = np.concatenate(ps, axis=1)
    ax, ay, s = oracle.alpha_points(tot, x, y)
    parts = [oracle.alpha_points(p, x, y) for p in ps]
    np.testing.assert_allclose(ax, sum(q[0] for q in parts), rtol=1e-13, atol=1e-12)
    np.testing.assert_allclose(ay, sum(q[1] for q in parts), rtol=1e-13, atol=1e-12)
    np.testing.assert_allclose(s, sum(np.abs(q[0]) + np.abs(q[1]) for q in parts), rtol=1e-13)


def test_grid_matches_points(oracle):
    rng = np.random.default_rng(9)
    p = np.concatenate([one(1, *rng.uniform(-30, 30, 2), 0.3, 0.4, 0.5, 90.0, 800.0),
                        one(0, 3.0, 3.0, sv=300.0)], axis=1)
    grid = (-10.0, -12.0, 0.5, 0.75, 17, 13)
    a, s = oracle.deflect_grid(p, grid, n_threads=2)
    jj, ii = np.mgrid[0:13, 0:17]
    ax, ay, s2 = oracle.alpha_points(p, (-10.0 + ii * 0.5).ravel(), (-12.0 + jj * 0.75).ravel())
    assert np.array_equal(a[..., 0].ravel(), ax) and np.array_equal(a[..., 1].ravel(), ay)
    assert np.array_equal(s.ravel(), s2)
