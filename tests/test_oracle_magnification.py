"""Pins of the oracle's magnifications and source-plane chi^2.

The Jacobian comes from dual numbers through the deflection code; it is
pinned to central differences of the (separately pinned) deflection, to the
closed-form convergence of each profile (trace = 2 kappa, Poisson) and to
curl-freeness.  Point and triangle magnifications and the source-plane chi^2
are pinned to the SIS closed forms of Sect. 2.1 (|alpha| = theta_E).
"""
import math

import numpy as np
import pytest

C_KMS = 299792.458
ARCSEC = 206264.80625


def b0(sv):
    return 4 * math.pi * (sv / C_KMS) ** 2 * ARCSEC


def one(kind, x=0.0, y=0.0, e=0.0, phi=0.0, rc=0.0, rcut=0.0, sv=500.0):
    return np.array([[kind], [x], [y], [e], [phi], [rc], [rcut], [sv]], dtype=float)


def mixed_lens(rng):
    return np.concatenate([one(1, *rng.uniform(-20, 20, 2), 0.35, 0.6, 0.8, 150.0, 900.0),
                           one(0, *rng.uniform(-20, 20, 2), sv=300.0),
                           one(2, *rng.uniform(-20, 20, 2), 0.12, 2.1, sv=400.0)], axis=1)


def test_jacobian_matches_central_differences(oracle):
    rng = np.random.default_rng(11)
    p = mixed_lens(rng)
    x, y = rng.uniform(-40, 40, (2, 60))
    J = oracle.jacobian_points(p, x, y)
    h = 1e-5
    axp, ayp, _ = oracle.alpha_points(p, x + h, y)
    axm, aym, _ = oracle.alpha_points(p, x - h, y)
    bxp, byp, _ = oracle.alpha_points(p, x, y + h)
    bxm, bym, _ = oracle.alpha_points(p, x, y - h)
    fd = np.stack([np.stack([(axp - axm), (bxp - bxm)], -1),
                   np.stack([(ayp - aym), (byp - bym)], -1)], 1) / (2 * h)
    np.testing.assert_allclose(J, fd, rtol=0, atol=1e-6 * max(1.0, np.abs(J).max()))


def test_jacobian_trace_is_twice_kappa(oracle):
    """Poisson's equation with each profile's closed-form convergence; the
    Jacobian of a gradient field is symmetric."""
    rng = np.random.default_rng(12)
    for _ in range(30):
        kind = int(rng.integers(0, 3))
        cx, cy = rng.uniform(-10, 10, 2)
        e, phi = rng.uniform(0, 0.6), rng.uniform(0, math.pi)
        a, s, sv = 10 ** rng.uniform(-1.5, 0.5), 10 ** rng.uniform(1.5, 2.5), rng.uniform(100, 1000)
        p = one(kind, cx, cy, e if kind else 0.0, phi, a, s, sv)
        x, y = rng.uniform(-30, 30, 2)
        J = oracle.jacobian_points(p, [x], [y])[0]
        c, sn = math.cos(phi), math.sin(phi)
        xp, yp = (x - cx) * c + (y - cy) * sn, (y - cy) * c - (x - cx) * sn
        if kind == 0:
            kap = b0(sv) / (2 * math.hypot(x - cx, y - cy))
        elif kind == 2:  # Laplacian of b0 sqrt(a1 x'^2 + a2 y'^2)
            a1, a2 = 1 - e, 1 + e
            R = math.sqrt(a1 * xp * xp + a2 * yp * yp)
            kap = b0(sv) * a1 * a2 * (xp * xp + yp * yp) / (2 * R ** 3)
        else:
            q = 1 - e
            pa = math.sqrt(q * q * (a * a + xp * xp) + yp * yp)
            ps = math.sqrt(q * q * (s * s + xp * xp) + yp * yp)
            kap = 0.5 * b0(sv) * s / (s - a) * (1 / pa - 1 / ps)
        assert J[0, 0] + J[1, 1] == pytest.approx(2 * kap, rel=1e-11, abs=1e-14)
        assert abs(J[0, 1] - J[1, 0]) <= 1e-13 * np.abs(J).max()


def test_sis_point_magnification(oracle):
    """SIS: radial eigenvalue 1, tangential 1 - r theta_E/|theta|, so
    mu = 1 / (1 - r theta_E / |theta|)."""
    rng = np.random.default_rng(13)
    sv = 900.0
    tE = b0(sv)
    p = one(0, 1.0, -2.0, sv=sv)
    x, y = rng.uniform(-60, 60, (2, 40))
    R = np.hypot(x - 1.0, y + 2.0)
    r = 0.7
    obs = dict(x=x, y=y, sigma=np.full(40, 0.01), sys=np.arange(40) // 2,
               dls_ds=np.full(20, r))
    _, mu = oracle.chi2_source(p, obs)
    np.testing.assert_allclose(mu, 1 / (1 - r * tE / R), rtol=1e-12)


def test_sis_source_chi2_closed_form(oracle):
    """Two SIS images of a source at beta0 on the x axis, at beta0 + theta_E
    and beta0 - theta_E; moving the first one outwards by d moves its source
    by d (radial derivative 1), so the barycentre moves by d/2 and
    chi^2_S = (d/2)^2 (mu_1^2 + mu_2^2) / sigma^2 with
    mu_1 = (beta0 + theta_E + d)/(beta0 + d) and mu_2 = (theta_E - beta0)/(-beta0)."""
    sv, beta0, d, sig = 1100.0, 3.0, 0.2, 0.05
    tE = b0(sv)
    p = one(0, sv=sv)
    obs = dict(x=[beta0 + tE + d, beta0 - tE], y=[0.0, 0.0], sigma=[sig, sig], sys=[0, 0],
               dls_ds=[1.0])
    c2, mu = oracle.chi2_source(p, obs)
    mu1 = (beta0 + tE + d) / (beta0 + d)
    mu2 = (tE - beta0) / (-beta0)
    assert mu[0] == pytest.approx(mu1, rel=1e-12) and mu[1] == pytest.approx(mu2, rel=1e-12)
    assert c2 == pytest.approx((d / 2) ** 2 * (mu1 ** 2 + mu2 ** 2) / sig ** 2, rel=1e-10)
    # exact images of one source: chi^2_S vanishes to rounding
    obs["x"] = [beta0 + tE, beta0 - tE]
    c2, _ = oracle.chi2_source(p, obs)
    assert c2 < 1e-20


def test_triangle_magnification_converges_to_point(oracle):
    """Small triangles: the area ratio tends to the SIS point magnification at
    the centroid, with the sign of the image parity (negative inside the
    Einstein radius)."""
    sv = 800.0
    tE = b0(sv)
    p = one(0, sv=sv)
    rng = np.random.default_rng(14)
    for h in (1e-2, 1e-3):
        n = int(round(120 / h)) + 1
        grid = (-60.0, -60.0, h, h, n, n)
        nx = grid[4]
        for _ in range(20):
            R = rng.uniform(0.3 * tE, 2.5 * tE)  # inside the grid (|theta| < 50)
            if abs(R - tE) < 0.1 * tE:
                continue
            ang = rng.uniform(0, 2 * math.pi)
            i = int((R * math.cos(ang) + 60) / h)
            j = int((R * math.sin(ang) + 60) / h)
            assert 0 <= i < nx - 1 and 0 <= j < nx - 1
            t = int(rng.integers(0, 2))
            tri = 2 * (j * (nx - 1) + i) + t
            mu = oracle.tri_magnification(p, grid, [tri], 1.0)[0]
            off = [(0, 0), (1, 0), (1, 1)] if t == 0 else [(0, 0), (1, 1), (0, 1)]
            cx = -60 + (i + sum(o[0] for o in off) / 3) * h
            cy = -60 + (j + sum(o[1] for o in off) / 3) * h
            Rc = math.hypot(cx, cy)
            exp = 1 / (1 - tE / Rc)
            assert np.sign(mu) == np.sign(exp)
            assert mu == pytest.approx(exp, rel=20 * h / abs(Rc - tE))
