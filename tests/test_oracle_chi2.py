"""Pins of the oracle's barycentres, chi^2 (Eq. 11) and frozen-assignment
gradient.

* barycentres of SIS images follow from |alpha| = theta_E (Sect. 2.1);
* noiseless observations (the SIS closed-form images) give chi^2 -> 0 at
  O(dx^4) as the grid is refined;
* a system with no predicted image pays the stated penalty per image;
* the dual-number gradient equals central finite differences of the
  frozen-assignment chi^2 (h = 1e-6 relative).
"""
import math

import numpy as np
import pytest

from paper_1902_03252_gb300 import workloads as W


def obs_dict(xy, sys, r, sigma=0.01):
    xy = np.asarray(xy, dtype=float).reshape(-1, 2)
    return dict(x=xy[:, 0].copy(), y=xy[:, 1].copy(), sigma=np.full(len(xy), sigma),
                sys=np.asarray(sys, dtype=np.int32), dls_ds=np.asarray(r, dtype=float))


def sis_images(beta, theta_e):
    b = math.hypot(*beta)
    u = (beta[0] / b, beta[1] / b)
    out = [(u[0] * (b + theta_e), u[1] * (b + theta_e))]
    if b < theta_e:
        out.append((u[0] * (b - theta_e), u[1] * (b - theta_e)))
    return out


def test_barycentre_of_sis_images(oracle):
    """beta = theta - theta_E theta_hat for the SIS; the barycentre is the mean."""
    w = W.c1()
    obs = obs_dict([(12.0, 0.0), (0.0, -5.0), (3.0, 4.0)], [0, 0, 1], [0.7, 0.7])
    b, d = oracle.barycentres(w.params[0], obs)
    np.testing.assert_allclose(b[0], [(2.0 + 0.0) / 2, (0.0 + 5.0) / 2], atol=1e-13)
    np.testing.assert_allclose(b[1], [3.0 - 6.0, 4.0 - 8.0], atol=1e-13)
    assert np.all(d > 0) and np.all(d < 1e-11)


def test_noiseless_chi2_converges_as_dx4(oracle):
    w = W.c1()
    p = w.params[0]
    rng = np.random.default_rng(21)
    ns = 40
    ang = rng.uniform(0, 2 * math.pi, ns)
    rad = rng.uniform(2.5, 6.5, ns)
    xy, sys = [], []
    for s in range(ns):
        for im in sis_images((rad[s] * math.cos(ang[s]), rad[s] * math.sin(ang[s])), 10.0):
            xy.append(im)
            sys.append(s)
    obs = obs_dict(xy, sys, [0.7] * ns)
    chis = []
    for n in (201, 401, 801):
        h = 60.0 / (n - 1)
        grid = (-30.0 + 0.013, -30.0 - 0.021, h, h, n, n)
        res = oracle.chi2(p, grid, obs)
        assert np.all(res["match_tri"] >= 0)
        np.testing.assert_allclose(res["bary"][:, 0], rad * np.cos(ang), atol=1e-12)
        chis.append(res["chi2"])
    slopes = [math.log2(chis[k] / chis[k + 1]) for k in range(2)]
    assert all(3.4 < s < 4.6 for s in slopes), (chis, slopes)


def test_penalty_for_unlensed_system(oracle):
    """A barycentre outside the mapped mesh has no predicted image: each of its
    observed images contributes (L_diag / sigma)^2."""
    w = W.c1()
    grid = w.grids[0].as_tuple()
    obs = obs_dict([(300.0, 0.0), (310.0, 5.0)], [0, 0], [0.7], sigma=0.02)
    res = oracle.chi2(w.params[0], grid, obs)
    diag = math.hypot(255 * grid[2], 255 * grid[3])
    assert res["chi2"] == pytest.approx(2 * (diag / 0.02) ** 2, rel=1e-15)
    assert np.all(res["match_tri"] == -1)


def test_nearest_match_and_frozen_value(oracle):
    """Each observed image takes the nearest predicted image of its system; the
    frozen-assignment chi^2 reproduces the full chi^2."""
    w = W.c1()
    grid = w.grids[0].as_tuple()
    ims = sis_images((2.0, 1.5), 10.0)
    obs = obs_dict([(ims[1][0] + 0.05, ims[1][1]), (ims[0][0], ims[0][1] - 0.04)], [0, 0], [0.7])
    res = oracle.chi2(w.params[0], grid, obs)
    mxy = res["match_xy"]
    assert math.hypot(mxy[0, 0] - ims[1][0], mxy[0, 1] - ims[1][1]) < 0.05
    assert math.hypot(mxy[1, 0] - ims[0][0], mxy[1, 1] - ims[0][1]) < 0.05
    direct = sum(((obs["x"][m] - mxy[m, 0]) ** 2 + (obs["y"][m] - mxy[m, 1]) ** 2) / 0.01 ** 2
                 for m in range(2))
    assert res["chi2"] == pytest.approx(direct, rel=1e-12)
    frozen = oracle.chi2_frozen(w.params[0], grid, obs, res["match_tri"])
    assert frozen == pytest.approx(res["chi2"], rel=1e-9)


def small_model(seed=41):
    rng = np.random.default_rng(seed)
    p = W.draw_piemd(rng, 4, 8.0, 300.0, 800.0)
    return p


def make_obs(oracle, p, grid, n_sys, seed):
    """Observed images: oracle images of random multiply-imaged sources + noise."""
    rng = np.random.default_rng(seed)
    xy, sys, rs = [], [], []
    while len(rs) < n_sys:
        src = rng.uniform(-3, 3, 2)
        r = rng.uniform(0.5, 0.9)
        H, _ = oracle.find_images(p, grid, [src], [r])
        if len(H) < 2:
            continue
        for h in H:
            xy.append((h["x"] + rng.normal(0, 0.01), h["y"] + rng.normal(0, 0.01)))
            sys.append(len(rs))
        rs.append(r)
    return obs_dict(xy, sys, rs)


@pytest.mark.parametrize("seed", [41, 42])
def test_gradient_matches_central_differences(oracle, seed):
    p = small_model(seed)
    grid = (-20.0, -20.0, 40.0 / 149, 40.0 / 149, 150, 150)
    obs = make_obs(oracle, p, grid, 3, seed)
    res = oracle.chi2(p, grid, obs)
    mt = res["match_tri"]
    c, g = oracle.chi2_grad(p, grid, obs, mt)
    assert c == pytest.approx(oracle.chi2_frozen(p, grid, obs, mt), rel=1e-14)
    rows = [1, 2, 3, 4, 5, 7]
    for k in range(p.shape[1]):
        for m, row in enumerate(rows):
            h = 1e-6 * max(abs(p[row, k]), 1e-2)
            pp, pm = p.copy(), p.copy()
            pp[row, k] += h
            pm[row, k] -= h
            fd = (oracle.chi2_frozen(pp, grid, obs, mt) - oracle.chi2_frozen(pm, grid, obs, mt)) / (2 * h)
            scale = max(abs(fd), 1e-6 * max(1.0, abs(c)))
            assert abs(g[k, m] - fd) < 1e-5 * scale + 1e-6, (k, m, g[k, m], fd)


def test_gradient_sis_centre_is_minus_spatial(oracle):
    """Moving a lens by d equals moving every image-plane point by -d: for a lone
    SIS, d chi^2/d x_c + d chi^2/d(obs shift) = 0 is checked through the
    frozen chi^2 with the observations and grid shifted together."""
    w = W.c1()
    p = w.params[0].copy()
    grid = w.grids[0].as_tuple()
    ims = sis_images((2.0, 1.5), 10.0)
    obs = obs_dict([(ims[0][0] + 0.013, ims[0][1] - 0.02), (ims[1][0] - 0.011, ims[1][1] + 0.007)],
                   [0, 0], [0.7])
    res = oracle.chi2(p, grid, obs)
    c, g = oracle.chi2_grad(p, grid, obs, res["match_tri"])
    h = 1e-6
    obs_p = dict(obs, x=obs["x"] - h)
    obs_m = dict(obs, x=obs["x"] + h)
    gp = (grid[0] - h,) + grid[1:]
    gm = (grid[0] + h,) + grid[1:]
    fd = (oracle.chi2_frozen(p, gp, obs_p, res["match_tri"])
          - oracle.chi2_frozen(p, gm, obs_m, res["match_tri"])) / (2 * h)
    assert g[0, 0] == pytest.approx(fd, rel=1e-5)
