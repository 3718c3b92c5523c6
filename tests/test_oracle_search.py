"""Pins of the oracle's triangle search (Fig. 1 relensing).

* exact rational brute force on tiny grids (Python fractions on the FP64
  mapped vertices) gives the same hit sets as the oracle's FP64 predicate;
* with no lens the mapped mesh is the regular image-plane mesh, so the tie
  rule must make every point inside it belong to exactly one triangle, even
  points exactly on shared edges and vertices;
* SIS image counts and positions follow the closed form of Eq. 1 with
  |alpha| = theta_E (two images inside the Einstein radius, one outside),
  converging at O(dx^2);
* the lens-equation residual of found images of a PIEMD cluster shrinks at
  O(dx^2).
"""
import math
from fractions import Fraction as F

import numpy as np
import pytest

from paper_1902_03252_gb300 import workloads as W


def grid_tuple(side, n, cx=0.0, cy=0.0):
    h = side / (n - 1)
    return (cx - side / 2, cy - side / 2, h, h, n, n)


def mapped_vertices(oracle, params, grid, r):
    """beta = theta - r alpha at every node, same IEEE operations as the oracle."""
    x0, y0, dx, dy, nx, ny = grid
    a, _ = oracle.deflect_grid(params, grid)
    ii = np.arange(nx, dtype=float)
    jj = np.arange(ny, dtype=float)
    tx = x0 + ii * dx
    ty = y0 + jj * dy
    bx = tx[None, :] - r * a[..., 0]
    by = ty[:, None] - r * a[..., 1]
    return bx, by


def tri_vertex_nodes(nx, tri):
    cell, t = divmod(tri, 2)
    i, j = cell % (nx - 1), cell // (nx - 1)
    v00 = (i, j)
    return (v00, (i + 1, j), (i + 1, j + 1)) if t == 0 else (v00, (i + 1, j + 1), (i, j + 1))


def exact_inside(A, B, C, P):
    """Exact rational predicate with the stated tie rule."""
    def e(a, b, p):
        return (b[0] - a[0]) * (p[1] - a[1]) - (b[1] - a[1]) * (p[0] - a[0])
    det = e(A, B, C)
    if det == 0:
        return False
    s = 1 if det > 0 else -1
    for a, b in ((A, B), (B, C), (C, A)):
        v = s * e(a, b, P)
        if v > 0:
            continue
        if v < 0:
            return False
        d = (b[0] - a[0], b[1] - a[1]) if s > 0 else (a[0] - b[0], a[1] - b[1])
        if not (d[1] > 0 or (d[1] == 0 and d[0] < 0)):
            return False
    return True


def brute_hits(bx, by, P, nx, ny):
    Pq = (F(P[0]), F(P[1]))
    out = set()
    for tri in range(2 * (nx - 1) * (ny - 1)):
        vs = [(F(bx[j, i]), F(by[j, i])) for (i, j) in tri_vertex_nodes(nx, tri)]
        if exact_inside(*vs, Pq):
            out.add(tri)
    return out


def cluster(n_pot=6, seed=11, half=6.0):
    rng = np.random.default_rng(seed)
    p = W.draw_piemd(rng, n_pot, half, 300.0, 900.0)
    return p


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_exact_rational_brute_force(oracle, seed):
    p = cluster(seed=seed + 20)
    grid = grid_tuple(24.0, 8)
    r = 0.6
    bx, by = mapped_vertices(oracle, p, grid, r)
    rng = np.random.default_rng(seed)
    # sources spread over the mapped mesh, plus points exactly on mapped vertices
    srcs = [(rng.uniform(bx.min(), bx.max()), rng.uniform(by.min(), by.max())) for _ in range(12)]
    srcs += [(bx[2, 3], by[2, 3]), (bx[5, 1], by[5, 1])]
    for P in srcs:
        H, _ = oracle.find_images(p, grid, [P], [r])
        got = {h["tri"] for h in H}
        assert got == brute_hits(bx, by, P, 8, 8), P


def test_tie_rule_partitions_the_plane(oracle):
    """No lens (sigma_v = 0): every point of the mesh, including points exactly
    on shared edges and vertices, lies in exactly one triangle."""
    p = np.array([[0], [0.0], [0.0], [0], [0], [0], [0], [0.0]], dtype=float)
    grid = (-2.0, -2.0, 1.0, 1.0, 5, 5)
    pts = []
    for x in np.arange(-1.5, 1.51, 0.5):        # interior vertices, edge midpoints, centres
        for y in np.arange(-1.5, 1.51, 0.5):
            pts.append((x, y))
    pts += [(-1.25, -1.25), (0.25, 0.75), (1.0, 0.25)]   # on diagonals and verticals
    for P in pts:
        H, _ = oracle.find_images(p, grid, [P], [1.0])
        assert len(H) == 1, (P, [h["tri"] for h in H])
        w = H[0]["w"]
        assert abs(sum(w) - 1) < 1e-15 and min(w) >= 0
        assert abs(H[0]["x"] - P[0]) < 1e-15 and abs(H[0]["y"] - P[1]) < 1e-15


def sis_images(beta, theta_e):
    """Closed-form SIS images from Eq. 1 with |alpha| = theta_E:
    theta = beta_hat (|beta| +/- theta_E), the minus image only if |beta| < theta_E."""
    b = math.hypot(*beta)
    u = (beta[0] / b, beta[1] / b)
    ims = [(u[0] * (b + theta_e), u[1] * (b + theta_e))]
    if b < theta_e:
        ims.append((u[0] * (b - theta_e), u[1] * (b - theta_e)))
    return ims


def split_central(H, grid, cx=0.0, cy=0.0):
    """Hits away from the singular SIS centre, and those within a cell of it.
    The triangles around the centre map onto the whole Einstein circle (the
    deflection is discontinuous there), so they can contain the source."""
    dx = grid[2]
    far = [h for h in H if math.hypot(h["x"] - cx, h["y"] - cy) > 2 * dx]
    near = [h for h in H if math.hypot(h["x"] - cx, h["y"] - cy) <= 2 * dx]
    return far, near


@pytest.mark.parametrize("beta,count", [((2.0, 1.5), 2), ((-4.0, 6.0), 2), ((9.0, 8.0), 1)])
def test_sis_image_count_and_positions(oracle, beta, count):
    w = W.c1()
    p, r = w.params[0], w.notes["dls_ds"]
    grid = w.grids[0].as_tuple()
    H, U = oracle.find_images(p, grid, [beta], [r])
    far, near = split_central(H, grid)
    assert len(far) == count and len(U) == 0
    assert len(near) <= 2
    exp = sis_images(beta, 10.0)
    dx = grid[2]
    for im in exp:
        d = min(math.hypot(h["x"] - im[0], h["y"] - im[1]) for h in far)
        # linear interpolation error in the source plane ~ curvature of the
        # lens map (theta_E/|theta|^2 for the SIS) times the squared cell
        # diagonal, carried to the image plane by the tangential magnification
        t = math.hypot(*im)
        mag = max(1.0, t / abs(t - 10.0))
        assert d < 2 * dx * dx * 10.0 / t ** 2 * mag, (im, d)


def test_sis_convergence_order(oracle):
    """Image positions converge to the closed form at O(dx^2): the RMS error
    over many sources drops by ~4 per halving of dx."""
    w = W.c1()
    p, r = w.params[0], w.notes["dls_ds"]
    rng = np.random.default_rng(12)
    ang = rng.uniform(0, 2 * math.pi, 16)
    rad = rng.uniform(1.0, 7.0, 16)
    betas = list(zip(rad * np.cos(ang), rad * np.sin(ang)))
    rms = []
    for n in (101, 201, 401):
        grid = grid_tuple(60.0, n, 0.013, -0.021)   # offset so no node sits on the centre
        H, _ = oracle.find_images(p, grid, betas, [r] * len(betas))
        sq = []
        for s, beta in enumerate(betas):
            far, _ = split_central([h for h in H if h["src"] == s], grid)
            assert len(far) == 2
            for im in sis_images(beta, 10.0):
                sq.append(min((h["x"] - im[0]) ** 2 + (h["y"] - im[1]) ** 2 for h in far))
        rms.append(math.sqrt(np.mean(sq)))
    slopes = [math.log2(rms[k] / rms[k + 1]) for k in range(2)]
    assert all(1.7 < s < 2.3 for s in slopes), (rms, slopes)


def test_einstein_ring(oracle):
    """beta = 0 gives the Einstein ring (Sect. 2.1): every hit away from the
    centre lies on |theta| = theta_E."""
    w = W.c1()
    p, r = w.params[0], w.notes["dls_ds"]
    grid = grid_tuple(30.0, 121, 0.011, 0.017)
    H, _ = oracle.find_images(p, grid, [(0.0, 0.0)], [r])
    far, _ = split_central(H, grid)
    assert len(far) > 100
    rad = np.array([math.hypot(h["x"], h["y"]) for h in far])
    assert np.all(np.abs(rad - 10.0) < 0.01)


def test_lens_equation_residual_order(oracle):
    """|x - r alpha(x) - beta| of every found image of a PIEMD cluster shrinks
    as dx^2 (refining the grid)."""
    p = cluster(n_pot=5, seed=31, half=8.0)
    r = 0.7
    src = [(0.3, -0.2), (-1.0, 0.8)]
    res = []
    for n in (101, 201, 401):
        grid = grid_tuple(40.0, n)
        H, U = oracle.find_images(p, grid, src, [r, r])
        assert len(U) == 0 and len(H) >= 2
        worst = 0.0
        for h in H:
            ax, ay, _ = oracle.alpha_points(p, [h["x"]], [h["y"]])
            bx, by = h["x"] - r * ax[0], h["y"] - r * ay[0]
            worst = max(worst, math.hypot(bx - src[h["src"]][0], by - src[h["src"]][1]))
        res.append(worst)
    slopes = [math.log2(res[k] / res[k + 1]) for k in range(2)]
    assert all(s > 1.5 for s in slopes), (res, slopes)


def test_degenerate_grids(oracle):
    p = cluster(n_pot=2)
    for grid in [(0.0, 0.0, 1.0, 1.0, 1, 1), (0.0, 0.0, 1.0, 1.0, 1, 5), (0.0, 0.0, 1.0, 1.0, 2, 1)]:
        H, U = oracle.find_images(p, grid, [(0.0, 0.0)], [0.5])
        assert H == [] and U == []
