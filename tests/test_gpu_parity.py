"""Parity of the CUDA path (through the C ABI) against the FP64 oracle.

Bars (written in each test):
* image sets: bit-exact (sample, source, triangle) sets, in FP64 and in mixed
  precision, apart from pairs the oracle itself classifies as undecidable
  between two FP64 evaluations (reported; expected to be none);
* FP64 deflections: within 1e-12 of sum_k |alpha_k| (transcendental ulps);
* FP32 deflections: within the node's own running error bound;
* positions: 1e-9" (FP64 path) and 1e-4" (mixed; the stated FP32 position
  bound is 2.5e-5");
* chi^2: consistent with those position tolerances.
"""
import json
import math
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1902_03252_gb300 import lt, workloads as W  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lt.load(build_if_missing=True)


def load_obs(cfg):
    with open(os.path.join(GOLDEN, f"obs_{cfg}.json")) as f:
        return json.load(f)


def mixed_cluster(seed, n_pot=20, half=25.0):
    """PIEMD + SIS + SIE mix for kind coverage."""
    rng = np.random.default_rng(seed)
    p = W.draw_piemd(rng, n_pot, half, 100.0, 900.0)
    p[0, ::7] = W.SIS
    p[0, 3::7] = W.SIE
    p[3, 3::7] = rng.uniform(0, 0.3, p[3, 3::7].shape)
    return p


def to_set(imgs):
    return {(int(r["src"]), int(r["tri"])) for r in imgs}


def oracle_set(H):
    return {(h["src"], h["tri"]) for h in H}


def run_find(m, grids, src_xy, r, prec, cap=4096):
    sx = torch.as_tensor(np.asarray(src_xy, dtype=np.float64), device="cuda")
    rr = torch.as_tensor(np.asarray(r, dtype=np.float64), device="cuda")
    out, n = m.find_images(grids, sx, rr, precision=prec, capacity=cap)
    st, stats = m.sync()
    return st, stats, lt.images_to_numpy(out, n), n.cpu().numpy()


# ------------------------------------------------------------------ deflection
@pytest.mark.parametrize("seed", [1, 2])
def test_deflect_fp64_matches_oracle(oracle, seed):
    p = mixed_cluster(seed)
    grid = (-40.0, -37.0, 80.0 / 211, 74.0 / 187, 212, 188)
    m = lt.Model(p.shape[1], 1)
    m.set_params(p[None])
    a = m.deflect_grid(grid, precision=lt.FP64).cpu().numpy()
    ref, asum = oracle.deflect_grid(p, grid, n_threads=4)
    err = np.abs(a - ref).max(axis=-1)
    assert np.all(err <= 1e-12 * (asum + 1.0)), err.max()


def test_deflect_fp64_bit_exact_correctly_rounded(oracle):
    """SIS and axis-aligned SIE (phi = 0: cos and sin exactly 1 and 0) use only
    correctly rounded FP64 operations (+, -, *, /, sqrt) in the oracle's order,
    so the FP64 grid, superposed in potential index order (Sect. 2.2.2),
    equals the oracle bit for bit.  300 potentials span several staged chunks;
    some centres fall exactly on nodes (the zero-distance branch)."""
    rng = np.random.default_rng(23)
    n = 300
    p = np.zeros((W.N_ROWS, n))
    p[0] = rng.choice([W.SIS, W.SIE], n)
    p[1] = rng.uniform(-40.0, 40.0, n)
    p[2] = rng.uniform(-40.0, 40.0, n)
    p[1, :20] = rng.integers(-80, 81, 20) * 0.5  # on nodes of the grid below
    p[2, :20] = rng.integers(-80, 81, 20) * 0.5
    p[3] = np.where(p[0] == W.SIE, rng.uniform(0.0, 0.6, n), 0.0)
    p[7] = rng.uniform(50.0, 400.0, n)
    p[7, :2] = [900.0, 700.0]
    grid = (-40.0, -40.0, 0.5, 0.5, 161, 161)
    m = lt.Model(n, 1)
    m.set_params(p[None])
    a = m.deflect_grid(grid, precision=lt.FP64).cpu().numpy()
    assert m.sync()[0] == lt.LT_OK
    m.close()
    ref, _ = oracle.deflect_grid(p, grid, n_threads=4)
    np.testing.assert_array_equal(a, ref)


@pytest.mark.parametrize("seed", [3, 4, 5])
def test_deflect_mixed_within_running_bound(oracle, seed):
    p = mixed_cluster(seed, n_pot=40)
    grid = (-50.0, -50.0, 100.0 / 299, 100.0 / 299, 300, 300)
    m = lt.Model(p.shape[1], 1)
    m.set_params(p[None])
    a, e = m.deflect_grid(grid, precision=lt.MIXED, with_error=True)
    a, e = a.cpu().numpy().astype(np.float64), e.cpu().numpy().astype(np.float64)
    ref, _ = oracle.deflect_grid(p, grid, n_threads=4)
    d = np.abs(a - ref).max(axis=-1)
    ratio = d / e
    print(f"FP32 error / running bound: max {ratio.max():.3g}, median {np.median(ratio):.3g}")
    assert np.all(np.isfinite(e)) and np.all(e > 0)
    assert ratio.max() <= 1.0


def test_deflect_bound_adversarial(oracle):
    """The running FP32 bound on the hardest inputs: PIEMD with ellipticity
    up to 0.9 (atanh's sensitivity grows as 1/q^2), cores from 1e-3" to 3",
    cuts from 1.5 to 1e4 times the core, SIE with eps up to 0.9, SIS; nodes
    on the potentials' centres, on their symmetry axes and within a core
    radius of them, far from the grid origin (|theta| up to 200")."""
    rng = np.random.default_rng(77)
    n = 60
    p = np.zeros((8, n))
    p[0] = rng.choice([W.SIS, W.PIEMD, W.SIE], n, p=[0.2, 0.6, 0.2])
    p[1:3] = rng.uniform(-150, 150, (2, n))
    p[3] = np.where(p[0] == W.SIS, 0.0, rng.uniform(0.0, 0.9, n))
    p[4] = rng.uniform(0, np.pi, n)
    p[5] = 10 ** rng.uniform(-3, 0.5, n)
    p[6] = p[5] * 10 ** rng.uniform(np.log10(1.5), 4, n)
    p[7] = 10 ** rng.uniform(1.5, 3.1, n)
    # nodes: each potential's centre, points on its rotated axes at 0.3, 1, 3
    # core radii and 1, 10 arcsec, snapped to a fine grid around it
    xs, ys = [], []
    for k in range(n):
        c, s = np.cos(p[4, k]), np.sin(p[4, k])
        for rad in (0.0, 0.3 * p[5, k], p[5, k], 3 * p[5, k], 1.0, 10.0):
            for ax in ((c, s), (-s, c)):
                xs.append(p[1, k] + rad * ax[0])
                ys.append(p[2, k] + rad * ax[1])
    xs, ys = np.asarray(xs), np.asarray(ys)
    # one grid per potential neighbourhood would be many calls: evaluate the
    # points as a 1-row grid each (a grid's node coordinates are x0 + i dx)
    m = lt.Model(n, 1)
    m.set_params(p[None])
    worst = 0.0
    for x, y in zip(xs, ys):
        grid = (float(x) - 1e-3, float(y), 1e-3, 1.0, 3, 1)
        a, e = m.deflect_grid(grid, precision=lt.MIXED, with_error=True)
        a = a.cpu().numpy().astype(np.float64).reshape(-1, 2)
        e = e.cpu().numpy().astype(np.float64).reshape(-1)
        gx = grid[0] + np.arange(3) * grid[2]
        ax, ay, _ = oracle.alpha_points(p, gx, np.full(3, grid[1]))
        d = np.maximum(np.abs(a[:, 0] - ax), np.abs(a[:, 1] - ay))
        # 1e30 only where a node's FP32 coordinates fall on an SIS/SIE centre
        assert np.all(np.isfinite(e)) and np.all(d <= e), (x, y, d, e)
        fin = e < 1e29
        if fin.any():
            worst = max(worst, float((d[fin] / e[fin]).max()))
    assert m.sync()[0] == lt.LT_OK
    print(f"adversarial nodes: largest error / bound {worst:.3g}")
    m.close()


def test_deflect_range_reduction_boundaries(oracle):
    """Nodes close to PIEMD cores, where the atan and atanh arguments cross
    their range-reduction thresholds (t^2 = 1, t^2 = 1/4) between
    neighbouring rows, so that one node of a thread's pair takes the reduced
    form and the other the polynomial: every node within its bound, in every
    launch shape (paired, odd and single nodes), with identical values."""
    rng = np.random.default_rng(77)
    n = 12
    p = np.zeros((8, n))
    p[0] = W.PIEMD
    p[1] = rng.uniform(-1.5, 1.5, n)
    p[2] = rng.uniform(-1.5, 1.5, n)
    p[3] = rng.uniform(0.05, 0.6, n)
    p[4] = rng.uniform(0.0, np.pi, n)
    p[5] = rng.uniform(0.03, 0.3, n)
    p[6] = rng.uniform(20.0, 150.0, n)
    p[7] = rng.uniform(150.0, 900.0, n)
    grid = (-2.0, -1.9, 4.0 / 160, 3.8 / 153, 161, 154)
    ref, _ = oracle.deflect_grid(p, grid, n_threads=4)
    m = lt.Model(n, 1)
    m.set_params(p[None])
    first = None
    for shape in range(m.num_shapes()):
        m.set_shape(shape)
        a, e = m.deflect_grid(grid, precision=lt.MIXED, with_error=True)
        assert m.sync()[0] == lt.LT_OK
        a, e = a.cpu().numpy().astype(np.float64), e.cpu().numpy().astype(np.float64)
        d = np.abs(a - ref).max(axis=-1)
        assert np.all(np.isfinite(e)) and (d / e).max() <= 1.0, (shape, (d / e).max())
        if first is None:
            first = (a, e)
        else:
            np.testing.assert_array_equal(a, first[0])
            np.testing.assert_array_equal(e, first[1])
    m.close()


@pytest.mark.parametrize("shape", range(8))
def test_deflect_every_shape_within_bound(oracle, shape):
    """Every launch shape of the FP32 deflection on 300 potentials of all
    three kinds -- more than one staged chunk of 256 -- over a grid whose node
    count is not a multiple of any work item: within the running bound, and
    values and bound identical across shapes."""
    rng = np.random.default_rng(40 + shape)
    p = W.draw_piemd(rng, 300, 40.0, 50.0, 900.0)
    p[0, ::5] = W.SIS
    p[0, 2::5] = W.SIE
    p[3, 2::5] = rng.uniform(0, 0.3, p[3, 2::5].shape)
    grid = (-45.0, -41.0, 90.0 / 250, 82.0 / 231, 251, 232)
    m = lt.Model(p.shape[1], 1)
    assert m._lib.lt_num_shapes() == 8
    m.set_params(p[None])
    m.set_shape(shape)
    a, e = m.deflect_grid(grid, precision=lt.MIXED, with_error=True)
    m.set_shape(0)
    a1, e1 = m.deflect_grid(grid, precision=lt.MIXED, with_error=True)
    assert m.sync()[0] == lt.LT_OK
    a, e = a.cpu().numpy().astype(np.float64), e.cpu().numpy().astype(np.float64)
    ref, _ = oracle.deflect_grid(p, grid, n_threads=4)
    d = np.abs(a - ref).max(axis=-1)
    assert np.all(np.isfinite(e)) and np.all(e > 0)
    assert (d / e).max() <= 1.0, (d / e).max()
    # a node's arithmetic does not depend on the shape (a thread's rows share
    # only its column's translation): the same values and bounds, bit for bit
    np.testing.assert_array_equal(a, a1.cpu().numpy().astype(np.float64))
    np.testing.assert_array_equal(e, e1.cpu().numpy().astype(np.float64))


def test_deflect_grids_in_turn_match_fresh_models():
    """The single-grid path keeps the FP32 node-coordinate table of its last
    grid: alternating grids (different origin, spacing and shape) must give
    bit for bit what a fresh model gives for each."""
    p = mixed_cluster(31, n_pot=25)
    grids = [(-30.0, -30.0, 60.0 / 199, 60.0 / 199, 200, 200),
             (-29.0, -31.0, 0.25, 0.3, 237, 181),
             (-30.0, -30.0, 60.0 / 199, 60.0 / 199, 200, 200)]
    fresh = []
    for g in grids[:2]:
        m = lt.Model(p.shape[1], 1)
        m.set_params(p[None])
        a, e = m.deflect_grid(g, precision=lt.MIXED, with_error=True)
        fresh.append((a.cpu().numpy(), e.cpu().numpy()))
        m.close()
    m = lt.Model(p.shape[1], 1)
    m.set_params(p[None])
    for k, g in enumerate(grids):
        a, e = m.deflect_grid(g, precision=lt.MIXED, with_error=True)
        ref = fresh[0 if k != 1 else 1]
        np.testing.assert_array_equal(a.cpu().numpy(), ref[0])
        np.testing.assert_array_equal(e.cpu().numpy(), ref[1])
    assert m.sync()[0] == lt.LT_OK
    m.close()


def test_deflect_c2_full_size_sampled(oracle):
    """The 2000^2, 100-PIEMD grid in the benchmark's launch configuration:
    every node within its bound on a sampled subset, FP64 on the same subset."""
    w = W.c2()
    grid = w.grids[0].as_tuple()
    m = lt.Model(w.n_pot, 1)
    m.set_params(w.params)
    a, e = m.deflect_grid(grid, precision=lt.MIXED, with_error=True)
    a64 = m.deflect_grid(grid, precision=lt.FP64)
    rng = np.random.default_rng(7)
    idx = rng.integers(0, 2000 * 2000, 4000)
    jj, ii = np.divmod(idx, 2000)
    x = grid[0] + ii * grid[2]
    y = grid[1] + jj * grid[3]
    rx, ry, asum = oracle.alpha_points(w.params[0], x, y)
    A = a.reshape(-1, 2).cpu().numpy()[idx].astype(np.float64)
    E = e.reshape(-1).cpu().numpy()[idx].astype(np.float64)
    A64 = a64.reshape(-1, 2).cpu().numpy()[idx]
    d32 = np.maximum(np.abs(A[:, 0] - rx), np.abs(A[:, 1] - ry))
    assert np.all(d32 <= E), (d32 / E).max()
    d64 = np.maximum(np.abs(A64[:, 0] - rx), np.abs(A64[:, 1] - ry))
    assert np.all(d64 <= 1e-12 * (asum + 1.0))


# -------------------------------------------------------------- image search
def check_images(oracle, p, grid, src, r, prec, pos_tol, exact_ties=False):
    """exact_ties: the lens uses only correctly rounded operations (SIS), so
    even pairs the oracle flags as ties must agree bit for bit."""
    m = lt.Model(p.shape[1], 1)
    m.set_params(p[None])
    st, stats, imgs, n = run_find(m, [grid], np.asarray(src)[None], np.asarray(r)[None], prec)
    assert st == lt.LT_OK
    H, U = oracle.find_images(p, grid, src, r, n_threads=4)
    und = {(u["src"], u["tri"]) for u in U}
    got, exp = to_set(imgs[0]), oracle_set(H)
    diff = got ^ exp
    assert diff <= und, (sorted(diff - und)[:10], len(got), len(exp))
    if exact_ties:
        assert not diff, sorted(diff)[:10]
    else:
        assert not und, f"{len(und)} FP64-undecidable pairs"
    ref = {(h["src"], h["tri"]): h for h in H}
    worst = 0.0
    for rec in imgs[0]:
        h = ref[(int(rec["src"]), int(rec["tri"]))]
        worst = max(worst, abs(rec["x"] - h["x"]), abs(rec["y"] - h["y"]))
    assert worst <= pos_tol, worst
    # sorted by (src, tri)
    keys = [(int(r_["src"]), int(r_["tri"])) for r_ in imgs[0]]
    assert keys == sorted(keys)
    return stats, worst


@pytest.mark.parametrize("prec,tol", [(lt.FP64, 1e-9), (lt.MIXED, 1e-4)])
def test_find_images_sis(oracle, prec, tol):
    w = W.c1()
    g = w.grids[0].as_tuple()
    # (0, 0) is the Einstein ring: on this grid, symmetric about the lens,
    # mapped cell diagonals pass exactly through the source (tie rule)
    src = [(2.0, 1.5), (0.0, 0.0), (-4.0, 6.0), (9.0, 8.0), (30.0, -2.0)]
    check_images(oracle, w.params[0], g, src, [0.7] * len(src), prec, tol, exact_ties=True)


def degenerate_lens():
    """The c1 SIS with zero-mass SIS, SIE (phi = 0) and PIEMD potentials and a
    light SIS centred exactly on grid nodes next to the images of the source
    (2, 1.5) at r = 0.7 (near (-6.0, -4.5) and (10.0, 7.5)).  Every operation
    of this lens is correctly rounded (a zero-mass PIEMD adds exactly zero)."""
    w = W.c1()
    g = w.grids[0].as_tuple()
    x0, y0, dx, dy = g[:4]
    node = lambda i, j: (x0 + i * dx, y0 + j * dy)  # the grid's own node formula
    i1, j1 = round((-6.0 - x0) / dx), round((-4.5 - y0) / dy)
    i2, j2 = round((10.0 - x0) / dx), round((7.5 - y0) / dy)
    spots = [(W.SIS, node(i1, j1), 0.0), (W.PIEMD, node(i1 + 1, j1), 0.0),
             (W.SIE, node(i2, j2), 0.0), (W.SIS, node(i2 + 2, j2 - 1), 40.0)]
    p = np.zeros((W.N_ROWS, 1 + len(spots)))
    p[:, 0] = w.params[0, :, 0]
    for k, (kind, (x, y), sv) in enumerate(spots, start=1):
        p[0, k], p[1, k], p[2, k], p[7, k] = kind, x, y, sv
        if kind != W.SIS:
            p[3, k] = 0.3
        if kind == W.PIEMD:
            p[5, k], p[6, k] = 0.5, 20.0
    centres = [(i1, j1), (i2, j2), (i2 + 2, j2 - 1)]  # SIS / SIE centres on nodes
    return p, g, centres


def test_deflect_degenerate_potentials(oracle):
    """Nodes on SIS / SIE centres (zero-mass ones included): the FP32
    deflection is finite there and equals the oracle's limit value, and the
    node's running bound is the 1e30 that marks no bound (never NaN), so no
    test is certified with it; every other node stays within its own bound."""
    p, g, centres = degenerate_lens()
    m = lt.Model(p.shape[1], 1)
    m.set_params(p[None])
    a, e = m.deflect_grid(g, precision=lt.MIXED, with_error=True)
    assert m.sync()[0] == lt.LT_OK
    a, e = a.cpu().numpy().astype(np.float64), e.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(a)) and not np.any(np.isnan(e))
    on = np.zeros(e.shape, bool)
    for i, j in centres:
        on[j, i] = True
    assert np.all(e[on] == float(np.float32(1e30))) and np.all(e[~on] < 1.0)
    ref, _ = oracle.deflect_grid(p, g, n_threads=4)
    d = np.abs(a - ref).max(axis=-1)
    assert np.all(d[~on] <= e[~on]), (d[~on] / e[~on]).max()
    # on the centre nodes the massive SIS alone contributes (0 at its centre,
    # exactly as the oracle); the difference is the FP32 rounding of the rest
    assert np.all(d[on] <= 1e-4)


@pytest.mark.parametrize("prec,tol", [(lt.FP64, 1e-9), (lt.MIXED, 1e-4)])
def test_find_images_degenerate_potentials(oracle, prec, tol):
    """Triangles with a vertex on a potential's centre (infinite FP32 bound)
    go to the FP64 stage; the image set still equals the oracle's, ties
    included (the lens's operations are all correctly rounded)."""
    p, g, _ = degenerate_lens()
    stats, _ = check_images(oracle, p, g, [(2.0, 1.5), (-1.0, 3.0)], [0.7, 0.7], prec, tol,
                            exact_ties=True)
    if prec == lt.MIXED:
        assert stats["fp64_items"] > 0, stats


@pytest.mark.parametrize("prec,tol", [(lt.FP64, 1e-9), (lt.MIXED, 1e-4)])
def test_find_images_zero_ratio(oracle, prec, tol):
    """D_ls/D_s = 0 (a source in the lens plane): beta = theta exactly, so the
    image is the source position itself, decided by the tie rule where the
    source sits on a node -- here nodes on SIS / SIE centres, whose infinite
    FP32 bound (1e30) leaves the test to the FP64 stage."""
    p, g, centres = degenerate_lens()
    x0, y0, dx, dy = g[:4]
    on = [(x0 + i * dx, y0 + j * dy) for i, j in centres]
    src = [(2.0, 1.5), on[0], on[1], on[2], (3.3, -7.1), (2.0, 1.5)]
    r = [0.0, 0.0, 0.0, 0.0, 0.0, 0.7]
    check_images(oracle, p, g, src, r, prec, tol, exact_ties=True)


@pytest.mark.parametrize("prec", [lt.FP64, lt.MIXED])
def test_invalid_sources_are_latched(oracle, prec):
    """A negative or NaN ratio, or a non-finite position, is outside the
    input domain: LT_ERR_NONFINITE is latched and that source has no images,
    while the valid sources' images equal the oracle's."""
    p, g, _ = degenerate_lens()
    src = [(2.0, 1.5), (2.0, 1.5), (-1.0, 3.0), (np.nan, 1.0), (-1.0, 3.0)]
    r = [0.7, -0.5, np.nan, 0.7, 0.7]
    valid = [0, 4]
    m = lt.Model(p.shape[1], 1)
    m.set_params(p[None])
    st, stats, imgs, n = run_find(m, [g], np.asarray(src)[None], np.asarray(r)[None], prec)
    assert st == lt.LT_ERR_NONFINITE
    got = to_set(imgs[0])
    assert {s_ for s_, _ in got} <= set(valid)
    H, _ = oracle.find_images(p, g, [src[k] for k in valid], [r[k] for k in valid], n_threads=4)
    assert got == {(valid[h["src"]], h["tri"]) for h in H}


@pytest.mark.parametrize("seed", [11, 12])
@pytest.mark.parametrize("prec,tol", [(lt.FP64, 1e-9), (lt.MIXED, 1e-4)])
def test_find_images_cluster(oracle, seed, prec, tol):
    p = mixed_cluster(seed, n_pot=30, half=20.0)
    grid = (-30.0, -30.0, 60.0 / 333, 60.0 / 333, 334, 334)
    rng = np.random.default_rng(seed)
    src = rng.uniform(-8, 8, (12, 2))
    r = rng.uniform(0.3, 0.9, 12)
    stats, worst = check_images(oracle, p, grid, src, r, prec, tol)
    print(f"prec {prec}: stats {stats}, worst position error {worst:.3g}")


@pytest.mark.parametrize("prec,tol", [(lt.FP64, 1e-9), (lt.MIXED, 1e-4)])
def test_find_images_many_sources(oracle, prec, tol):
    """600 sources: more than one staged chunk of sources in the search
    kernel (256 at a time), against the oracle's image set and positions."""
    p = mixed_cluster(21, n_pot=25, half=20.0)
    grid = (-30.0, -30.0, 60.0 / 299, 60.0 / 299, 300, 300)
    rng = np.random.default_rng(21)
    src = rng.uniform(-10, 10, (600, 2))
    r = rng.uniform(0.3, 0.9, 600)
    m = lt.Model(p.shape[1], 1, hit_capacity=1 << 15)
    m.set_params(p[None])
    st, stats, imgs, n = run_find(m, [grid], src[None], r[None], prec, cap=1 << 15)
    assert st == lt.LT_OK, (st, stats)
    H, U = oracle.find_images(p, grid, src, r, n_threads=8, capacity=1 << 15)
    assert not U
    assert to_set(imgs[0]) == oracle_set(H)
    ref = {(h["src"], h["tri"]): h for h in H}
    worst = max(max(abs(rec["x"] - ref[(int(rec["src"]), int(rec["tri"]))]["x"]),
                    abs(rec["y"] - ref[(int(rec["src"]), int(rec["tri"]))]["y"])) for rec in imgs[0])
    assert worst <= tol, worst
    m.close()


# ------------------------------------------------------------------- chi^2
def check_chi2(oracle, w, o, prec, grids=None, graph=False):
    grids = grids or [g.as_tuple() for g in w.grids]
    obs = lt.Observations.from_dict(o)
    m = lt.Model(w.n_pot, w.batch)
    m.set_params(w.params)
    c2 = m.chi2(grids, obs, precision=prec, graph=graph)
    st, stats = m.sync()
    assert st == lt.LT_OK, st
    mt, mxy, bary = m.last_matches(len(o["x"]), len(o["dls_ds"]))
    c2, mt, mxy, bary = c2.cpu().numpy(), mt.cpu().numpy(), mxy.cpu().numpy(), bary.cpu().numpy()
    tol = 1e-4 if prec == lt.MIXED else 1e-9
    for b in range(w.batch):
        ref = oracle.chi2(w.params[b], grids[b], o, n_threads=4)
        assert ref["n_undecidable"] == 0
        np.testing.assert_allclose(bary[b], ref["bary"], rtol=0, atol=1e-11)
        assert np.array_equal(mt[b], ref["match_tri"]), (b, mt[b], ref["match_tri"])
        ok = ref["match_tri"] >= 0
        assert np.all(np.abs(mxy[b][ok] - ref["match_xy"][ok]) <= tol)
        res = np.hypot(np.asarray(o["x"]) - ref["match_xy"][:, 0],
                       np.asarray(o["y"]) - ref["match_xy"][:, 1])
        ctol = np.sum((2 * res * tol * 1.5 + 2 * tol * tol) / np.asarray(o["sigma"]) ** 2)
        assert abs(c2[b] - ref["chi2"]) <= ctol + 1e-12 * ref["chi2"], (b, c2[b], ref["chi2"])
    return c2, stats


@pytest.mark.parametrize("prec", [lt.FP64, lt.MIXED])
def test_chi2_c1(oracle, prec):
    check_chi2(oracle, W.c1(), load_obs("c1"), prec)


@pytest.mark.parametrize("prec", [lt.FP64, lt.MIXED])
def test_chi2_c4(oracle, prec):
    check_chi2(oracle, W.c4(), load_obs("c4"), prec)


@pytest.mark.parametrize("prec", [lt.FP64, lt.MIXED])
def test_chi2_invalid_system_is_latched(oracle, prec):
    """A system with a negative D_ls/D_s (outside the input domain) gets no
    predicted images: LT_ERR_NONFINITE is latched, its observed images take
    the penalty (L_diag/sigma)^2 of an unlensed system, and every other
    system's matches and chi^2 terms equal the oracle's."""
    w = W.c4()
    o = load_obs("c4")
    bad = 3
    ob = dict(o, dls_ds=[(-0.5 if s_ == bad else r_) for s_, r_ in enumerate(o["dls_ds"])])
    m = lt.Model(w.n_pot, 1)
    m.set_params(w.params)
    grid = w.grids[0].as_tuple()
    c2 = m.chi2([grid], lt.Observations.from_dict(ob), precision=prec)
    st, _ = m.sync()
    assert st == lt.LT_ERR_NONFINITE
    mt, mxy, _ = m.last_matches(len(o["x"]), len(o["dls_ds"]))
    c2, mt, mxy = float(c2.cpu().numpy()[0]), mt.cpu().numpy()[0], mxy.cpu().numpy()[0]
    ref = oracle.chi2(w.params[0], grid, o, n_threads=4)
    sys_ = np.asarray(o["sys"])
    assert np.all(mt[sys_ == bad] < 0)
    assert np.array_equal(mt[sys_ != bad], ref["match_tri"][sys_ != bad])
    x, y, sig = np.asarray(o["x"]), np.asarray(o["y"]), np.asarray(o["sigma"])
    res2 = (x - ref["match_xy"][:, 0]) ** 2 + (y - ref["match_xy"][:, 1]) ** 2
    diag = math.hypot((grid[4] - 1) * grid[2], (grid[5] - 1) * grid[3])
    pen = diag ** 2 / sig ** 2
    term = np.where(ref["match_tri"] >= 0, res2 / sig ** 2, pen)
    expect = float(np.sum(np.where(sys_ == bad, pen, term)))
    tol = 1e-4 if prec == lt.MIXED else 1e-9
    ok = (sys_ != bad) & (ref["match_tri"] >= 0)
    ctol = np.sum((2 * np.sqrt(res2[ok]) * tol * 1.5 + 2 * tol * tol) / sig[ok] ** 2)
    assert abs(c2 - expect) <= ctol + 1e-12 * expect, (c2, expect)


def test_chi2_batched_uneven(oracle):
    """Eight perturbed samples on grids of uneven sizes in one call."""
    w = W.c3(batch=8)
    o = load_obs("c3")
    rng = np.random.default_rng(3)
    grids = [W.Grid.square(200.0, int(n)).as_tuple() for n in rng.integers(300, 700, 8)]
    check_chi2(oracle, w, o, lt.MIXED, grids=grids)


def test_chunked_batch_matches_one_chunk(monkeypatch):
    """A node-workspace budget of 2 MB puts every sample of the batch in a
    chunk of its own (separate launches, item tables, FP64 node tables):
    the results equal those of one chunk for the whole batch, bit for bit."""
    w = W.c3(batch=8)
    o = load_obs("c3")
    rng = np.random.default_rng(5)
    grids = [W.Grid.square(200.0, int(n)).as_tuple() for n in rng.integers(300, 700, 8)]
    obs = lt.Observations.from_dict(o)
    res = []
    for budget in (None, "2"):
        if budget:
            monkeypatch.setenv("LT_WORKSPACE_MB", budget)
        m = lt.Model(w.n_pot, w.batch)
        m.set_params(w.params)
        c2, g = m.chi2_grad(grids, obs)
        st, stats = m.sync()
        assert st == lt.LT_OK
        mt, mxy, _ = m.last_matches(len(o["x"]), len(o["dls_ds"]))
        res.append((c2.cpu().numpy(), g.cpu().numpy(), mt.cpu().numpy(), mxy.cpu().numpy()))
        m.close()
    for a, b in zip(res[0], res[1]):
        np.testing.assert_array_equal(a, b)


def test_graph_replay_matches_direct(oracle):
    w = W.c4()
    o = load_obs("c4")
    obs = lt.Observations.from_dict(o)
    m = lt.Model(w.n_pot, 1)
    m.set_params(w.params)
    g = [w.grids[0].as_tuple()]
    direct = m.chi2(g, obs, precision=lt.MIXED).clone()
    outs = [m.chi2(g, obs, precision=lt.MIXED, graph=True).clone() for _ in range(3)]
    assert m.sync()[0] == lt.LT_OK
    for o_ in outs:
        assert torch.equal(o_, direct)


def test_back_to_back_evaluations_match_isolated(oracle):
    """Evaluations queued back to back on one stream, each with new device
    parameters, without a host synchronisation between them (the kernels of
    the chain launch programmatically, each waiting for its predecessor at its
    start), give the same chi^2 as the same evaluations run one at a time."""
    w = W.c4()
    o = load_obs("c4")
    obs = lt.Observations.from_dict(o)
    m = lt.Model(w.n_pot, 1)
    g = [w.grids[0].as_tuple()]
    base = torch.as_tensor(w.params, dtype=torch.float64, device="cuda")
    params = []
    for k in range(12):
        p = base.clone()
        p[0, 1, k % w.n_pot] += 0.05 * (k + 1)  # move one potential's centre
        p[0, 7, (3 * k) % w.n_pot] *= 1.0 + 0.01 * k  # and another's sigma_v
        params.append(p)
    outs = torch.empty(len(params), dtype=torch.float64, device="cuda")
    for k, p in enumerate(params):
        m.set_params(p)
        m.chi2(g, obs, precision=lt.MIXED, out=outs[k:k + 1])
    queued = outs.cpu().numpy()
    assert m.sync()[0] == lt.LT_OK
    for k, p in enumerate(params):
        m.set_params(p)
        one = m.chi2(g, obs, precision=lt.MIXED).clone()
        torch.cuda.synchronize()
        assert one.item() == queued[k], (k, one.item(), queued[k])
    assert len(set(queued.tolist())) > 1  # the evaluations differ from one another
    m.close()


# -------------------------------------------------------------- edge cases
def test_edge_cases(oracle):
    w = W.c1()
    m = lt.Model(1, 1)
    m.set_params(w.params)
    # a 1 x 1 grid and a 1-row grid have no triangles
    for g in [(0.0, 0.0, 1.0, 1.0, 1, 1), (0.0, 0.0, 1.0, 1.0, 7, 1)]:
        st, stats, imgs, n = run_find(m, [g], [[(0.5, 0.5)]], [[0.7]], lt.MIXED)
        assert st == lt.LT_OK and n[0] == 0
    # no sources
    out, n = m.find_images([w.grids[0]], None, None, precision=lt.MIXED, capacity=16)
    assert m.sync()[0] == lt.LT_OK and int(n.cpu()[0]) == 0
    # capacity overflow is reported, and the true count returned
    st, stats, imgs, n = run_find(m, [w.grids[0]], [[(0.0, 0.0)]], [[0.7]], lt.MIXED, cap=8)
    assert st == lt.LT_ERR_OVERFLOW and n[0] > 8 and len(imgs[0]) == 8
    # invalid parameters are latched
    bad = w.params.copy()
    bad[0, 7, 0] = np.nan
    m.set_params(bad)
    assert m.sync()[0] == lt.LT_ERR_NONFINITE
    bad = W.c2().params[:, :, :3].copy()
    bad[0, 5, 1] = -1.0  # negative core radius
    m3 = lt.Model(3, 1)
    m3.set_params(bad)
    assert m3.sync()[0] == lt.LT_ERR_NONFINITE
    # argument errors
    with pytest.raises(lt.LTError):
        m.deflect_grid((0.0, 0.0, -1.0, 1.0, 4, 4))
    with pytest.raises(lt.LTError):
        m.deflect_grid((0.0, 0.0, 1.0, 1.0, 4, 4), sample=3)


# ---------------------------------------------------------------- gradient
def grad_close(g, ref):
    """1e-3 relative per component, with a floor of 1e-6 of the largest
    component of the same sample (components that cancel to ~0)."""
    floor = 1e-6 * np.abs(ref).max()
    err = np.abs(g - ref)
    return np.all(err <= 1e-3 * np.abs(ref) + floor), (err / (np.abs(ref) + floor)).max()


@pytest.mark.parametrize("prec", [lt.MIXED, lt.FP64])
def test_gradient_matches_oracle_c4(oracle, prec):
    """d chi^2 / d(x, y, e, phi, r_core, sigma_v) of 100 PIEMD on the 1000^2
    grid with 20 systems: the adjoint against the oracle's dual-number
    gradient (same frozen assignment)."""
    w = W.c4()
    o = load_obs("c4")
    obs = lt.Observations.from_dict(o)
    m = lt.Model(w.n_pot, 1)
    m.set_params(w.params)
    grid = w.grids[0].as_tuple()
    c2, g = m.chi2_grad([grid], obs, precision=prec)
    assert m.sync()[0] == lt.LT_OK
    mt, _, _ = m.last_matches(len(o["x"]), len(o["dls_ds"]))
    mt = mt.cpu().numpy()[0]
    ref = oracle.chi2(w.params[0], grid, o, n_threads=4)
    assert np.array_equal(mt, ref["match_tri"])
    rc, rg = oracle.chi2_grad(w.params[0], grid, o, ref["match_tri"])
    ok, worst = grad_close(g.cpu().numpy()[0], rg)
    print(f"gradient worst relative error {worst:.3g}")
    assert ok, worst


def test_gradient_matches_central_differences(oracle):
    """The adjoint against FP64 central differences (h = 1e-6 relative) of the
    oracle's frozen-assignment chi^2 on a small mixed-kind model."""
    p = mixed_cluster(21, n_pot=12, half=15.0)
    grid = (-25.0, -25.0, 50.0 / 249, 50.0 / 249, 250, 250)
    rng = np.random.default_rng(21)
    xy, sys, rs = [], [], []
    while len(rs) < 4:
        src, r = rng.uniform(-5, 5, 2), rng.uniform(0.4, 0.9)
        H, _ = oracle.find_images(p, grid, [src], [r])
        if len(H) < 2:
            continue
        for h in H:
            xy.append((h["x"] + rng.normal(0, 0.01), h["y"] + rng.normal(0, 0.01)))
            sys.append(len(rs))
        rs.append(r)
    xy = np.array(xy)
    o = dict(x=xy[:, 0], y=xy[:, 1], sigma=np.full(len(xy), 0.01), sys=np.array(sys),
             dls_ds=np.array(rs))
    m = lt.Model(p.shape[1], 1)
    m.set_params(p[None])
    c2, g = m.chi2_grad([grid], lt.Observations.from_dict(o), precision=lt.MIXED)
    assert m.sync()[0] == lt.LT_OK
    mt = m.last_matches(len(xy), len(rs))[0].cpu().numpy()[0]
    g = g.cpu().numpy()[0]
    fd = np.zeros_like(g)
    for k in range(p.shape[1]):
        for c, row in enumerate([1, 2, 3, 4, 5, 7]):
            if p[0, k] == W.SIS and row in (3, 4, 5):
                continue
            if p[0, k] == W.SIE and row == 5:
                continue
            h = 1e-6 * max(abs(p[row, k]), 1e-2)
            pp, pm = p.copy(), p.copy()
            pp[row, k] += h
            pm[row, k] -= h
            fd[k, c] = (oracle.chi2_frozen(pp, grid, o, mt) - oracle.chi2_frozen(pm, grid, o, mt)) / (2 * h)
    ok, worst = grad_close(g, fd)
    print(f"adjoint vs central differences: worst relative error {worst:.3g}")
    assert ok, worst
