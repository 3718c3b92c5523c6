"""Parity at the workloads' full sizes, in the configuration the benchmark runs.

* c2 (100 PIEMD, 2000^2, 20 systems): the oracle's whole chi^2 evaluation
  (matches, positions, chi^2) against both precisions, and the complete image
  set of every system -- each (system, triangle) pair the oracle finds, and
  no other -- with every image position.
* c3 (1024 perturbed samples, grids 500^2..2000^2, one call): the full oracle
  evaluation and the complete image sets of eight samples drawn from the
  batch.
* c5 (1000 PIEMD, 4000^2, 100 systems): one sample against the oracle's full
  evaluation on all host cores (image sets, matches, chi^2; slow), and on two
  samples the outputs the oracle checks one by one -- barycentres, the FP64
  containment and barycentric position of every matched triangle, sampled
  node deflections within their bound -- and sampled gradient components
  against central differences of the oracle's frozen-assignment chi^2.
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
THREADS = os.cpu_count() or 4


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lt.load(build_if_missing=True)


def load_obs(cfg):
    with open(os.path.join(GOLDEN, f"obs_{cfg}.json")) as f:
        return json.load(f)


def chi2_tol(o, ref_xy, tol):
    res = np.hypot(np.asarray(o["x"]) - ref_xy[:, 0], np.asarray(o["y"]) - ref_xy[:, 1])
    return np.sum((2 * res * tol * 1.5 + 2 * tol * tol) / np.asarray(o["sigma"]) ** 2)


def run(w, o, grids, prec, grad=False, capacity=0):
    m = lt.Model(w.n_pot, w.batch, hit_capacity=capacity)
    m.set_params(w.params)
    obs = lt.Observations.from_dict(o)
    if grad:
        c2, g = m.chi2_grad(grids, obs, precision=prec)
    else:
        c2, g = m.chi2(grids, obs, precision=prec), None
    st, stats = m.sync()
    assert st == lt.LT_OK, st
    mt, mxy, bary = m.last_matches(len(o["x"]), len(o["dls_ds"]))
    out = dict(chi2=c2.cpu().numpy(), mt=mt.cpu().numpy(), mxy=mxy.cpu().numpy(),
               bary=bary.cpu().numpy(), stats=stats, grad=None if g is None else g.cpu().numpy())
    m.close()
    return out


def gpu_image_sets(w, grids, bary, r, prec, capacity):
    """Images of the given barycentres (the oracle's: the same source
    positions on both sides) found by lt_find_images on the whole batch, as one
    {(src, tri): (x, y)} dict per sample."""
    m = lt.Model(w.n_pot, w.batch, hit_capacity=capacity)
    m.set_params(w.params)
    sx = torch.as_tensor(np.ascontiguousarray(bary, dtype=np.float64), device="cuda")
    rr = torch.as_tensor(np.ascontiguousarray(r, dtype=np.float64), device="cuda")
    out, n = m.find_images(grids, sx, rr, precision=prec, capacity=capacity)
    st, stats = m.sync()
    assert st == lt.LT_OK, (st, stats)
    imgs = lt.images_to_numpy(out, n)
    m.close()
    return [{(int(h["src"]), int(h["tri"])): (float(h["x"]), float(h["y"])) for h in im}
            for im in imgs], stats


def assert_same_images(got, ref_hits, tol, what):
    """The GPU image set equals the oracle's exactly; positions within tol."""
    ref = {(h["src"], h["tri"]): (h["x"], h["y"]) for h in ref_hits}
    assert not any(h["undecidable"] for h in ref_hits), what
    missing, extra = set(ref) - set(got), set(got) - set(ref)
    assert not missing and not extra, (what, sorted(missing)[:5], sorted(extra)[:5])
    d = max((max(abs(got[k][0] - ref[k][0]), abs(got[k][1] - ref[k][1])) for k in ref),
            default=0.0)
    assert d <= tol, (what, d)
    return len(ref)


@pytest.mark.parametrize("prec,tol", [(lt.MIXED, 1e-4), (lt.FP64, 1e-9)])
def test_c2_full_chi2(oracle, prec, tol):
    w = W.c2()
    o = load_obs("c2")
    grid = w.grids[0].as_tuple()
    r = run(w, o, [grid], prec)
    ref = oracle.chi2(w.params[0], grid, o, n_threads=THREADS)
    assert ref["n_undecidable"] == 0
    assert np.array_equal(r["mt"][0], ref["match_tri"])
    ok = ref["match_tri"] >= 0
    assert np.abs(r["mxy"][0][ok] - ref["match_xy"][ok]).max() <= tol
    np.testing.assert_allclose(r["bary"][0], ref["bary"], rtol=0, atol=1e-10)
    assert abs(r["chi2"][0] - ref["chi2"]) <= chi2_tol(o, ref["match_xy"], tol) + 1e-12 * ref["chi2"]
    # the complete image set of every system, found from the oracle's barycentres
    sets, stats = gpu_image_sets(w, [grid], ref["bary"][None], np.asarray(o["dls_ds"])[None],
                                 prec, 4096)
    n = assert_same_images(sets[0], ref["hits"], tol, "c2")
    print(f"c2 precision {prec}: {n} images identical to the oracle's; stats {stats}")


def test_c3_full_batch_sampled(oracle):
    w = W.c3()
    o = load_obs("c3")
    grids = [g.as_tuple() for g in w.grids]
    r = run(w, o, grids, lt.MIXED)
    rng = np.random.default_rng(33)
    picks = rng.choice(w.batch, 8, replace=False)
    # barycentres of every sample (cheap), so that the image search runs on the
    # whole batch in its batched configuration
    bary = np.stack([oracle.barycentres(w.params[b], o)[0] for b in range(w.batch)])
    rr = np.broadcast_to(np.asarray(o["dls_ds"]), (w.batch, len(o["dls_ds"])))
    sets, stats = gpu_image_sets(w, grids, bary, rr, lt.MIXED, 4096)
    total = 0
    for b in picks:
        ref = oracle.chi2(w.params[b], grids[b], o, n_threads=THREADS)
        assert ref["n_undecidable"] == 0
        assert np.array_equal(r["mt"][b], ref["match_tri"]), b
        ok = ref["match_tri"] >= 0
        assert np.abs(r["mxy"][b][ok] - ref["match_xy"][ok]).max() <= 1e-4
        assert abs(r["chi2"][b] - ref["chi2"]) <= chi2_tol(o, ref["match_xy"], 1e-4) + \
            1e-12 * ref["chi2"]
        np.testing.assert_array_equal(bary[b], ref["bary"])
        total += assert_same_images(sets[b], ref["hits"], 1e-4, f"c3 sample {b}")
    print(f"c3: {total} images of 8 samples identical to the oracle's; batch stats {stats}")


@pytest.mark.slow
def test_c5_full_sample_against_full_oracle(oracle):
    """One c5 sample (1000 PIEMD, 4000^2 nodes, 100 systems) against the
    oracle's complete evaluation on all host cores: every image of every
    system, the matches, the positions and chi^2, in mixed precision."""
    w = W.c5(batch=1)
    o = load_obs("c5")
    grid = w.grids[0].as_tuple()
    cap = 1 << 17
    r = run(w, o, [grid], lt.MIXED, capacity=cap)
    ref = oracle.chi2(w.params[0], grid, o, n_threads=THREADS, capacity=1 << 18)
    assert ref["n_undecidable"] == 0
    assert np.array_equal(r["mt"][0], ref["match_tri"])
    ok = ref["match_tri"] >= 0
    assert np.abs(r["mxy"][0][ok] - ref["match_xy"][ok]).max() <= 1e-4
    np.testing.assert_allclose(r["bary"][0], ref["bary"], rtol=0, atol=1e-10)
    assert abs(r["chi2"][0] - ref["chi2"]) <= chi2_tol(o, ref["match_xy"], 1e-4) + \
        1e-12 * ref["chi2"]
    sets, stats = gpu_image_sets(w, [grid], ref["bary"][None], np.asarray(o["dls_ds"])[None],
                                 lt.MIXED, cap)
    n = assert_same_images(sets[0], ref["hits"], 1e-4, "c5")
    print(f"c5: {n} images identical to the oracle's; stats {stats}")


def tri_nodes(grid, tri):
    x0, y0, dx, dy, nx, ny = grid
    cell, t = divmod(int(tri), 2)
    i, j = cell % (nx - 1), cell // (nx - 1)
    v = [(i, j), (i + 1, j), (i + 1, j + 1)] if t == 0 else [(i, j), (i + 1, j + 1), (i, j + 1)]
    return [(x0 + a * dx, y0 + b * dy) for a, b in v]


def test_c5_full_size_local_checks(oracle):
    w = W.c5(batch=2)
    o = load_obs("c5")
    grid = w.grids[0].as_tuple()
    # 100 systems in a strongly folded lens: size the per-sample lists for it
    r = run(w, o, [grid] * w.batch, lt.MIXED, grad=True, capacity=1 << 17)
    print("c5 stats", r["stats"])
    ox, oy = np.asarray(o["x"]), np.asarray(o["y"])
    sys_, rr = np.asarray(o["sys"]), np.asarray(o["dls_ds"])
    for b in range(w.batch):
        p = w.params[b]
        bary, _ = oracle.barycentres(p, o)
        np.testing.assert_allclose(r["bary"][b], bary, rtol=0, atol=1e-10)
        for m in range(len(ox)):
            tri = r["mt"][b, m]
            if tri < 0:
                continue
            V = tri_nodes(grid, tri)
            i = sys_[m]
            # the oracle's own FP64 predicate on this triangle alone
            H, U = oracle.find_images(p, (V[0][0], V[0][1], grid[2], grid[3], 2, 2),
                                      [bary[i]], [rr[i]])
            t_local = 0 if tri % 2 == 0 else 1
            got = [h for h in H if h["tri"] == t_local]
            assert len(got) == 1 and not U, (b, m, tri)
            assert abs(got[0]["x"] - r["mxy"][b, m, 0]) <= 1e-4
            assert abs(got[0]["y"] - r["mxy"][b, m, 1]) <= 1e-4
    # sampled deflections of sample 0 within their bound
    m = lt.Model(w.n_pot, 1)
    m.set_params(w.params[:1])
    a, e = m.deflect_grid(grid, precision=lt.MIXED, with_error=True)
    rng = np.random.default_rng(55)
    idx = rng.integers(0, grid[4] * grid[5], 500)
    jj, ii = np.divmod(idx, grid[4])
    ax, ay, _ = oracle.alpha_points(w.params[0], grid[0] + ii * grid[2], grid[1] + jj * grid[3])
    A = a.reshape(-1, 2).cpu().numpy()[idx].astype(np.float64)
    E = e.reshape(-1).cpu().numpy()[idx].astype(np.float64)
    assert np.all(np.maximum(np.abs(A[:, 0] - ax), np.abs(A[:, 1] - ay)) <= E)
    m.close()
    # sampled gradient components of sample 0 against central differences
    g = r["grad"][0]
    mt = r["mt"][0]
    p = w.params[0]
    rows = [1, 2, 3, 4, 5, 7]
    big = np.argsort(-p[7])[:3]  # the most massive potentials
    for k in list(big) + [int(rng.integers(0, w.n_pot))]:
        for c in (0, 1, 5):
            row = rows[c]
            h = 1e-6 * max(abs(p[row, k]), 1e-2)
            pp, pm = p.copy(), p.copy()
            pp[row, k] += h
            pm[row, k] -= h
            fd = (oracle.chi2_frozen(pp, grid, o, mt) - oracle.chi2_frozen(pm, grid, o, mt)) / (2 * h)
            floor = 1e-6 * np.abs(g).max()
            assert abs(g[k, c] - fd) <= 1e-3 * abs(fd) + floor, (k, c, g[k, c], fd)


def test_c5_work_overflow_is_reported():
    """A c5 sample has a few thousand ambiguous (triangle, source) pairs: with
    a per-sample capacity of 256 the FP64 work list overflows, which sync
    reports as LT_ERR_OVERFLOW with the dropped count, never silently."""
    w = W.c5(batch=1)
    o = load_obs("c5")
    m = lt.Model(w.n_pot, 1, hit_capacity=256)
    m.set_params(w.params)
    m.chi2([w.grids[0].as_tuple()], lt.Observations.from_dict(o), precision=lt.MIXED)
    st, stats = m.sync()
    assert st == lt.LT_ERR_OVERFLOW
    assert stats["work_overflow"] > 0
    m.close()


def test_find_images_beyond_int32_nodes(oracle):
    """The largest case: a 46400^2 grid, 2.15e9 nodes (more than 2^31, a 34 GB
    node workspace), one SIS (c1), four sources in mixed precision -- the
    64-bit index paths of the deflection, the search and the image records.
    The grid's top rows hold cells beyond 2^31 and triangle ids beyond 2^32,
    where the outer image of the source (0, 1.9) falls.  The grid is dyadic
    (dx = 2^-9), so a patch of it starting at node (i0, j0) has bit-identical
    node coordinates: the oracle searches patches around the closed-form SIS
    image positions and the lens centre (a node, where the FP32 bound is
    1e30), and the union of its images, with ids mapped to the full grid,
    must equal the GPU's image set (exact ties included: the source (2, 1.5)
    has its images on nodes, and every operation of the lens is correctly
    rounded), with the positions."""
    w = W.c1()
    p = w.params[0]
    n = 46400
    dx = 2.0 ** -9
    x0 = -(n // 2) * dx
    y0 = 12.0 - (n - 1) * dx
    grid = (x0, y0, dx, dx, n, n)
    src = np.array([(0.0, 1.9), (2.0, 1.5), (-4.0, 6.0), (0.3, -0.2)])
    r = np.full(len(src), 0.7)
    m = lt.Model(1, 1, hit_capacity=4096)
    m.set_params(p[None])
    sx = torch.as_tensor(src[None], device="cuda")
    rr = torch.as_tensor(r[None], device="cuda")
    out, cnt = m.find_images([grid], sx, rr, precision=lt.MIXED, capacity=4096)
    st, stats = m.sync()
    assert st == lt.LT_OK, (st, stats)
    imgs = lt.images_to_numpy(out, cnt)[0]
    m.close()
    del out
    torch.cuda.empty_cache()
    got = {(int(h["src"]), int(h["tri"])): h for h in imgs}
    # closed form: the SIS maps theta to beta = theta - r b0 theta/|theta|, so
    # the images lie on the source's direction at |beta| + r b0 and r b0 - |beta|
    thE = 0.7 * (4.0 * math.pi * (p[7, 0] / 299792.458) ** 2 * 206264.80625)
    half = 16
    exp = {}
    for k, (bx, by) in enumerate(src):
        b = math.hypot(bx, by)
        spots = [(bx / b * (b + thE), by / b * (b + thE)),
                 (-bx / b * (thE - b), -by / b * (thE - b)), (0.0, 0.0)]
        for (tx, ty) in spots:
            i0 = max(0, int(round((tx - x0) / dx)) - half)
            j0 = max(0, int(round((ty - y0) / dx)) - half)
            i1 = min(n - 1, i0 + 2 * half)
            j1 = min(n - 1, j0 + 2 * half)
            if i1 - i0 < 2 or j1 - j0 < 2:  # the image is off the grid
                continue
            pw = i1 - i0 + 1
            patch = (x0 + i0 * dx, y0 + j0 * dx, dx, dx, pw, j1 - j0 + 1)
            H, _ = oracle.find_images(p, patch, [(bx, by)], [0.7], n_threads=4)
            for h in H:
                cell = h["tri"] // 2
                ci, cj = cell % (pw - 1), cell // (pw - 1)
                tri = 2 * ((j0 + cj) * (n - 1) + (i0 + ci)) + h["tri"] % 2
                exp[(k, tri)] = h
    assert max(t for _, t in exp) > 2 ** 32  # ids beyond 32 bits are exercised
    assert set(got) == set(exp), (sorted(set(got) ^ set(exp))[:10], len(got), len(exp))
    worst = max(max(abs(got[key]["x"] - h["x"]), abs(got[key]["y"] - h["y"]))
                for key, h in exp.items())
    assert worst <= 1e-4, worst
