"""FP64 CPU oracle for the image-plane chi^2 path (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product (the CUDA library and its
binding) never does: it shares no code with this oracle.

The C++ source ``lt_oracle.cpp`` is compiled with ``-ffp-contract=off`` so
every floating-point operation is a separately rounded IEEE double, on x86
and Arm alike.  See that file for the step-by-step statement of the method.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lt_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "liblt_oracle.so")

PARAM_ROWS = ("kind", "x", "y", "e", "phi", "r_core", "r_cut", "sigma_v")
GRAD_ROWS = ("x", "y", "e", "phi", "r_core", "sigma_v")


class Hit(C.Structure):
    _fields_ = [("src", C.c_int32), ("undecidable", C.c_int32), ("tri", C.c_int64),
                ("x", C.c_double), ("y", C.c_double), ("w", C.c_double * 3)]


class Pair(C.Structure):
    _fields_ = [("src", C.c_int32), ("inside", C.c_int32), ("tri", C.c_int64)]


def build(force: bool = False) -> str:
    """Compile the oracle library (g++, OpenMP, no FP contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-fopenmp", _SRC, "-o", tmp]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int32)
        lp = C.POINTER(C.c_int64)
        L.lto_alpha_points.argtypes = [dp, C.c_int, C.c_int, dp, dp, dp, dp, dp]
        L.lto_deflect_grid.argtypes = [dp, C.c_int, C.c_double, C.c_double, C.c_double,
                                       C.c_double, C.c_int, C.c_int, C.c_int, dp, dp]
        L.lto_find_images.argtypes = [dp, C.c_int, C.c_double, C.c_double, C.c_double,
                                      C.c_double, C.c_int, C.c_int, C.c_int, dp, dp, dp,
                                      C.c_int, C.c_int64, C.POINTER(Hit), C.c_int64,
                                      C.POINTER(Pair), lp]
        L.lto_find_images.restype = C.c_int64
        L.lto_barycentres.argtypes = [dp, C.c_int, C.c_int, dp, dp, ip, C.c_int, dp, dp, dp]
        L.lto_chi2.argtypes = [dp, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double,
                               C.c_int, C.c_int, C.c_int, dp, dp, dp, ip, C.c_int, dp,
                               C.c_int, C.c_int64, C.POINTER(Hit), dp, lp, dp, dp, lp, lp]
        L.lto_chi2_frozen.argtypes = [dp, C.c_int, C.c_double, C.c_double, C.c_double,
                                      C.c_double, C.c_int, C.c_int, C.c_int, dp, dp, dp, ip,
                                      C.c_int, dp, lp, dp]
        L.lto_chi2_grad.argtypes = [dp, C.c_int, C.c_double, C.c_double, C.c_double,
                                    C.c_double, C.c_int, C.c_int, C.c_int, dp, dp, dp, ip,
                                    C.c_int, dp, lp, dp, dp]
        L.lto_jacobian_points.argtypes = [dp, C.c_int, C.c_int, dp, dp, dp]
        L.lto_chi2_source.argtypes = [dp, C.c_int, C.c_int, dp, dp, dp, ip, C.c_int, dp, dp, dp]
        L.lto_tri_magnification.argtypes = [dp, C.c_int, C.c_double, C.c_double, C.c_double,
                                            C.c_double, C.c_int, C.c_int, C.c_int, lp, dp, dp]
        _lib = L
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(C.POINTER(C.c_int32))


def _l(a):
    a = np.ascontiguousarray(a, dtype=np.int64)
    return a, a.ctypes.data_as(C.POINTER(C.c_int64))


def _params(params):
    p = np.ascontiguousarray(params, dtype=np.float64)
    assert p.ndim == 2 and p.shape[0] == 8, "params must be [8][n_pot] for one sample"
    return p


def alpha_points(params, x, y):
    """Deflection (ax, ay) and sum_k |alpha_k| at points x, y (one sample)."""
    p, pp = _d(_params(params))
    x, xp = _d(np.atleast_1d(x))
    y, yp = _d(np.atleast_1d(y))
    n = x.size
    ax, axp = _d(np.zeros(n))
    ay, ayp = _d(np.zeros(n))
    s, sp = _d(np.zeros(n))
    lib().lto_alpha_points(pp, p.shape[1], n, xp, yp, axp, ayp, sp)
    return ax, ay, s


def deflect_grid(params, grid, n_threads: int = 1):
    """alpha over a grid (x0, y0, dx, dy, nx, ny): [ny][nx][2] and sum|alpha_k|."""
    x0, y0, dx, dy, nx, ny = grid
    p, pp = _d(_params(params))
    out, op = _d(np.zeros((ny, nx, 2)))
    s, sp = _d(np.zeros((ny, nx)))
    lib().lto_deflect_grid(pp, p.shape[1], x0, y0, dx, dy, nx, ny, n_threads, op, sp)
    return out, s


def find_images(params, grid, src_xy, dls_ds, d_src=None, n_threads: int = 1,
                capacity: int = 1 << 16, und_capacity: int = 1 << 12):
    """Hits (list of dict) and undecidable pairs for explicit source positions."""
    x0, y0, dx, dy, nx, ny = grid
    p, pp = _d(_params(params))
    src, sp = _d(np.asarray(src_xy, dtype=np.float64).reshape(-1, 2))
    r, rp = _d(np.atleast_1d(dls_ds))
    n_src = src.shape[0]
    if d_src is None:
        d_src = np.zeros(n_src)
    ds, dsp = _d(d_src)
    hits = (Hit * capacity)()
    und = (Pair * und_capacity)()
    n_und = C.c_int64(0)
    n = lib().lto_find_images(pp, p.shape[1], x0, y0, dx, dy, nx, ny, n_src, sp, rp, dsp,
                              n_threads, capacity, hits, und_capacity, und, C.byref(n_und))
    if n > capacity:
        raise RuntimeError(f"oracle hit capacity {capacity} < {n}")
    H = [dict(src=h.src, tri=h.tri, x=h.x, y=h.y, w=tuple(h.w), undecidable=h.undecidable)
         for h in hits[:n]]
    U = [dict(src=u.src, tri=u.tri, inside=u.inside) for u in und[:min(n_und.value, und_capacity)]]
    return H, U


def barycentres(params, obs):
    """Per-system barycentres [n_sys][2] and their FP64 uncertainty [n_sys]."""
    p, pp = _d(_params(params))
    ox, oxp = _d(obs["x"])
    oy, oyp = _d(obs["y"])
    osys, osp = _i(obs["sys"])
    r, rp = _d(obs["dls_ds"])
    n_sys = r.size
    b, bp = _d(np.zeros((n_sys, 2)))
    d, dpp = _d(np.zeros(n_sys))
    lib().lto_barycentres(pp, p.shape[1], ox.size, oxp, oyp, osp, n_sys, rp, bp, dpp)
    return b, d


def chi2(params, grid, obs, n_threads: int = 1, capacity: int = 1 << 16):
    """Full chi^2 of Eq. 11 for one sample; returns a dict of all intermediates."""
    x0, y0, dx, dy, nx, ny = grid
    p, pp = _d(_params(params))
    ox, oxp = _d(obs["x"])
    oy, oyp = _d(obs["y"])
    sg, sgp = _d(obs["sigma"])
    osys, osp = _i(obs["sys"])
    r, rp = _d(obs["dls_ds"])
    n_obs, n_sys = ox.size, r.size
    hits = (Hit * capacity)()
    c2 = C.c_double(0.0)
    mt, mtp = _l(np.zeros(n_obs))
    mxy, mxyp = _d(np.zeros((n_obs, 2)))
    b, bp = _d(np.zeros((n_sys, 2)))
    nh = C.c_int64(0)
    nu = C.c_int64(0)
    rc = lib().lto_chi2(pp, p.shape[1], x0, y0, dx, dy, nx, ny, n_obs, oxp, oyp, sgp, osp,
                        n_sys, rp, n_threads, capacity, hits, C.byref(c2), mtp, mxyp, bp,
                        C.byref(nh), C.byref(nu))
    if rc != 0:
        raise RuntimeError(f"oracle hit capacity {capacity} < {nh.value}")
    H = [dict(src=h.src, tri=h.tri, x=h.x, y=h.y, w=tuple(h.w), undecidable=h.undecidable)
         for h in hits[:nh.value]]
    return dict(chi2=c2.value, match_tri=mt.copy(), match_xy=mxy.copy(), bary=b.copy(),
                hits=H, n_undecidable=nu.value)


def chi2_frozen(params, grid, obs, match_tri):
    """chi^2 with the triangle assignment held fixed (value only)."""
    x0, y0, dx, dy, nx, ny = grid
    p, pp = _d(_params(params))
    ox, oxp = _d(obs["x"])
    oy, oyp = _d(obs["y"])
    sg, sgp = _d(obs["sigma"])
    osys, osp = _i(obs["sys"])
    r, rp = _d(obs["dls_ds"])
    mt, mtp = _l(match_tri)
    c2 = C.c_double(0.0)
    lib().lto_chi2_frozen(pp, p.shape[1], x0, y0, dx, dy, nx, ny, ox.size, oxp, oyp, sgp,
                          osp, r.size, rp, mtp, C.byref(c2))
    return c2.value


def chi2_grad(params, grid, obs, match_tri):
    """(chi^2, d chi^2/d params [n_pot][6]) with the assignment held fixed."""
    x0, y0, dx, dy, nx, ny = grid
    p, pp = _d(_params(params))
    ox, oxp = _d(obs["x"])
    oy, oyp = _d(obs["y"])
    sg, sgp = _d(obs["sigma"])
    osys, osp = _i(obs["sys"])
    r, rp = _d(obs["dls_ds"])
    mt, mtp = _l(match_tri)
    c2 = C.c_double(0.0)
    g, gp = _d(np.zeros((p.shape[1], 6)))
    lib().lto_chi2_grad(pp, p.shape[1], x0, y0, dx, dy, nx, ny, ox.size, oxp, oyp, sgp, osp,
                        r.size, rp, mtp, C.byref(c2), gp)
    return c2.value, g


def jacobian_points(params, x, y):
    """d alpha / d theta at points: [n][2][2] (rows alpha_x, alpha_y)."""
    p, pp = _d(_params(params))
    x, xp = _d(np.atleast_1d(x))
    y, yp = _d(np.atleast_1d(y))
    j, jp = _d(np.zeros((x.size, 2, 2)))
    lib().lto_jacobian_points(pp, p.shape[1], x.size, xp, yp, jp)
    return j


def chi2_source(params, obs):
    """Source-plane chi^2 of one sample and the point magnification mu at
    every observed image."""
    p, pp = _d(_params(params))
    ox, oxp = _d(obs["x"])
    oy, oyp = _d(obs["y"])
    sg, sgp = _d(obs["sigma"])
    osys, osp = _i(obs["sys"])
    r, rp = _d(obs["dls_ds"])
    mu, mup = _d(np.zeros(ox.size))
    c2 = C.c_double(0.0)
    lib().lto_chi2_source(pp, p.shape[1], ox.size, oxp, oyp, sgp, osp, r.size, rp,
                          C.byref(c2), mup)
    return c2.value, mu


def tri_magnification(params, grid, tri, r):
    """Signed triangle magnification (image area / lensed area) of grid triangles."""
    x0, y0, dx, dy, nx, ny = grid
    p, pp = _d(_params(params))
    t, tp = _l(np.atleast_1d(tri))
    rr, rp = _d(np.broadcast_to(np.asarray(r, dtype=np.float64), t.shape))
    mu, mup = _d(np.zeros(t.size))
    lib().lto_tri_magnification(pp, p.shape[1], x0, y0, dx, dy, nx, ny, t.size, tp, rp, mup)
    return mu


def dls_ds(z_l, z_s, omega_m=0.3, omega_lambda=0.7):
    """D_ls/D_s by adaptive quadrature of the comoving distance (scipy), for
    flat or open cosmologies: D_M12 / D_M2 with D_M the transverse comoving
    distance and D_M12 = D_M2 sqrt(1 + Ok D_M1^2) - D_M1 sqrt(1 + Ok D_M2^2)."""
    from scipy import integrate
    ok = 1.0 - omega_m - omega_lambda

    def dc(z):
        f = lambda x: 1.0 / np.sqrt(omega_m * (1 + x) ** 3 + ok * (1 + x) ** 2 + omega_lambda)
        return integrate.quad(f, 0.0, z, epsabs=0, epsrel=1e-13, limit=200)[0]

    def dm(z):
        d = dc(z)
        return np.sinh(np.sqrt(ok) * d) / np.sqrt(ok) if ok > 1e-12 else d
    m1, m2 = dm(z_l), dm(z_s)
    okc = max(ok, 0.0)
    return (m2 * np.sqrt(1 + okc * m1 * m1) - m1 * np.sqrt(1 + okc * m2 * m2)) / m2


# ------------------------------------------------- the paper's mixed rule
PAPER_PIXEL = 0.03          # arcsec: the pixel size the criteria are stated for
PAPER_T12 = 0.0092          # arcsec: |dx - delta_1,2| below this => DP (magnification > 3.26)
PAPER_T34 = 0.0104          # arcsec: |delta_3,4| above this => DP
PAPER_CLUSTER_B0 = 1.0      # arcsec: b0 at or above this is a cluster-scale halo
PAPER_HALF_CLUSTER = 200    # 400 x 400 pixel DP patch around cluster-scale halos
PAPER_HALF_GALAXY = 10      # 20 x 20 pixel DP patch around galaxy-scale halos


def paper_flags(alpha, grid, params, dtype=np.float32):
    """Nodes the paper's mixed rule recomputes in double precision (Sect. 3.3
    and App. A.3): [ny][nx] bool.

    alpha: [ny][nx][2] single-precision gradient grid (the rule is evaluated on
    the SP values, as in the paper); grid: (x0, y0, dx, dy, nx, ny); params:
    [8][n_pot] of one sample.

    1. Distortion criteria.  With the left neighbour (theta_1 - dx) and the
       lower neighbour (theta_2 - dy) of a node,
         delta_1 = a_1(node) - a_1(left),  delta_2 = a_2(node) - a_2(lower),
         delta_3 = a_1(node) - a_1(lower), delta_4 = a_2(node) - a_2(left);
       the node is flagged if |dx - delta_1| or |dy - delta_2| is below the
       0.0092" threshold (axis magnification above 3.26, with D_ls/D_s = 1,
       the paper's worst case), or |delta_3| or |delta_4| exceeds 0.0104".
       Both thresholds are stated for 0.03" pixels; a grid uses them scaled
       by its spacing along the difference (dx for delta_1 and delta_4, dy
       for delta_2 and delta_3) over 0.03", and the pixel length of the
       delta_1,2 criterion is that spacing.  Nodes of the first row and column
       have no neighbour and no criterion.  The differences and comparisons
       are taken in `dtype` (single precision: the grid's own).
    2. Halo patches: 400 x 400 pixels around every cluster-scale halo
       (b0 >= 1") and 20 x 20 around every galaxy-scale one, centred on the
       node nearest the halo centre (ties away from zero; rows and columns
       [c - half, c + half)).  A potential of zero mass is no halo and has
       no patch.
    """
    x0, y0, dx, dy, nx, ny = grid
    a = np.asarray(alpha).astype(dtype)
    assert a.shape == (ny, nx, 2), a.shape
    hx, hy = dtype(dx), dtype(dy)
    t12x = dtype(PAPER_T12) * hx / dtype(PAPER_PIXEL)
    t12y = dtype(PAPER_T12) * hy / dtype(PAPER_PIXEL)
    t34x = dtype(PAPER_T34) * hx / dtype(PAPER_PIXEL)
    t34y = dtype(PAPER_T34) * hy / dtype(PAPER_PIXEL)
    a1, a2 = a[..., 0], a[..., 1]
    d1 = a1[1:, 1:] - a1[1:, :-1]
    d2 = a2[1:, 1:] - a2[:-1, 1:]
    d3 = a1[1:, 1:] - a1[:-1, 1:]
    d4 = a2[1:, 1:] - a2[1:, :-1]
    flags = np.zeros((ny, nx), bool)
    flags[1:, 1:] = ((np.abs(hx - d1) < t12x) | (np.abs(hy - d2) < t12y) |
                     (np.abs(d3) > t34y) | (np.abs(d4) > t34x))
    p = _params(params)
    b0 = 4.0 * np.pi * (p[7] / 299792.458) ** 2 * 206264.80625
    for k in range(p.shape[1]):
        if not b0[k] > 0.0:
            continue
        half = PAPER_HALF_CLUSTER if b0[k] >= PAPER_CLUSTER_B0 else PAPER_HALF_GALAXY
        fi, fj = (p[1, k] - x0) / dx, (p[2, k] - y0) / dy
        ic = int(np.copysign(np.floor(abs(fi) + 0.5), fi))
        jc = int(np.copysign(np.floor(abs(fj) + 0.5), fj))
        r0, r1 = max(jc - half, 0), max(min(jc + half, ny), 0)
        c0, c1 = max(ic - half, 0), max(min(ic + half, nx), 0)
        flags[r0:r1, c0:c1] = True
    return flags
