"""Pins of the oracle's statement of the paper's mixed rule (Sect. 3.3 and
App. A.3): deflection fields whose distortion criteria have closed forms.

* A uniform mass sheet, alpha = kappa theta, maps a pixel of side h onto one
  of side |1 - kappa| h along both axes: delta_1 = delta_2 = kappa h and
  delta_3 = delta_4 = 0.  The criteria of the first kind fire exactly when the
  axis magnification 1/|1 - kappa| exceeds 3.26 (|1 - kappa| h < 0.0092" at
  h = 0.03"), those of the second kind never.
* A pure cross term, alpha = (g theta_2, g theta_1), has delta_1 = delta_2 = 0
  and delta_3 = delta_4 = g h: only the second kind fires, for g h > 0.0104".
* Halo patches: 400 x 400 pixels around a cluster-scale halo, 20 x 20 around
  a galaxy-scale one, none around a massless potential.
"""
import math

import numpy as np
import pytest

SIS, PIEMD, SIE = 0, 1, 2


def grid_of(n, h=0.03, x0=-3.0, y0=-2.0):
    return (x0, y0, h, h, n, n)


def nodes(grid):
    x0, y0, dx, dy, nx, ny = grid
    jj, ii = np.mgrid[0:ny, 0:nx]
    return x0 + ii * dx, y0 + jj * dy


def massless(n_pot=1):
    p = np.zeros((8, n_pot))
    p[0] = SIE
    return p


def sigma_for_b0(b0):
    return 299792.458 * math.sqrt(b0 / (4 * math.pi * 206264.80625))


def test_thresholds_are_the_paper_magnification(oracle):
    # 0.0092" on a 0.03" pixel is the axis magnification 3.26
    assert 0.03 / oracle.PAPER_T12 == pytest.approx(3.26, abs=0.005)


@pytest.mark.parametrize("kappa,fires", [(0.0, False), (0.5, False), (0.68, False),
                                         (0.72, True), (0.9, True), (1.1, True),
                                         (1.25, True), (1.32, False), (2.0, False)])
def test_mass_sheet_first_criteria(oracle, kappa, fires):
    g = grid_of(40)
    X, Y = nodes(g)
    alpha = np.stack([kappa * X, kappa * Y], axis=-1)
    f = oracle.paper_flags(alpha, g, massless())
    assert not f[0].any() and not f[:, 0].any()  # no neighbour, no criterion
    assert f[1:, 1:].all() == fires and f[1:, 1:].any() == fires


@pytest.mark.parametrize("gam,fires", [(0.0, False), (0.3, False), (0.34, False),
                                       (0.35, True), (-0.5, True), (1.0, True)])
def test_cross_term_second_criteria(oracle, gam, fires):
    g = grid_of(30)
    X, Y = nodes(g)
    alpha = np.stack([gam * Y, gam * X], axis=-1)
    f = oracle.paper_flags(alpha, g, massless())
    assert f[1:, 1:].all() == fires and f[1:, 1:].any() == fires
    # only one component moves per difference: fields with just one of the
    # two cross terms fire too (delta_3 alone, delta_4 alone)
    if fires:
        only3 = oracle.paper_flags(np.stack([gam * Y, 0 * X], -1), g, massless())
        only4 = oracle.paper_flags(np.stack([0 * Y, gam * X], -1), g, massless())
        assert only3[1:, 1:].all() and only4[1:, 1:].all()


def test_thresholds_scale_with_the_spacing(oracle):
    # the same sheet on a grid twice as fine fires at the same kappa
    for h in (0.015, 0.06):
        g = grid_of(20, h=h)
        X, Y = nodes(g)
        assert oracle.paper_flags(np.stack([0.9 * X, 0.9 * Y], -1), g, massless())[1:, 1:].all()
        assert not oracle.paper_flags(np.stack([0.5 * X, 0.5 * Y], -1), g, massless()).any()


@pytest.mark.parametrize("b0,half", [(20.0, 200), (0.01, 10), (0.0, 0)])
def test_halo_patches(oracle, b0, half):
    n = 900
    g = grid_of(n, x0=0.0, y0=0.0)
    p = massless()
    ic, jc = 450, 430
    p[1, 0], p[2, 0] = ic * 0.03 + 0.004, jc * 0.03 - 0.011  # nearest node (ic, jc)
    p[7, 0] = sigma_for_b0(b0) if b0 > 0 else 0.0
    f = oracle.paper_flags(np.zeros((n, n, 2)), g, p)
    exp = np.zeros((n, n), bool)
    if half:
        exp[jc - half:jc + half, ic - half:ic + half] = True
    assert np.array_equal(f, exp)


def test_patch_clipped_at_the_grid_edge(oracle):
    n = 100
    g = grid_of(n, x0=0.0, y0=0.0)
    p = massless()
    p[1, 0], p[2, 0] = 3 * 0.03, 97 * 0.03
    p[7, 0] = sigma_for_b0(0.5)
    f = oracle.paper_flags(np.zeros((n, n, 2)), g, p)
    exp = np.zeros((n, n), bool)
    exp[87:100, 0:13] = True
    assert np.array_equal(f, exp)
