"""D_ls/D_s from redshifts: the oracle's adaptive quadrature pinned to the
closed forms of three Friedmann models, and the library's host code
(lt_dls_ds) against both."""
import math

import pytest

from paper_1902_03252_gb300 import lt


@pytest.fixture(scope="module")
def lib():
    from paper_1902_03252_gb300 import _build
    try:
        _build.build()
    except RuntimeError as e:
        pytest.skip(f"cannot build the library here: {e}")
    return lt


def closed_forms(zl, zs):
    """(omega_m, omega_lambda, D_ls/D_s) of the Einstein-de Sitter, de Sitter
    and Milne models, whose comoving distances have closed forms."""
    dc = lambda z: 2 * (1 - 1 / math.sqrt(1 + z))       # EdS: D_C = 2 (1 - 1/sqrt(1+z))
    eds = (dc(zs) - dc(zl)) / dc(zs)
    ds = (zs - zl) / zs                                  # de Sitter: D_C = z
    dm = lambda z: ((1 + z) - 1 / (1 + z)) / 2           # Milne: D_M = sinh(ln(1+z))
    m1, m2 = dm(zl), dm(zs)
    milne = (m2 * math.sqrt(1 + m1 * m1) - m1 * math.sqrt(1 + m2 * m2)) / m2
    return [(1.0, 0.0, eds), (0.0, 1.0, ds), (0.0, 0.0, milne)]


@pytest.mark.parametrize("zl,zs", [(0.3, 2.0), (0.05, 0.5), (1.0, 6.0)])
def test_oracle_closed_forms(oracle, zl, zs):
    for om, ol, exp in closed_forms(zl, zs):
        assert oracle.dls_ds(zl, zs, om, ol) == pytest.approx(exp, rel=1e-12), (om, ol)


def test_oracle_limits(oracle):
    # a source just behind the lens sees no lensing; a lens at z = 0 gives 1
    assert oracle.dls_ds(0.5, 0.5 + 1e-9) == pytest.approx(0.0, abs=1e-8)
    assert oracle.dls_ds(1e-12, 2.0) == pytest.approx(1.0, rel=1e-9)


def test_closed_forms(lib):
    zl, zs = 0.3, 2.0
    # Einstein-de Sitter: D_C = 2 (1 - 1/sqrt(1+z))
    dc = lambda z: 2 * (1 - 1 / math.sqrt(1 + z))
    assert lib.dls_ds(zl, zs, 1.0, 0.0) == pytest.approx((dc(zs) - dc(zl)) / dc(zs), rel=1e-13)
    # de Sitter: D_C = z
    assert lib.dls_ds(zl, zs, 0.0, 1.0) == pytest.approx((zs - zl) / zs, rel=1e-13)
    # Milne (empty, open): D_M = ((1+z) - 1/(1+z)) / 2
    dm = lambda z: ((1 + z) - 1 / (1 + z)) / 2
    m1, m2 = dm(zl), dm(zs)
    exp = (m2 * math.sqrt(1 + m1 * m1) - m1 * math.sqrt(1 + m2 * m2)) / m2
    assert lib.dls_ds(zl, zs, 0.0, 0.0) == pytest.approx(exp, rel=1e-12)


@pytest.mark.parametrize("zl,zs,om,ol", [(0.3, 2.0, 0.3, 0.7), (0.05, 0.5, 0.27, 0.73),
                                          (0.5, 6.0, 0.3, 0.7), (0.2, 1.0, 0.2, 0.5)])
def test_matches_oracle(lib, oracle, zl, zs, om, ol):
    assert lib.dls_ds(zl, zs, om, ol) == pytest.approx(oracle.dls_ds(zl, zs, om, ol), rel=1e-12)


def test_rejects_bad_input(lib):
    for args in [(2.0, 1.0, 0.3, 0.7), (-0.1, 1.0, 0.3, 0.7), (0.3, 2.0, 0.5, 0.7)]:
        with pytest.raises(lt.LTError):
            lib.dls_ds(*args)
