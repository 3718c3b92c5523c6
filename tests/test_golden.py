"""Stored fixtures under tests/golden/ (written by tests/golden/make_golden.py,
which calls only the oracle and the seeded generators)."""
import json
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def test_c1_closed_form(oracle):
    """The SIS worked case: the two closed-form images (Eq. 1 with
    |alpha| = theta_E) are (10.0, 7.5) and (-6.0, -4.5); the oracle's hits
    away from the singular centre lie within the O(dx^2) interpolation error
    of them, and re-running the oracle reproduces the stored hits exactly."""
    g = load("c1_sis.json")
    exp = g["closed_form_images"]
    assert exp[0] == pytest.approx([10.0, 7.5], abs=1e-12)
    assert exp[1] == pytest.approx([-6.0, -4.5], abs=1e-12)
    dx = g["grid"][2]
    far = [h for h in g["oracle_hits"] if math.hypot(h["x"], h["y"]) > 2 * dx]
    assert len(far) == 2
    for im in exp:
        assert min(math.hypot(h["x"] - im[0], h["y"] - im[1]) for h in far) < 0.01
    from paper_1902_03252_gb300 import workloads as W
    w = W.c1()
    H, _ = oracle.find_images(w.params[0], tuple(g["grid"]), [g["beta"]], [g["dls_ds"]])
    assert [(h["tri"], h["x"], h["y"]) for h in H] == \
        [(h["tri"], h["x"], h["y"]) for h in g["oracle_hits"]]


@pytest.mark.parametrize("cfg", ["c1", "c2", "c3", "c4", "c5"])
def test_observation_files(cfg):
    """Every stored observation file is well formed: each system has at least
    two images, sigma = 0.01", D_ls/D_s within the drawn range."""
    path = os.path.join(GOLDEN, f"obs_{cfg}.json")
    if not os.path.exists(path):
        pytest.skip(f"{path} not generated")
    o = load(f"obs_{cfg}.json")
    n = len(o["x"])
    assert len(o["y"]) == n == len(o["sigma"]) == len(o["sys"])
    counts = np.bincount(o["sys"], minlength=len(o["dls_ds"]))
    assert np.all(counts >= 2 if cfg != "c1" else counts == 2)
    assert np.all(np.asarray(o["sigma"]) == 0.01)
    assert all(0.3 <= r <= 0.9 for r in o["dls_ds"])
