"""Write the stored inputs and expected values under tests/golden/.

Calls only the FP64 oracle (``oracle/``) and the seeded generators
(``paper_1902_03252_gb300.workloads``); nothing here touches the CUDA path.

Outputs
  c1_sis.json   the SIS worked case: closed-form images of the source
                (2.0", 1.5") behind an SIS with effective Einstein radius 10"
                (lens equation Eq. 1 with |alpha| = theta_E, Sect. 2.1) and the
                oracle's hits on the 256^2 grid.
  obs_<cfg>.json  observed multiple images of each workload: the oracle's
                images of sources drawn uniformly in the central half of the
                field, kept when multiply imaged, plus N(0, 0.01") noise per
                coordinate (the relensing data of Sect. 2.2.1).  For c1 the
                images are the closed form plus noise.

Usage: python tests/golden/make_golden.py [c1 c2 c3 c4 c5]
"""
from __future__ import annotations

import json
import math
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1902_03252_gb300 import workloads as W  # noqa: E402

SIGMA_OBS = 0.01
THREADS = os.cpu_count() or 1


def _dump(name, obj):
    path = os.path.join(HERE, name)
    with open(path, "w") as f:
        json.dump(obj, f, indent=1)
    print("wrote", path)


def sis_closed_form(beta, theta_e):
    b = math.hypot(*beta)
    u = (beta[0] / b, beta[1] / b)
    ims = [(u[0] * (b + theta_e), u[1] * (b + theta_e))]
    if b < theta_e:
        ims.append((u[0] * (b - theta_e), u[1] * (b - theta_e)))
    return ims


def make_c1():
    w = W.c1()
    beta, r, te = w.notes["source"], w.notes["dls_ds"], w.notes["theta_e"]
    ims = sis_closed_form(beta, te)
    g = w.grids[0].as_tuple()
    H, U = oracle.find_images(w.params[0], g, [beta], [r])
    _dump("c1_sis.json", {
        "citation": "Eq. 1 (lens equation) with |alpha| = theta_E for the SIS (Sect. 2.1, Eq. 10): "
                    "images at beta_hat (|beta| +/- theta_E), the minus image only for |beta| < theta_E",
        "beta": list(beta), "theta_e": te, "dls_ds": r, "grid": list(g),
        "closed_form_images": [list(i) for i in ims],
        "oracle_hits": [{"tri": h["tri"], "x": h["x"], "y": h["y"]} for h in H],
        "oracle_undecidable": len(U),
    })
    noise = W.position_noise(1, len(ims), SIGMA_OBS)
    xy = np.array(ims) + noise
    _dump("obs_c1.json", {
        "config": "c1", "grid": list(g), "x": xy[:, 0].tolist(), "y": xy[:, 1].tolist(),
        "sigma": [SIGMA_OBS] * len(ims), "sys": [0] * len(ims), "dls_ds": [r],
        "src_true": [list(beta)],
        "how": "SIS closed-form images plus N(0, 0.01\") noise (seeded)",
    })


def mapped_candidates(cfg_index: int, base_params, n: int, half_field: float):
    """Candidate sources for a super-critical cluster: the source-plane
    positions beta = theta - r alpha(theta) (oracle) of image-plane points
    drawn uniformly over the field (half-width half_field / 2), so that every
    candidate has at least one image.  Used where the summed convergence is
    so high that the map is one-to-one except near the field edge, where the
    critical curves lie."""
    cand = W.source_candidates(cfg_index, n, half_field)
    ax, ay, _ = oracle.alpha_points(base_params, cand[:, 0], cand[:, 1])
    out = cand.copy()
    out[:, 0] = cand[:, 0] - cand[:, 2] * ax
    out[:, 1] = cand[:, 1] - cand[:, 2] * ay
    return out


def make_obs(cfg_name: str, cfg_index: int, base_params, grid: W.Grid, n_src: int,
             half_field: float, n_candidates: int, mapped: bool = False):
    t0 = time.time()
    cand = (mapped_candidates(cfg_index, base_params, n_candidates, half_field) if mapped
            else W.source_candidates(cfg_index, n_candidates, half_field))
    H, U = oracle.find_images(base_params, grid.as_tuple(), cand[:, :2], cand[:, 2],
                              n_threads=THREADS, capacity=1 << 20)
    by_src = {}
    for h in H:
        by_src.setdefault(h["src"], []).append(h)
    keep = [s for s in range(n_candidates) if len(by_src.get(s, [])) >= 2][:n_src]
    if len(keep) < n_src:
        raise RuntimeError(f"{cfg_name}: only {len(keep)} multiply imaged sources")
    xs, ys, sys_, r = [], [], [], []
    for i, s in enumerate(keep):
        for h in by_src[s]:
            xs.append(h["x"])
            ys.append(h["y"])
            sys_.append(i)
        r.append(float(cand[s, 2]))
    noise = W.position_noise(cfg_index, len(xs), SIGMA_OBS)
    xy = np.column_stack([xs, ys]) + noise
    _dump(f"obs_{cfg_name}.json", {
        "config": cfg_name, "grid": list(grid.as_tuple()),
        "x": xy[:, 0].tolist(), "y": xy[:, 1].tolist(), "sigma": [SIGMA_OBS] * len(xs),
        "sys": sys_, "dls_ds": r, "src_true": cand[keep, :2].tolist(),
        "how": ("oracle images of multiply imaged candidate sources (" +
                ("lens-mapped image-plane points of the whole field"
                 if mapped else "uniform in the central half of the field") +
                ") on the stated grid, plus N(0, 0.01\") noise per coordinate"),
        "n_undecidable": len(U),
    })
    print(f"{cfg_name}: {len(keep)} systems, {len(xs)} images, {time.time() - t0:.1f}s")


def main(which):
    if "c1" in which:
        make_c1()
    if "c2" in which:
        w = W.c2()
        make_obs("c2", 2, w.params[0], w.obs_grid, w.n_src, 100.0, 300)
    if "c3" in which:
        w = W.c3(batch=1)
        make_obs("c3", 3, w.notes["base"], w.obs_grid, w.n_src, 100.0, 200)
    if "c4" in which:
        w = W.c4()
        make_obs("c4", 4, w.params[0], w.obs_grid, w.n_src, 100.0, 300)
    if "c5" in which:
        w = W.c5(batch=1)
        make_obs("c5", 5, w.notes["base"], w.obs_grid, w.n_src, 400.0, 1000, mapped=True)


if __name__ == "__main__":
    main(sys.argv[1:] or ["c1", "c2", "c3", "c4", "c5"])
