"""One small invocation of every kernel of the library, for profiling: the
mixed and FP64 chi^2 with gradient on the 1000^2 workload (100 PIEMD, 20
systems), the deflection grid in all three precisions, the source-plane chi^2
and the magnifications.  Run it under a profiler, e.g.

    ncu --clock-control none --metrics <list> python -m paper_1902_03252_gb300.profile_all
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1902_03252_gb300 import lt, workloads as W  # noqa: E402


def main():
    import torch
    w = W.c4()
    with open(os.path.join(ROOT, "tests", "golden", "obs_c4.json")) as f:
        o = json.load(f)
    grid = [w.grids[0].as_tuple()]
    m = lt.Model(w.n_pot, 1)
    m.set_params(w.params)
    obs = lt.Observations.from_dict(o)
    for prec in (lt.MIXED, lt.FP64):
        m.chi2_grad(grid, obs, precision=prec)
    m.last_magnifications(obs)
    m.chi2_source(obs)
    small = (-50.0, -50.0, 0.25, 0.25, 401, 401)
    for prec in (lt.MIXED, lt.FP64, lt.PAPER):
        m.deflect_grid(small, precision=prec)
    st, stats = m.sync()
    torch.cuda.synchronize()
    print("status", st, stats)
    m.close()
    return 0 if st == lt.LT_OK else 1


if __name__ == "__main__":
    sys.exit(main())
