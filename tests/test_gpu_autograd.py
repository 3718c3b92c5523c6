"""The torch.autograd path (lt.chi2_autograd): its backward pass is the
library's adjoint, scaled by the upstream gradient and laid out like the
parameter tensor, and it agrees with the oracle's dual-number gradient."""
import json
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


def test_autograd_matches_adjoint_and_oracle(oracle):
    w = W.c3(batch=3)
    with open(os.path.join(GOLDEN, "obs_c3.json")) as f:
        o = json.load(f)
    grids = [g.as_tuple() for g in w.grids]
    obs = lt.Observations.from_dict(o)
    m = lt.Model(w.n_pot, w.batch)
    params = torch.tensor(w.params, dtype=torch.float64, device="cuda", requires_grad=True)
    c2 = lt.chi2_autograd(m, params, grids, obs)
    weights = torch.tensor([1.0, -2.0, 0.5], dtype=torch.float64, device="cuda")
    (c2 * weights).sum().backward()
    st, _ = m.sync()
    assert st == lt.LT_OK
    gp = params.grad.cpu().numpy()
    # rows without a gradient
    assert np.all(gp[:, 0, :] == 0) and np.all(gp[:, 6, :] == 0)
    # the adjoint itself
    c2b, g = m.chi2_grad(grids, obs)
    g = g.cpu().numpy()
    np.testing.assert_array_equal(c2.detach().cpu().numpy(), c2b.cpu().numpy())
    for b, wb in enumerate([1.0, -2.0, 0.5]):
        np.testing.assert_allclose(gp[b][list(lt.GRAD_ROWS)], wb * g[b].T, rtol=1e-15, atol=0)
    # the oracle's gradient with the same frozen assignment
    mt, _, _ = m.last_matches(len(o["x"]), len(o["dls_ds"]))
    mt = mt.cpu().numpy()
    for b in range(w.batch):
        _, rg = oracle.chi2_grad(w.params[b], grids[b], o, mt[b])
        scale = np.abs(rg).max()
        np.testing.assert_allclose(g[b], rg, rtol=1e-3, atol=1e-6 * scale)
    m.close()


def test_no_grad_forward_is_plain_chi2():
    w = W.c1()
    with open(os.path.join(GOLDEN, "obs_c1.json")) as f:
        o = json.load(f)
    obs = lt.Observations.from_dict(o)
    m = lt.Model(w.n_pot, 1)
    params = torch.tensor(w.params, dtype=torch.float64, device="cuda")
    c2 = lt.chi2_autograd(m, params, [w.grids[0].as_tuple()], obs, precision=lt.FP64)
    ref = m.chi2([w.grids[0].as_tuple()], obs, precision=lt.FP64)
    assert float(c2[0]) == float(ref[0])
    m.close()
