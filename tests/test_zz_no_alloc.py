"""The allocation-free deflection entry point, lt_deflect_grid_noalloc.

It exists for callers that cannot allocate device memory (allocator hooks,
memory-pool callbacks, plugins of applications that own every device
allocation): its scratch is a fixed device array inside the library.  These
tests call it through the C ABI on two calls in a row with different models,
so that the second call runs on the scratch contents the first one left
behind, and check each call
* against the FP64 oracle directly: every node within the FP32 running error
  bound the call itself returns, the bar of the other deflection tests;
* against the model-based lt_deflect_grid in mixed precision: the same
  arithmetic in the same order, so deflection and bound are bit-identical;
* for allocations: the device's free memory is the same before and after a
  call.
This file is collected last; it passes alone in a fresh process and after the
others.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1902_03252_gb300 import lt, workloads as W  # noqa: E402

MAX_POT = 4096


@pytest.fixture(scope="module")
def noalloc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    L = lt.load(build_if_missing=True)
    f = L.lt_deflect_grid_noalloc
    f.argtypes = [C.c_void_p, C.c_int32, C.POINTER(lt.Grid), C.c_void_p, C.c_void_p,
                  C.c_void_p, C.c_size_t]
    f.restype = C.c_int
    return f


def call(f, params, grid):
    """One call on the current stream; outputs pre-filled with NaN."""
    p = torch.as_tensor(np.ascontiguousarray(params), dtype=torch.float64, device="cuda")
    g = lt.grids_array([grid])
    ny, nx = g[0].ny, g[0].nx
    a = torch.full((ny, nx, 2), float("nan"), dtype=torch.float32, device="cuda")
    e = torch.full((ny, nx), float("nan"), dtype=torch.float32, device="cuda")
    st = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    rc = f(p.data_ptr(), p.shape[1], g, a.data_ptr(), e.data_ptr(), st.data_ptr(),
           torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return rc, a, e, int(st.item())


def reference(params, grid):
    m = lt.Model(params.shape[1], 1)
    m.set_params(params[None])
    a, e = m.deflect_grid(grid, precision=lt.MIXED, with_error=True)
    assert m.sync()[0] == lt.LT_OK
    out = a.cpu().numpy().astype(np.float64), e.cpu().numpy().astype(np.float64)
    m.close()
    return out


def models():
    big = W.c2().params[0]                      # 100 PIEMD
    rng = np.random.default_rng(5)
    small = W.draw_piemd(rng, 37, 30.0, 100.0, 900.0)
    small[0, ::5] = W.SIS                       # mixed kinds, fewer potentials
    small[0, 2::5] = W.SIE
    small[3, 2::5] = rng.uniform(0, 0.3, small[3, 2::5].shape)
    return [big, small]


def test_two_calls_in_a_row_match_oracle_and_model_path(noalloc, oracle):
    grid = (-100.0, -100.0, 200.0 / 499, 200.0 / 499, 500, 500)
    for params in models():
        ref_a, ref_e = reference(params, grid)
        rc, a, e, st = call(noalloc, params, grid)
        assert rc == lt.LT_OK and st == lt.LT_OK
        a, e = a.cpu().numpy().astype(np.float64), e.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(a)) and np.all(np.isfinite(e)) and np.all(e > 0)
        # the oracle: |alpha_FP32 - alpha_FP64| within the call's own bound
        exact, _ = oracle.deflect_grid(params, grid, n_threads=4)
        assert np.all(np.abs(a - exact).max(axis=-1) <= e)
        # the model path: bit-identical deflection and bound
        np.testing.assert_array_equal(a, ref_a)
        np.testing.assert_array_equal(e, ref_e)


def test_call_allocates_no_device_memory(noalloc):
    grid = (-100.0, -100.0, 200.0 / 299, 200.0 / 299, 300, 300)
    params = models()[1]
    call(noalloc, params, grid)  # first call: module and scratch set-up
    p = torch.as_tensor(np.ascontiguousarray(params), dtype=torch.float64, device="cuda")
    g = lt.grids_array([grid])
    a = torch.empty((300, 300, 2), dtype=torch.float32, device="cuda")
    e = torch.empty((300, 300), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        rc = noalloc(p.data_ptr(), p.shape[1], g, a.data_ptr(), e.data_ptr(), None,
                     torch.cuda.current_stream().cuda_stream)
        assert rc == lt.LT_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_rejects_models_beyond_its_scratch(noalloc):
    grid = (0.0, 0.0, 1.0, 1.0, 8, 8)
    p = np.zeros((8, MAX_POT + 1))
    rc, a, e, st = call(noalloc, p, grid)
    assert rc == lt.LT_ERR_INVALID_ARG
    assert st == -1 and torch.isnan(a).all()  # nothing was launched
