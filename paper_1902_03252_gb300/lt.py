"""ctypes binding of the C ABI in include/lt.h (argument marshalling only).

Every step of the chi^2 path runs in the CUDA library; PyTorch provides
device memory and the current stream.  Importing this module does not load
the library; the first call does, and raises if it has not been built or no
CUDA device is present -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import _build

LT_OK, LT_ERR_INVALID_ARG, LT_ERR_CUDA, LT_ERR_NOMEM, LT_ERR_OVERFLOW, LT_ERR_TIMEOUT, \
    LT_ERR_NONFINITE = range(7)
LT_SIS, LT_PIEMD, LT_SIE = 0, 1, 2
FP64, MIXED, PAPER = 0, 1, 2
N_ROWS, N_GRAD = 8, 6
POS_TOL = 2.5e-5

EXPORTED = ("lt_model_create", "lt_model_destroy", "lt_last_error", "lt_status_string",
            "lt_model_set_params", "lt_deflect_grid", "lt_find_images", "lt_chi2",
            "lt_chi2_grad", "lt_last_matches", "lt_model_sync", "lt_chi2_graph",
            "lt_autotune", "lt_profile_enable", "lt_profile_read", "lt_dls_ds",
            "lt_chi2_source", "lt_last_magnifications", "lt_model_set_shape",
            "lt_num_shapes", "lt_profile_stages", "lt_version")


class Grid(C.Structure):
    _fields_ = [("x0", C.c_double), ("y0", C.c_double), ("dx", C.c_double), ("dy", C.c_double),
                ("nx", C.c_int32), ("ny", C.c_int32)]


class ModelDesc(C.Structure):
    _fields_ = [("n_pot", C.c_int32), ("batch", C.c_int32), ("hit_capacity", C.c_int64)]


class Image(C.Structure):
    _fields_ = [("sample", C.c_int32), ("src", C.c_int32), ("tri", C.c_int64),
                ("x", C.c_double), ("y", C.c_double), ("w", C.c_double * 3),
                ("fp64", C.c_int32), ("reserved", C.c_int32)]


class Obs(C.Structure):
    _fields_ = [("n_obs", C.c_int32), ("n_sys", C.c_int32), ("x", C.c_void_p),
                ("y", C.c_void_p), ("sigma", C.c_void_p), ("sys", C.c_void_p),
                ("dls_ds", C.c_void_p)]


class Stats(C.Structure):
    _fields_ = [("hits", C.c_int64), ("ambiguous", C.c_int64), ("refined", C.c_int64),
                ("fp64_nodes", C.c_int64), ("work_overflow", C.c_int64),
                ("tight_nodes", C.c_int64), ("fp64_items", C.c_int64)]


class Profile(C.Structure):
    _fields_ = [("launches", C.c_int64 * 5), ("ms", C.c_double * 5),
                ("node_pot", C.c_double * 2)]


# stages 0-3 run in sequence on the caller's stream; "bary" runs on the
# model's side stream, overlapping the deflection
PROFILE_KINDS = ("deflect", "search", "resolve", "chi2", "bary")

IMAGE_DTYPE = np.dtype([("sample", "<i4"), ("src", "<i4"), ("tri", "<i8"), ("x", "<f8"),
                        ("y", "<f8"), ("w", "<f8", (3,)), ("fp64", "<i4"), ("reserved", "<i4")])
assert IMAGE_DTYPE.itemsize == C.sizeof(Image) == 64


class LTError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load the CUDA library (optionally building it first)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"CUDA library not built: {path} missing "
                               "(run `python -c \"import __graft_entry__ as g; g.build()\"`)")
        _build.build()
    L = C.CDLL(path)
    vp, i32, i64, st = C.c_void_p, C.c_int32, C.c_int64, C.c_int
    up = C.c_size_t  # uintptr_t
    L.lt_model_create.argtypes = [C.POINTER(ModelDesc), C.POINTER(vp)]
    L.lt_model_destroy.argtypes = [vp]
    L.lt_model_destroy.restype = None
    L.lt_last_error.argtypes = [vp]
    L.lt_last_error.restype = C.c_char_p
    L.lt_status_string.argtypes = [st]
    L.lt_status_string.restype = C.c_char_p
    L.lt_version.restype = C.c_char_p
    L.lt_model_set_params.argtypes = [vp, vp, C.c_int, up]
    L.lt_deflect_grid.argtypes = [vp, i32, C.POINTER(Grid), st, vp, vp, up]
    L.lt_find_images.argtypes = [vp, C.POINTER(Grid), i32, vp, vp, st, i64, vp, vp, up]
    L.lt_chi2.argtypes = [vp, C.POINTER(Grid), C.POINTER(Obs), st, vp, up]
    L.lt_chi2_graph.argtypes = [vp, C.POINTER(Grid), C.POINTER(Obs), st, vp, up]
    L.lt_chi2_grad.argtypes = [vp, C.POINTER(Grid), C.POINTER(Obs), st, vp, vp, up]
    L.lt_last_matches.argtypes = [vp, vp, vp, vp, up]
    L.lt_chi2_source.argtypes = [vp, C.POINTER(Obs), vp, vp, up]
    L.lt_model_set_shape.argtypes = [vp, i32]
    L.lt_num_shapes.restype = i32
    L.lt_last_magnifications.argtypes = [vp, C.POINTER(Obs), vp, up]
    L.lt_model_sync.argtypes = [vp, up, C.POINTER(Stats)]
    L.lt_autotune.argtypes = [vp, C.POINTER(Grid), up, C.POINTER(i32)]
    L.lt_profile_enable.argtypes = [vp, C.c_int]
    L.lt_profile_read.argtypes = [vp, C.POINTER(Profile), C.c_int]
    L.lt_profile_stages.argtypes = [vp, C.c_uint32]
    L.lt_dls_ds.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double,
                            C.POINTER(C.c_double)]
    for name in EXPORTED:
        f = getattr(L, name)
        if f.restype is C.c_int or name in ("lt_model_create", "lt_model_set_params",
                                            "lt_deflect_grid", "lt_find_images", "lt_chi2",
                                            "lt_chi2_graph", "lt_chi2_grad", "lt_last_matches",
                                            "lt_model_sync", "lt_autotune",
                                            "lt_profile_enable", "lt_profile_read",
                                            "lt_dls_ds", "lt_chi2_source",
                                            "lt_last_magnifications", "lt_model_set_shape",
                                            "lt_profile_stages"):
            f.restype = st
    _lib = L
    return L


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("no CUDA device: this library has no CPU path")
    return torch


def _stream(stream=None) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _ptr(t) -> int:
    return int(t.data_ptr()) if t is not None else 0


def grids_array(grids):
    """Marshal a sequence of grids ((x0, y0, dx, dy, nx, ny) or objects with
    ``as_tuple``) into a host lt_grid array."""
    arr = (Grid * len(grids))()
    for k, g in enumerate(grids):
        t = g.as_tuple() if hasattr(g, "as_tuple") else tuple(g)
        arr[k] = Grid(float(t[0]), float(t[1]), float(t[2]), float(t[3]), int(t[4]), int(t[5]))
    return arr


@dataclass
class Observations:
    """Observed images on the device (float64 / int32 torch tensors)."""
    x: object
    y: object
    sigma: object
    sys: object
    dls_ds: object

    @staticmethod
    def from_numpy(x, y, sigma, sys, dls_ds, device="cuda"):
        torch = _torch()
        d = lambda a, t: torch.as_tensor(np.ascontiguousarray(a), dtype=t, device=device)
        return Observations(d(x, torch.float64), d(y, torch.float64), d(sigma, torch.float64),
                            d(sys, torch.int32), d(dls_ds, torch.float64))

    @staticmethod
    def from_dict(o, device="cuda"):
        return Observations.from_numpy(o["x"], o["y"], o["sigma"], o["sys"], o["dls_ds"], device)

    def c_struct(self) -> Obs:
        return Obs(int(self.x.numel()), int(self.dls_ds.numel()), _ptr(self.x), _ptr(self.y),
                   _ptr(self.sigma), _ptr(self.sys), _ptr(self.dls_ds))


class Model:
    """A batch of lens-parameter samples on the current CUDA device."""

    def __init__(self, n_pot: int, batch: int = 1, hit_capacity: int = 0):
        self._lib = load()
        _torch()
        h = C.c_void_p()
        st = self._lib.lt_model_create(C.byref(ModelDesc(n_pot, batch, hit_capacity)), C.byref(h))
        if st != LT_OK:
            raise LTError(st, f"lt_model_create failed: {self._lib.lt_status_string(st).decode()}")
        self.h = h
        self.n_pot, self.batch = n_pot, batch

    def close(self):
        if getattr(self, "h", None):
            self._lib.lt_model_destroy(self.h)
            self.h = None

    __del__ = close

    def _check(self, st, what):
        if st != LT_OK:
            raise LTError(st, f"{what}: {self._lib.lt_last_error(self.h).decode()}")

    def set_params(self, params, stream=None):
        """params: [batch][8][n_pot] float64 (numpy on the host or a CUDA tensor)."""
        torch = _torch()
        if isinstance(params, torch.Tensor) and params.is_cuda:
            p = params.detach().to(torch.float64).contiguous()
            assert tuple(p.shape) == (self.batch, N_ROWS, self.n_pot), tuple(p.shape)
            self._keep = p
            self._check(self._lib.lt_model_set_params(self.h, _ptr(p), 1, _stream(stream)),
                        "lt_model_set_params")
        else:
            p = np.ascontiguousarray(params, dtype=np.float64)
            assert p.shape == (self.batch, N_ROWS, self.n_pot), p.shape
            self._keep = p
            self._check(self._lib.lt_model_set_params(self.h, p.ctypes.data, 0, _stream(stream)),
                        "lt_model_set_params")

    def deflect_grid(self, grid, precision=MIXED, sample=0, with_error=False, stream=None):
        """[ny][nx][2] deflection (float32 for MIXED, float64 for FP64 and PAPER)
        as a CUDA tensor, plus the per-node FP32 error bound (MIXED) or the
        FP64-recomputation map (PAPER) when ``with_error``."""
        torch = _torch()
        g = grids_array([grid])
        nx, ny = g[0].nx, g[0].ny
        dt = torch.float32 if precision == MIXED else torch.float64
        a = torch.empty((ny, nx, 2), dtype=dt, device="cuda")
        e = torch.empty((ny, nx), dtype=torch.float32, device="cuda") if with_error else None
        self._check(self._lib.lt_deflect_grid(self.h, sample, g, precision, _ptr(a), _ptr(e),
                                              _stream(stream)), "lt_deflect_grid")
        return (a, e) if with_error else a

    def find_images(self, grids, src_xy, dls_ds, precision=MIXED, capacity=4096, stream=None):
        """Images of explicit sources: src_xy [batch][n_src][2], dls_ds [batch][n_src]
        (CUDA float64 tensors).  Returns (images uint8 view [batch][capacity][64], counts)."""
        torch = _torch()
        g = grids_array(grids)
        n_src = int(src_xy.shape[1]) if src_xy is not None else 0
        out = torch.empty((self.batch, capacity, 64), dtype=torch.uint8, device="cuda")
        n = torch.empty((self.batch,), dtype=torch.int64, device="cuda")
        self._check(self._lib.lt_find_images(self.h, g, n_src, _ptr(src_xy), _ptr(dls_ds),
                                             precision, capacity, _ptr(out), _ptr(n),
                                             _stream(stream)), "lt_find_images")
        return out, n

    def chi2(self, grids, obs: Observations, precision=MIXED, out=None, graph=False, stream=None):
        torch = _torch()
        g = grids_array(grids)
        if out is None:
            out = torch.empty((self.batch,), dtype=torch.float64, device="cuda")
        self._obs = obs
        fn = self._lib.lt_chi2_graph if graph else self._lib.lt_chi2
        self._check(fn(self.h, g, C.byref(obs.c_struct()), precision, _ptr(out), _stream(stream)),
                    "lt_chi2")
        return out

    def chi2_grad(self, grids, obs: Observations, precision=MIXED, stream=None):
        torch = _torch()
        g = grids_array(grids)
        c2 = torch.empty((self.batch,), dtype=torch.float64, device="cuda")
        gr = torch.empty((self.batch, self.n_pot, N_GRAD), dtype=torch.float64, device="cuda")
        self._obs = obs
        self._check(self._lib.lt_chi2_grad(self.h, g, C.byref(obs.c_struct()), precision,
                                           _ptr(c2), _ptr(gr), _stream(stream)), "lt_chi2_grad")
        return c2, gr

    def num_shapes(self) -> int:
        """Number of launch shapes of the FP32 deflection (lt_num_shapes)."""
        return int(self._lib.lt_num_shapes())

    def set_shape(self, shape: int):
        """Pin the FP32 deflection launch shape (index into the shape table)."""
        self._check(self._lib.lt_model_set_shape(self.h, int(shape)), "lt_model_set_shape")

    def chi2_source(self, obs: Observations, stream=None):
        """Source-plane chi^2 [batch] and point magnifications [batch][n_obs]."""
        torch = _torch()
        c2 = torch.empty((self.batch,), dtype=torch.float64, device="cuda")
        mu = torch.empty((self.batch, int(obs.x.numel())), dtype=torch.float64, device="cuda")
        self._check(self._lib.lt_chi2_source(self.h, C.byref(obs.c_struct()), _ptr(c2), _ptr(mu),
                                             _stream(stream)), "lt_chi2_source")
        return c2, mu

    def last_magnifications(self, obs: Observations, stream=None):
        """Signed triangle magnification of each observed image's matched
        predicted image in the last chi^2 evaluation [batch][n_obs] (NaN: no match)."""
        torch = _torch()
        mu = torch.empty((self.batch, int(obs.x.numel())), dtype=torch.float64, device="cuda")
        self._check(self._lib.lt_last_magnifications(self.h, C.byref(obs.c_struct()), _ptr(mu),
                                                     _stream(stream)), "lt_last_magnifications")
        return mu

    def last_matches(self, n_obs, n_sys, stream=None):
        torch = _torch()
        mt = torch.empty((self.batch, n_obs), dtype=torch.int64, device="cuda")
        mxy = torch.empty((self.batch, n_obs, 2), dtype=torch.float64, device="cuda")
        b = torch.empty((self.batch, n_sys, 2), dtype=torch.float64, device="cuda")
        self._check(self._lib.lt_last_matches(self.h, _ptr(mt), _ptr(mxy), _ptr(b),
                                              _stream(stream)), "lt_last_matches")
        return mt, mxy, b

    def sync(self, stream=None):
        """Wait for the model's work; returns (status, stats dict)."""
        s = Stats()
        st = self._lib.lt_model_sync(self.h, _stream(stream), C.byref(s))
        return st, {k: getattr(s, k) for k, _ in Stats._fields_}

    def profile(self, on: bool = True, stages=None):
        """Enable / disable per-stage CUDA-event timing of later calls; stages:
        optional subset of PROFILE_KINDS (default: all)."""
        if stages is None:
            self._check(self._lib.lt_profile_enable(self.h, 1 if on else 0), "lt_profile_enable")
        else:
            mask = sum(1 << PROFILE_KINDS.index(k) for k in stages) if on else 0
            self._check(self._lib.lt_profile_stages(self.h, mask), "lt_profile_stages")

    def profile_read(self, reset: bool = True):
        """Per-kernel launches and summed milliseconds since the last reset."""
        p = Profile()
        self._check(self._lib.lt_profile_read(self.h, C.byref(p), 1 if reset else 0),
                    "lt_profile_read")
        out = {k: {"launches": p.launches[i], "ms": p.ms[i]} for i, k in enumerate(PROFILE_KINDS)}
        out["deflect"]["node_pot_fp32"] = p.node_pot[0]
        out["deflect"]["node_pot_fp64"] = p.node_pot[1]
        return out

    def autotune(self, grid, stream=None):
        ch = C.c_int32(-1)
        self._check(self._lib.lt_autotune(self.h, grids_array([grid]), _stream(stream),
                                          C.byref(ch)), "lt_autotune")
        return ch.value


# parameter rows that the adjoint differentiates, in its column order:
# x, y, e, phi, r_core, sigma_v
GRAD_ROWS = (1, 2, 3, 4, 5, 7)
_chi2_fn = None


def _chi2_function():
    global _chi2_fn
    if _chi2_fn is None:
        torch = _torch()

        class Chi2(torch.autograd.Function):
            """chi^2 of every sample as a differentiable function of the
            parameter tensor; the backward pass is the library's adjoint
            (lt_chi2_grad, triangle assignment held fixed)."""

            @staticmethod
            def forward(ctx, params, model, grids, obs, precision):
                model.set_params(params)
                if ctx.needs_input_grad[0]:
                    c2, g = model.chi2_grad(grids, obs, precision=precision)
                    ctx.save_for_backward(g)
                else:
                    c2 = model.chi2(grids, obs, precision=precision)
                return c2

            @staticmethod
            def backward(ctx, gout):
                (g,) = ctx.saved_tensors  # [batch][n_pot][6]
                b, n_pot, _ = g.shape
                gp = torch.zeros((b, N_ROWS, n_pot), dtype=torch.float64, device=g.device)
                gp[:, list(GRAD_ROWS), :] = (g * gout.to(g.dtype)[:, None, None]).transpose(1, 2)
                return gp, None, None, None, None

        _chi2_fn = Chi2
    return _chi2_fn


def chi2_autograd(model, params, grids, obs, precision=MIXED):
    """chi^2 [batch] of ``params`` ([batch][8][n_pot] float64 CUDA tensor) with
    autograd support.  Gradients flow to the rows x, y, e, phi, r_core and
    sigma_v; kind (discrete) and r_cut are held constant (their gradient is
    zero)."""
    return _chi2_function().apply(params, model, grids, obs, precision)


def dls_ds(z_l: float, z_s: float, omega_m: float = 0.3, omega_lambda: float = 0.7) -> float:
    """D_ls/D_s for a lens at z_l and a source at z_s (host computation)."""
    out = C.c_double(0.0)
    st = load().lt_dls_ds(z_l, z_s, omega_m, omega_lambda, C.byref(out))
    if st != LT_OK:
        raise LTError(st, "lt_dls_ds: invalid redshifts or cosmology")
    return out.value


def images_to_numpy(out, counts):
    """Decode find_images output into per-sample numpy record arrays."""
    o = out.cpu().numpy()
    n = counts.cpu().numpy()
    res = []
    for b in range(o.shape[0]):
        k = int(min(n[b], o.shape[1]))
        res.append(np.frombuffer(o[b, :k].tobytes(), dtype=IMAGE_DTYPE))
    return res
