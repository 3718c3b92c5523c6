"""Seeded synthetic workloads for the image-plane chi^2 path.

This module only draws random numbers and lays out grids; it performs none of
the lensing arithmetic (no deflection, no lens equation, no triangle test).
Both the CUDA path and the FP64 oracle take what it produces as plain inputs.

Parameter layout (shared with the C ABI): one float64 array of shape
``[batch][8][n_pot]`` whose rows are ``kind, x, y, e, phi, r_core, r_cut,
sigma_v`` (arcsec, arcsec, arcsec, -, rad, arcsec, arcsec, km/s).  ``kind`` is
0 = SIS, 1 = PIEMD (dPIE), 2 = SIE (the paper's Algorithm 1).

Workloads (the paper's benchmark description is Sect. 4; the cluster,
batched, gradient and large cases are synthetic stand-ins with the shapes of
a LENSTOOL model fit, Sect. 2.2.1):

* ``c1``  one SIS at the origin, effective Einstein radius 10", D_ls/D_s = 0.7,
          256^2 nodes over 100"x100", point source at (2.0", 1.5").
* ``c2``  100 PIEMD, centres U[-100,100]^2, e U[0,0.5], phi U[0,pi),
          r_core U[0.05,1], r_cut U[50,200], sigma_v log-U[50,1200];
          20 sources with D_ls/D_s U[0.3,0.9]; 2000^2 nodes over 200".
* ``c3``  1024 samples of a 50-PIEMD base draw, each continuous parameter
          times (1 + 0.01 N(0,1)); grid sides U_int[500,2000] over 200";
          10 sources.
* ``c4``  100 PIEMD, 20 sources, 1000^2 nodes over 200" (gradient case).
* ``c5``  1000 PIEMD, sigma_v log-U[30,1500] in a 400" field, 4000^2 nodes,
          100 sources, 64 perturbed samples.
* ``hff`` the paper's HFF-like benchmark (Sect. 4): 6730^2 pixels at 0.03",
          2 cluster SIE (sigma_v 1000 and 700 km/s, eps 0.05 and 0.04) and 700
          galaxy SIE (sigma_v U[10,15] km/s, eps U[0,0.15]).

Seeds: ``config_index * 1000 + stream``; every stream is a numpy
``default_rng`` so the draws are identical on every machine.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SIS, PIEMD, SIE = 0, 1, 2
N_ROWS = 8  # kind, x, y, e, phi, r_core, r_cut, sigma_v
C_KMS = 299792.458
ARCSEC_PER_RAD = 206264.80625


@dataclass
class Grid:
    """Node (i, j) sits at (x0 + i*dx, y0 + j*dy), i < nx, j < ny."""

    x0: float
    y0: float
    dx: float
    dy: float
    nx: int
    ny: int

    @staticmethod
    def square(side: float, n: int) -> "Grid":
        """n x n nodes spanning [-side/2, side/2]^2, both edges included."""
        h = side / (n - 1)
        return Grid(-side / 2, -side / 2, h, h, n, n)

    @property
    def nodes(self) -> int:
        return self.nx * self.ny

    @property
    def triangles(self) -> int:
        return 2 * (self.nx - 1) * (self.ny - 1)

    def as_tuple(self):
        return (self.x0, self.y0, self.dx, self.dy, self.nx, self.ny)


@dataclass
class Workload:
    name: str
    params: np.ndarray            # [batch][8][n_pot] float64
    grids: list                   # [batch] Grid
    n_src: int                    # systems (sources) per sample
    seed_base: int
    obs_grid: Grid | None = None  # grid the stored observations were found on
    notes: dict = field(default_factory=dict)

    @property
    def batch(self) -> int:
        return self.params.shape[0]

    @property
    def n_pot(self) -> int:
        return self.params.shape[2]

    def node_pot(self) -> int:
        return sum(g.nodes for g in self.grids) * self.n_pot


def _rng(cfg_index: int, stream: int) -> np.random.Generator:
    return np.random.default_rng(cfg_index * 1000 + stream)


def sigma_for_einstein_radius(theta_e: float, dls_ds: float) -> float:
    """Velocity dispersion (km/s) whose SIS has effective Einstein radius
    ``theta_e`` (arcsec) for a source at D_ls/D_s = ``dls_ds``.

    Input preparation only: inverts the SIS normalisation of Sect. 2.1
    (theta_E = 4 pi (sigma_v/c)^2 D_LS/D_OS) so a workload can be stated by
    its Einstein radius.
    """
    return C_KMS * math.sqrt(theta_e / (dls_ds * 4.0 * math.pi * ARCSEC_PER_RAD))


def draw_piemd(rng: np.random.Generator, n_pot: int, half_field: float,
               sigma_lo: float, sigma_hi: float) -> np.ndarray:
    """One cluster draw of ``n_pot`` PIEMD potentials, shape [8][n_pot]."""
    p = np.zeros((N_ROWS, n_pot))
    p[0] = PIEMD
    p[1] = rng.uniform(-half_field, half_field, n_pot)
    p[2] = rng.uniform(-half_field, half_field, n_pot)
    p[3] = rng.uniform(0.0, 0.5, n_pot)
    p[4] = rng.uniform(0.0, math.pi, n_pot)
    p[5] = rng.uniform(0.05, 1.0, n_pot)
    p[6] = rng.uniform(50.0, 200.0, n_pot)
    p[7] = np.exp(rng.uniform(math.log(sigma_lo), math.log(sigma_hi), n_pot))
    return p


def perturb(base: np.ndarray, rng: np.random.Generator, batch: int,
            rel: float = 0.01) -> np.ndarray:
    """MCMC-like proposals: every continuous parameter times (1 + rel N(0,1)).

    e is clamped to [0, 0.9], r_core to >= 1e-3", r_cut to > 1.5 r_core.
    """
    out = np.repeat(base[None], batch, axis=0).copy()
    noise = rng.standard_normal((batch, N_ROWS - 1, base.shape[1]))
    out[:, 1:, :] *= 1.0 + rel * noise
    out[:, 3, :] = np.clip(out[:, 3, :], 0.0, 0.9)
    out[:, 5, :] = np.maximum(out[:, 5, :], 1e-3)
    out[:, 6, :] = np.maximum(out[:, 6, :], 1.5 * out[:, 5, :])
    out[:, 7, :] = np.abs(out[:, 7, :])
    return out


def source_candidates(cfg_index: int, n: int, half_field: float,
                      r_lo: float = 0.3, r_hi: float = 0.9) -> np.ndarray:
    """Candidate sources, shape [n][3] = (beta_x, beta_y, D_ls/D_s).

    Positions are uniform in the central half of the field; the caller keeps
    those that the oracle finds multiply imaged (strong-lensing systems).
    """
    rng = _rng(cfg_index, 500)
    xy = rng.uniform(-half_field / 2, half_field / 2, (n, 2))
    r = rng.uniform(r_lo, r_hi, n)
    return np.column_stack([xy, r])


def position_noise(cfg_index: int, n: int, sigma: float = 0.01) -> np.ndarray:
    """Astrometric noise for ``n`` observed images, shape [n][2] (arcsec)."""
    return _rng(cfg_index, 600).normal(0.0, sigma, (n, 2))


def c1() -> Workload:
    r = 0.7
    p = np.zeros((1, N_ROWS, 1))
    p[0, :, 0] = [SIS, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0,
                  sigma_for_einstein_radius(10.0, r)]
    g = Grid.square(100.0, 256)
    return Workload("c1", p, [g], 1, 1000, obs_grid=g,
                    notes={"source": (2.0, 1.5), "dls_ds": r, "theta_e": 10.0})


def c2() -> Workload:
    p = draw_piemd(_rng(2, 0), 100, 100.0, 50.0, 1200.0)[None]
    g = Grid.square(200.0, 2000)
    return Workload("c2", p, [g], 20, 2000, obs_grid=g)


def c3(batch: int = 1024) -> Workload:
    base = draw_piemd(_rng(3, 0), 50, 100.0, 50.0, 1200.0)
    rng = _rng(3, 1)
    params = perturb(base, rng, 1024)[:batch]
    sides = _rng(3, 2).integers(500, 2001, 1024)[:batch]
    grids = [Grid.square(200.0, int(n)) for n in sides]
    return Workload("c3", params, grids, 10, 3000,
                    obs_grid=Grid.square(200.0, 2000), notes={"base": base})


def c4() -> Workload:
    p = draw_piemd(_rng(4, 0), 100, 100.0, 50.0, 1200.0)[None]
    g = Grid.square(200.0, 1000)
    return Workload("c4", p, [g], 20, 4000, obs_grid=g)


def c5(batch: int = 64) -> Workload:
    base = draw_piemd(_rng(5, 0), 1000, 200.0, 30.0, 1500.0)
    params = perturb(base, _rng(5, 1), 64)[:batch]
    g = Grid.square(400.0, 4000)
    # observations are found on a coarser grid of the same field (oracle cost)
    return Workload("c5", params, [g] * batch, 100, 5000,
                    obs_grid=Grid.square(400.0, 1000), notes={"base": base})


def hff(n: int = 6730, pixel: float = 0.03) -> Workload:
    """The paper's HFF-like benchmark lens (Sect. 4), SIE potentials."""
    rng = _rng(6, 0)
    side = (n - 1) * pixel
    half = side / 2
    n_gal = 700
    p = np.zeros((N_ROWS, 2 + n_gal))
    p[0] = SIE
    # two cluster-scale halos near the field centre (Abell 2744-like merger)
    p[1, :2] = rng.uniform(-0.15 * half, 0.15 * half, 2)
    p[2, :2] = rng.uniform(-0.15 * half, 0.15 * half, 2)
    p[3, :2] = [0.05, 0.04]
    p[7, :2] = [1000.0, 700.0]
    p[1, 2:] = rng.uniform(-half, half, n_gal)
    p[2, 2:] = rng.uniform(-half, half, n_gal)
    p[3, 2:] = rng.uniform(0.0, 0.15, n_gal)
    p[7, 2:] = rng.uniform(10.0, 15.0, n_gal)
    p[4] = rng.uniform(0.0, math.pi, 2 + n_gal)
    g = Grid(-half, -half, pixel, pixel, n, n)
    return Workload("hff", p[None], [g], 0, 6000)




def c2_proposal(rank: int) -> np.ndarray:
    """The c2 lens as proposal number ``rank`` of independent sampler chains,
    shape [1][8][n_pot]: rank 0 is the c2 draw itself, every other rank a
    perturbation of it (each continuous parameter times 1 + 0.01 N(0,1),
    seeded by the rank), so that every rank evaluates its own proposal."""
    base = c2().params[0]
    if rank == 0:
        return base[None].copy()
    return perturb(base, _rng(2, 100 + rank), 1)


CONFIGS = {"c1": c1, "c2": c2, "c3": c3, "c4": c4, "c5": c5, "hff": hff}
