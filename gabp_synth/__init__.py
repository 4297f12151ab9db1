"""Seeded synthetic inputs for the Gaussian belief propagation data-assimilation problem.

This module is shared by the CPU oracle, the tests and the benchmark, so it holds
only random draws and data synthesis; none of the message-passing arithmetic lives
here.  It produces, for a 2-D grid of ``nx * ny`` nodes at unit spacing:

* a ground-truth field ``truth`` drawn from the SPDE prior of Sec. 3.1 (Eq. for the
  discretised SPDE, ``L f = w``, ``w ~ N(0, I)``, gamma = 1), with
  ``L = kappa^2 I - Delta_h`` and a zero-Neumann (cell-centred ghost) boundary.
  ``L`` is diagonalised by the orthonormal 2-D DCT-II, so the sample is drawn
  spectrally with ``scipy.fft``;
* observation locations in grid units (``obs_x`` along columns, ``obs_y`` along rows,
  both in ``[0, n-1]``), either uniform-random points (the paper's synthetic
  experiment observes a random subset of the grid, Sec. 4.1) or straight
  satellite-like ground tracks (the paper's large-scale example uses satellite
  ground tracks, Sec. 4.2);
* observed values ``y = truth(obs) + sigma * eps`` where ``truth(obs)`` is the
  bilinear reading of the truth field (``scipy.ndimage.map_coordinates``, order 1)
  and ``eps ~ N(0, 1)``;
* per-observation noise variances ``noise_var = sigma^2``.

Track reading (the configurations only give "tracks at uniform-random angles and
offsets, one sample per 1.5 cells"): each track is a line through a uniform-random
point at angle ``theta ~ U[0, pi)``, wrapped around the domain like a repeating
orbit, and sampled every 1.5 cells along its length.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Problem", "neumann_eigenvalues", "sample_truth", "uniform_points", "track_points",
    "make_problem", "config_small", "config_tracks_1024", "config_roofline_4096",
    "config_batch", "config_warm_train", "config_warm_eval", "scaled_config",
]


@dataclass
class Problem:
    nx: int
    ny: int
    kappa: float
    obs_x: np.ndarray            # (m,) float64, column coordinate in [0, nx-1]
    obs_y: np.ndarray            # (m,) float64, row coordinate in [0, ny-1]
    y: np.ndarray                # (m,) float64 observed values
    noise_var: np.ndarray        # (m,) float64 observation noise variances
    truth: np.ndarray | None = None  # (ny, nx) float64 ground truth, row-major
    meta: dict = field(default_factory=dict)
    gamma: float = 1.0               # prior scale (precision gamma L^T L)

    @property
    def n(self) -> int:
        return self.nx * self.ny

    @property
    def m(self) -> int:
        return int(self.obs_x.shape[0])


def neumann_eigenvalues(nx: int, ny: int, kappa: float) -> np.ndarray:
    """Eigenvalues of ``L = kappa^2 I + (graph Laplacian, zero-Neumann)`` on the DCT-II basis.

    Returned with shape ``(ny, nx)``: ``kappa^2 + 4 sin^2(pi l / 2 ny) + 4 sin^2(pi k / 2 nx)``.
    """
    kx = 4.0 * np.sin(np.pi * np.arange(nx) / (2.0 * nx)) ** 2
    ky = 4.0 * np.sin(np.pi * np.arange(ny) / (2.0 * ny)) ** 2
    return kappa * kappa + ky[:, None] + kx[None, :]


def sample_truth(nx: int, ny: int, kappa: float, rng: np.random.Generator) -> np.ndarray:
    """Draw ``f`` with ``L f = w``, ``w ~ N(0, I)`` (gamma = 1), by an exact spectral solve."""
    from scipy import fft as sfft

    w = rng.standard_normal((ny, nx))
    lam = neumann_eigenvalues(nx, ny, kappa)
    return sfft.idctn(sfft.dctn(w, type=2, norm="ortho") / lam, type=2, norm="ortho")


def uniform_points(nx: int, ny: int, count: int, rng: np.random.Generator):
    x = rng.uniform(0.0, nx - 1.0, count)
    y = rng.uniform(0.0, ny - 1.0, count)
    return x, y


def track_points(nx: int, ny: int, n_tracks: int, per_track: int, rng: np.random.Generator,
                 spacing: float = 1.5):
    """Samples along ``n_tracks`` wrapped straight tracks, ``per_track`` samples each."""
    xs, ys = [], []
    wx, wy = nx - 1.0, ny - 1.0
    for _ in range(n_tracks):
        theta = rng.uniform(0.0, math.pi)
        x0 = rng.uniform(0.0, wx)
        y0 = rng.uniform(0.0, wy)
        t = spacing * np.arange(per_track)
        xs.append(np.mod(x0 + t * math.cos(theta), wx))
        ys.append(np.mod(y0 + t * math.sin(theta), wy))
    if not xs:
        return np.zeros(0), np.zeros(0)
    x = np.concatenate(xs)
    y = np.concatenate(ys)
    # wrapping maps onto [0, w); keep everything inside the closed domain
    return np.clip(x, 0.0, wx), np.clip(y, 0.0, wy)


def _read_bilinear(truth: np.ndarray, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    from scipy import ndimage

    if x.size == 0:
        return np.zeros(0)
    return ndimage.map_coordinates(truth, np.vstack([y, x]), order=1, mode="nearest")


def make_problem(nx: int, ny: int, kappa: float, seed: int, *, n_uniform: int = 0,
                 n_tracks: int = 0, per_track: int = 0, sigma=0.1,
                 with_truth: bool = True) -> Problem:
    """Build one seeded problem.  ``sigma`` is a scalar or a ``(lo, hi)`` uniform range."""
    rng = np.random.default_rng(seed)
    truth = sample_truth(nx, ny, kappa, rng)
    ux, uy = uniform_points(nx, ny, n_uniform, rng)
    tx, ty = track_points(nx, ny, n_tracks, per_track, rng)
    ox = np.concatenate([tx, ux]).astype(np.float64)
    oy = np.concatenate([ty, uy]).astype(np.float64)
    m = ox.shape[0]
    if isinstance(sigma, tuple):
        sig = rng.uniform(sigma[0], sigma[1], m)
    else:
        sig = np.full(m, float(sigma))
    eps = rng.standard_normal(m)
    y = _read_bilinear(truth, ox, oy) + sig * eps
    return Problem(nx, ny, float(kappa), ox, oy, y.astype(np.float64), (sig * sig).astype(np.float64),
                   truth if with_truth else None,
                   dict(seed=seed, n_uniform=n_uniform, n_tracks=n_tracks, per_track=per_track,
                        sigma=sigma))


# --- the workloads -----------------------------------------------------------------------

def config_small(seed: int = 0) -> Problem:
    """64 x 64, kappa 0.3, 500 uniform observations, sigma 0.1 (FP64 messages, damping 0.5,
    200 iterations)."""
    return make_problem(64, 64, 0.3, seed, n_uniform=500, sigma=0.1)


def config_tracks_1024(seed: int = 0) -> Problem:
    """1024 x 1024, kappa 0.05, 24 tracks of ~40k samples in total, sigma 0.05 (FP32 messages,
    damping 0.3, iterate to relative residual 1e-5)."""
    per = int(round(40_000 / 24))
    return make_problem(1024, 1024, 0.05, seed, n_tracks=24, per_track=per, sigma=0.05)


def config_roofline_4096(seed: int = 0) -> Problem:
    """4096 x 4096, kappa 0.02, 96 tracks (~1.2M samples) plus 200k uniform points,
    sigma ~ U[0.02, 0.1] per observation (FP32 messages, compensated belief sums)."""
    per = int(round(1_200_000 / 96))
    return make_problem(4096, 4096, 0.02, seed, n_uniform=200_000, n_tracks=96, per_track=per,
                        sigma=(0.02, 0.1))


def scaled_config(side: int, kappa: float, seed: int, n_tracks: int, *, n_uniform: int = 0,
                  per_track: int | None = None, sigma=0.05) -> Problem:
    """A square problem with ``n_tracks`` tracks of length 2.5 * side (1.5-cell spacing)."""
    if per_track is None:
        per_track = int(round(2.5 * side / 1.5))
    return make_problem(side, side, kappa, seed, n_uniform=n_uniform, n_tracks=n_tracks,
                        per_track=per_track, sigma=sigma)


def paper_synthetic(side: int, frac: float, seed: int, *, sigma_y: float = 0.01, length: float = 0.15,
                    sigma: float = 1.1) -> Problem:
    """The synthetic setting of the grid-size / observation-density comparison (Sec. 4.1 with
    the hyperparameters of App. E): Matern prior with alpha = 2, nu = 1, lengthscale
    ``length`` and marginal standard deviation ``sigma`` on the unit square, discretised on
    side x side nodes of spacing h = 1 / side; a fraction ``frac`` of the grid points observed
    (uniformly, without replacement) with noise standard deviation ``sigma_y``.

    kappa = sqrt(2 nu) / length and gamma = h^2 / (sigma^2 q) with q = 4 pi kappa^2 (d = 2,
    nu = 1).  The library's grids have unit spacing; since L_h = h^-2 L_1(kappa h), the same
    prior is kappa' = kappa h and gamma' = gamma / h^4 at unit spacing, which is what the
    returned problem carries."""
    h = 1.0 / side
    kappa = math.sqrt(2.0) / length
    q = 4.0 * math.pi * kappa * kappa
    gamma_u = (h * h / (sigma * sigma * q)) / h ** 4
    kappa_u = kappa * h
    rng = np.random.default_rng(70_000 + 1000 * side + seed)
    truth = sample_truth(side, side, kappa_u, rng) / math.sqrt(gamma_u)
    m = int(round(frac * side * side))
    idx = np.sort(rng.choice(side * side, m, replace=False))
    ox = (idx % side).astype(np.float64)
    oy = (idx // side).astype(np.float64)
    y = truth.reshape(-1)[idx] + sigma_y * rng.standard_normal(m)
    return Problem(side, side, float(kappa_u), ox, oy, y, np.full(m, sigma_y * sigma_y), truth,
                   dict(seed=seed, frac=frac, sigma_y=sigma_y, length=length, sigma=sigma), gamma=float(gamma_u))


def config_batch(seed: int = 0, count: int = 64, lo: int = 128, hi: int = 1024) -> list[Problem]:
    """``count`` independent instances: side log-uniform in [lo, hi], kappa ~ U[0.02, 0.2],
    4-32 tracks each (track length 2.5 * side), sigma 0.05."""
    rng = np.random.default_rng(10_000 + seed)
    out = []
    for i in range(count):
        side = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        kappa = float(rng.uniform(0.02, 0.2))
        tracks = int(rng.integers(4, 33))
        out.append(scaled_config(side, kappa, seed * 1000 + i, tracks))
    return out


def config_warm_train(index: int, side: int = 512) -> Problem:
    """Training instance ``index``: side 512, kappa ~ U[0.02, 0.2], 8-32 tracks."""
    rng = np.random.default_rng(50_000 + index)
    kappa = float(rng.uniform(0.02, 0.2))
    tracks = int(rng.integers(8, 33))
    return scaled_config(side, kappa, 60_000 + index, tracks)


def config_warm_eval(seed: int = 0, side: int = 2048) -> Problem:
    """Evaluation instance: side 2048, kappa 0.03, 48 tracks."""
    return scaled_config(side, 0.03, 90_000 + seed, 48)
