"""Seeded synthetic workloads for separable W-projection gridding.

Every generator draws from ``numpy.random.Generator(PCG64(seed))`` with
``seed = SEED_BASE * 10 + k`` (k = workload number) in a fixed order:
antennas (if any) -> u, v, w -> visibility values -> weights.  Nothing here
computes a gridding kernel, a cell index or an image: the arrays are inputs
only, shared by the FP64 oracle and the CUDA path.

Coordinates follow Sec. 2 of the paper: u, v, w in wavelengths, w along the
phase centre.  The Earth-rotation tracks use the textbook ENU -> equatorial
-> (u, v, w) rotation (Thompson, Moran & Swenson, eq. 4.1) for a coplanar
array (Sec. 3 assumes w = d.u for a coplanar array).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 151107152
C_LIGHT = 299792458.0
OMEGA_EARTH = 7.2921159e-5  # rad/s, sidereal rate


@dataclasses.dataclass
class Workload:
    name: str
    grid_size: int
    fov: float          # image extent in direction cosine (radians, small angle)
    support: int
    oversample: int
    n_wplanes: int
    w_max: float
    u: np.ndarray       # float64 [nvis], wavelengths
    v: np.ndarray
    w: np.ndarray
    vis: np.ndarray     # complex64 [nvis]
    weight: np.ndarray  # float32 [nvis]
    gamma: float = 5.0 / 24.0
    kb_beta: float | None = None
    extra: dict = dataclasses.field(default_factory=dict)

    def __post_init__(self):
        if self.kb_beta is None:
            self.kb_beta = 2.34 * self.support

    @property
    def nvis(self) -> int:
        return int(self.u.shape[0])

    def params(self) -> dict:
        return dict(grid_size=self.grid_size, fov=self.fov, support=self.support,
                    oversample=self.oversample, n_wplanes=self.n_wplanes,
                    w_max=self.w_max, gamma=self.gamma, kb_beta=self.kb_beta)

    def subsample(self, n: int, seed: int = 0) -> "Workload":
        """A seeded subset of n visibilities (same geometry and parameters)."""
        rng = np.random.Generator(np.random.PCG64(SEED_BASE * 10 + 900 + seed))
        idx = np.sort(rng.choice(self.nvis, size=min(n, self.nvis), replace=False))
        return dataclasses.replace(
            self, name=f"{self.name}[sub{len(idx)}]", u=self.u[idx], v=self.v[idx],
            w=self.w[idx], vis=self.vis[idx], weight=self.weight[idx],
            extra=dict(self.extra, subsample_index=idx))


def _rng(k: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE * 10 + k))


def _values(rng: np.random.Generator, n: int):
    re = rng.standard_normal(n, dtype=np.float32)
    im = rng.standard_normal(n, dtype=np.float32)
    vis = np.empty(n, np.complex64)
    vis.real = re
    vis.imag = im
    weight = rng.uniform(0.5, 1.0, n).astype(np.float32)
    return vis, weight


def small_disk(nvis: int = 20_000) -> Workload:
    """Workload 1: 20,000 visibilities, (u, v) uniform in a disk of radius 120
    cells on a 256 x 256 grid with a 2 degree field of view, w uniform in
    [-2000, 2000]; support 8, oversampling 8, 32 w-planes."""
    rng = _rng(1)
    fov = math.radians(2.0)
    du = 1.0 / fov
    r = 120.0 * np.sqrt(rng.random(nvis))
    phi = 2.0 * np.pi * rng.random(nvis)
    u = r * np.cos(phi) * du
    v = r * np.sin(phi) * du
    w = rng.uniform(-2000.0, 2000.0, nvis)
    vis, weight = _values(rng, nvis)
    return Workload("small_disk_20k_N256_S8", 256, fov, 8, 8, 32, 2000.0,
                    u, v, w, vis, weight)


def _array_tracks(rng, nant, diameter_m, ndumps, dump_s, dec_deg, lat_deg, freqs_hz):
    """Earth-rotation (u, v, w) tracks of a coplanar array, order
    [dump][baseline][channel], in wavelengths."""
    r = 0.5 * diameter_m * np.sqrt(rng.random(nant))
    phi = 2.0 * np.pi * rng.random(nant)
    east = r * np.cos(phi)
    north = r * np.sin(phi)
    lat = math.radians(lat_deg)
    dec = math.radians(dec_deg)
    # ENU (up = 0) -> equatorial XYZ
    X = -math.sin(lat) * north
    Y = east
    Z = math.cos(lat) * north
    i, j = np.triu_indices(nant, k=1)
    dX, dY, dZ = X[j] - X[i], Y[j] - Y[i], Z[j] - Z[i]
    H = OMEGA_EARTH * dump_s * (np.arange(ndumps) - 0.5 * (ndumps - 1))
    sH, cH = np.sin(H)[:, None], np.cos(H)[:, None]
    um = sH * dX + cH * dY
    vm = -math.sin(dec) * cH * dX + math.sin(dec) * sH * dY + math.cos(dec) * dZ
    wm = math.cos(dec) * cH * dX - math.cos(dec) * sH * dY + math.sin(dec) * dZ
    inv_lam = np.asarray(freqs_hz, np.float64) / C_LIGHT
    shape = (ndumps, len(dX), len(inv_lam))
    u = (um[:, :, None] * inv_lam[None, None, :]).reshape(-1)
    v = (vm[:, :, None] * inv_lam[None, None, :]).reshape(-1)
    w = (wm[:, :, None] * inv_lam[None, None, :]).reshape(-1)
    return u, v, w, shape


def meerkat_like(ndumps: int = 1000, nchan: int = 16, k: int = 2) -> Workload:
    """Workload 2: 64 antennas uniform in an 8 km diameter disk, 2016
    baselines x 1000 dumps of 8 s at declination -30 deg (site latitude
    -30.7 deg) x 16 channels over 1.0-1.4 GHz = 32,256,000 visibilities;
    4096^2 grid, 1 degree field of view, support 16, oversampling 16,
    128 w-planes, w_max = max |w| of the data."""
    rng = _rng(k)
    freqs = np.linspace(1.0e9, 1.4e9, nchan)
    u, v, w, shape = _array_tracks(rng, 64, 8000.0, ndumps, 8.0, -30.0, -30.7, freqs)
    vis, weight = _values(rng, u.shape[0])
    w_max = float(np.max(np.abs(w)))
    return Workload(f"meerkat_like_{u.shape[0]}_N4096_S16", 4096, math.radians(1.0),
                    16, 16, 128, w_max, u, v, w, vis, weight,
                    extra=dict(shape=shape, freqs=freqs))


def point_source_model(N: int = 2048, nsrc: int = 500, k: int = 4):
    """Workload 4 model: N x N float32 image, 500 point sources with fluxes
    log-uniform in [1e-3, 1] at pixel centres uniform within 0.5 deg of the
    phase centre (fov = 1 deg), plus N(0, 1e-4^2) per pixel.  Returns
    (image [m][l], visibility workload of 2016 baselines x 1984 dumps at
    1.4 GHz, support 16, oversampling 16, 64 w-planes)."""
    rng = _rng(k)
    fov = math.radians(1.0)
    flux = np.exp(rng.uniform(math.log(1e-3), math.log(1.0), nsrc))
    rp = (N / 2) * np.sqrt(rng.random(nsrc))
    ph = 2.0 * np.pi * rng.random(nsrc)
    a = np.clip(N // 2 + np.round(rp * np.cos(ph)).astype(np.int64), 0, N - 1)
    b = np.clip(N // 2 + np.round(rp * np.sin(ph)).astype(np.int64), 0, N - 1)
    img = (1e-4 * rng.standard_normal((N, N))).astype(np.float32)
    np.add.at(img, (b, a), flux.astype(np.float32))
    u, v, w, shape = _array_tracks(rng, 64, 8000.0, 1984, 8.0, -30.0, -30.7, [1.4e9])
    vis, weight = _values(rng, u.shape[0])
    w_max = float(np.max(np.abs(w)))
    wl = Workload(f"predict_{u.shape[0]}_N{N}_S16", N, fov, 16, 16, 64, w_max,
                  u, v, w, vis, weight, extra=dict(shape=shape))
    return img, wl


def wstack_layers(nlayers: int = 16, nchan: int = 8, N: int = 2048,
                  total: int = 64_000_000, k: int = 5):
    """Workload 5: nlayers x nchan separate N x N grids with visibility counts
    log-uniform in [1e4, 2e6], rescaled towards `total` and clamped to that
    range; (u, v) uniform in a disk of radius 0.45 N cells; residual w uniform
    in [-1000, 1000]; support 12, oversampling 16, 32 w-planes.  Returns
    (list of per-grid counts, Workload with all visibilities concatenated
    grid by grid, offsets [ngrids + 1])."""
    rng = _rng(k)
    ng = nlayers * nchan
    counts = np.exp(rng.uniform(math.log(1e4), math.log(2e6), ng))
    counts = np.clip(np.round(counts * (total / counts.sum())), 1e4, 2e6).astype(np.int64)
    fov = math.radians(1.0)
    du = 1.0 / fov
    n = int(counts.sum())
    r = 0.45 * N * np.sqrt(rng.random(n))
    phi = 2.0 * np.pi * rng.random(n)
    u = r * np.cos(phi) * du
    v = r * np.sin(phi) * du
    w = rng.uniform(-1000.0, 1000.0, n)
    vis, weight = _values(rng, n)
    offsets = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    wl = Workload(f"wstack_{ng}x{N}_S12", N, fov, 12, 16, 32, 1000.0,
                  u, v, w, vis, weight, extra=dict(offsets=offsets, counts=counts))
    return wl


def random_case(seed: int, nvis: int, grid_size: int, support: int, oversample: int,
                n_wplanes: int, w_max: float = 500.0, fov: float = math.radians(2.0),
                radius_cells: float | None = None, edge_fraction: float = 0.0,
                gamma: float = 5.0 / 24.0) -> Workload:
    """A small seeded case for parity tests.  (u, v) uniform in a disk of
    `radius_cells` (default: just inside the droppable edge) and w uniform in
    [-1.05 w_max, 1.05 w_max], so a few visibilities fall off the grid or
    beyond w_max.  `edge_fraction` of the points are placed on exact
    oversample ties and on the first/last valid footprint positions."""
    rng = np.random.Generator(np.random.PCG64(SEED_BASE * 10 + 100 + seed))
    du = 1.0 / fov
    if radius_cells is None:
        radius_cells = grid_size / 2 - support / 2 + 1.5
    r = radius_cells * np.sqrt(rng.random(nvis))
    phi = 2.0 * np.pi * rng.random(nvis)
    xcell = r * np.cos(phi)
    ycell = r * np.sin(phi)
    nedge = int(edge_fraction * nvis)
    if nedge:
        # offsets in cells from the centre that sit on oversample ties
        # (half-way between two oversampled positions) and on the first and
        # last footprint positions that stay on the grid
        half = grid_size // 2
        lo = -half + support // 2 - 1
        hi = half - support // 2 - 1
        cand = np.array([lo, lo - 1, hi, hi + 1, 0], np.float64)
        pick = cand[rng.integers(0, len(cand), size=(2, nedge))]
        frac = (rng.integers(0, oversample, size=(2, nedge)) + 0.5) / oversample
        frac[:, : nedge // 2] = 0.0
        xcell[:nedge] = pick[0] + frac[0]
        ycell[:nedge] = pick[1] + frac[1]
    u = xcell * du
    v = ycell * du
    w = rng.uniform(-1.05 * w_max, 1.05 * w_max, nvis)
    vis, weight = _values(rng, nvis)
    return Workload(f"random{seed}_{nvis}_N{grid_size}_S{support}", grid_size, fov,
                    support, oversample, n_wplanes, w_max, u, v, w, vis, weight,
                    gamma=gamma)


WORKLOADS = {
    "small_disk": small_disk,
    "meerkat_like": meerkat_like,
    "point_source_model": point_source_model,
    "wstack_layers": wstack_layers,
}
