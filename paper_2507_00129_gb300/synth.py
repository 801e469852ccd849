"""Seeded synthetic Lyman-alpha forest catalogues.

This module only draws inputs: sky positions, quasar redshifts, pixel grids,
comoving distances, deltas and weights.  It contains none of the estimator's
arithmetic (no separations, binning, projection or pair sums), so the CUDA
library and the CPU oracle can both consume its output without sharing any
method code.

The paper measures on SDSS DR16 deltas and on a DESI Y5 mock (Section 3.2,
Table 1); neither is available here.  The catalogues below stand in for them
with the shapes the paper quotes: about 200 pixels per eBOSS forest and about
700 per DESI forest (Section 2.1), sky areas of Table 1 scaled down, the
rest-frame Lyman-alpha window 1040-1200 A and observed wavelengths above
3600 A.

Recipe (one ``numpy.random.default_rng(seed)`` stream, in this order):

1. ``ra ~ U[ra0, ra1)``, ``sin(dec) ~ U[sin(dec0), sin(dec1)]`` (uniform in area)
2. ``z_q ~ U[2.1, 3.5]``
3. grid ``"log10"``: lambda_k = 10**(log10(3600) + 3e-4 k), k >= 1;
   grid ``"linear"``: lambda_k = 3600 + 0.8 k, k >= 1.  A forest keeps the
   grid pixels with 1040 (1+z_q) <= lambda_k <= 1200 (1+z_q).
   If ``length_range`` is set, ``L_q ~ U{lo..hi}`` and ``u ~ U[0,1)`` are drawn
   per forest and the forest keeps a contiguous window of ``min(L_q, n_nat)``
   pixels starting at ``floor(u * (n_nat - L + 1))``.
4. per pixel ``sigma ~ lognormal(ln 0.15, 0.3)``, ``w = 1/sigma^2``
5. per pixel ``delta ~ N(0, delta_sigma^2)``
6. if ``tilt``: per forest ``a ~ N(0, 0.1^2)``, ``b ~ N(0, 1)`` and
   ``delta += a + b (Lambda - ln(1120 (1+z_q)))`` with Lambda = ln lambda.

Comoving distances use flat LCDM with ``omega_m`` (0.315 by default), no
radiation, c/H0 = 2997.92458 Mpc/h, evaluated once on the wavelength grid by
Gauss-Legendre quadrature (relative error below 1e-13).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional, Sequence

import numpy as np

LYA_REST_A = 1215.67
C_OVER_H0 = 2997.92458  # Mpc/h
LAMBDA_MIN_OBS = 3600.0
RF_MIN, RF_MAX = 1040.0, 1200.0


@dataclasses.dataclass
class Bins:
    """(r_par, r_perp) grid: n_par x n_perp rectangles of width r_max / n."""

    n_par: int
    n_perp: int
    r_par_max: float
    r_perp_max: float

    @property
    def nbins(self) -> int:
        return self.n_par * self.n_perp


@dataclasses.dataclass
class Catalog:
    """Flat pixel arrays plus per-forest offsets (forest f owns
    ``offsets[f]:offsets[f+1]``); distances strictly increase inside a forest."""

    ra: np.ndarray        # [n_forests] float64, radians
    dec: np.ndarray       # [n_forests] float64, radians
    offsets: np.ndarray   # [n_forests + 1] int64
    dist: np.ndarray      # [n_pix] float64, comoving distance, Mpc/h
    loglam: np.ndarray    # [n_pix] float64, natural log of observed wavelength
    delta: np.ndarray     # [n_pix] float32
    weight: np.ndarray    # [n_pix] float32
    name: str = ""
    zq: Optional[np.ndarray] = None   # [n_forests] float64, redshift of each forest's quasar

    @property
    def n_forests(self) -> int:
        return int(self.ra.shape[0])

    @property
    def n_pix(self) -> int:
        return int(self.dist.shape[0])

    def forest(self, f: int) -> slice:
        return slice(int(self.offsets[f]), int(self.offsets[f + 1]))

    def lengths(self) -> np.ndarray:
        return np.diff(self.offsets)


@dataclasses.dataclass
class Spec:
    n_forests: int
    seed: int
    region: str = "cap"               # "cap" (around the north pole) or "box"
    area_deg2: float = 600.0          # for "cap"
    box_deg: float = 3.0              # for "box": RA in [0, box), Dec in [-box/2, box/2]
    grid: str = "log10"               # "log10" (SDSS-like) or "linear" (DESI-like)
    delta_sigma: float = 0.2
    length_range: Optional[Sequence[int]] = None
    tilt: bool = False
    omega_m: float = 0.315


# ----------------------------------------------------------------------------
# cosmology (input generation only)
# ----------------------------------------------------------------------------
_GL_X, _GL_W = np.polynomial.legendre.leggauss(24)


def _inv_e(z: np.ndarray, omega_m: float) -> np.ndarray:
    return 1.0 / np.sqrt(omega_m * (1.0 + z) ** 3 + (1.0 - omega_m))


def comoving_distance(z, omega_m: float = 0.315) -> np.ndarray:
    """Line-of-sight comoving distance in Mpc/h for flat LCDM (no radiation).

    Integrates c/H0 * 1/E(z) with 24-point Gauss-Legendre on sub-intervals of
    width <= 0.02, which is exact to below 1e-14 relative for 0 <= z <= 10.
    """
    z = np.atleast_1d(np.asarray(z, dtype=np.float64))
    order = np.argsort(z)
    zs = z[order]
    out = np.empty_like(zs)
    acc = 0.0
    prev = 0.0
    for k, zk in enumerate(zs):
        if zk > prev:
            n_sub = max(1, int(math.ceil((zk - prev) / 0.02)))
            edges = np.linspace(prev, zk, n_sub + 1)
            lo, hi = edges[:-1, None], edges[1:, None]
            mid, half = 0.5 * (lo + hi), 0.5 * (hi - lo)
            vals = _inv_e(mid + half * _GL_X[None, :], omega_m)
            acc += float(np.sum(half[:, 0] * (vals @ _GL_W)))
            prev = zk
        out[k] = acc
    res = np.empty_like(out)
    res[order] = out * C_OVER_H0
    return res


# ----------------------------------------------------------------------------
# catalogue generation
# ----------------------------------------------------------------------------
def _grid_lambda(grid: str, lam_max: float) -> np.ndarray:
    if grid == "log10":
        step = 3e-4
        kmax = int(math.floor((math.log10(lam_max) - math.log10(LAMBDA_MIN_OBS)) / step)) + 2
        k = np.arange(1, kmax + 1, dtype=np.float64)
        return 10.0 ** (math.log10(LAMBDA_MIN_OBS) + step * k)
    if grid == "linear":
        step = 0.8
        kmax = int(math.floor((lam_max - LAMBDA_MIN_OBS) / step)) + 2
        k = np.arange(1, kmax + 1, dtype=np.float64)
        return LAMBDA_MIN_OBS + step * k
    raise ValueError(f"unknown grid {grid!r}")


def cap_half_angle_deg(area_deg2: float) -> float:
    """Half-opening angle of a spherical cap of the given area."""
    area_sr = area_deg2 * (math.pi / 180.0) ** 2
    return math.degrees(math.acos(1.0 - area_sr / (2.0 * math.pi)))


def generate(spec: Spec, name: str = "") -> Catalog:
    rng = np.random.default_rng(spec.seed)
    n = spec.n_forests
    # 1. positions, uniform in area
    if spec.region == "box":
        b = math.radians(spec.box_deg)
        ra = rng.uniform(0.0, b, n)
        sd = rng.uniform(math.sin(-0.5 * b), math.sin(0.5 * b), n)
    elif spec.region == "cap":
        th = math.radians(cap_half_angle_deg(spec.area_deg2))
        ra = rng.uniform(0.0, 2.0 * math.pi, n)
        sd = rng.uniform(math.cos(th), 1.0, n)
    else:
        raise ValueError(spec.region)
    dec = np.arcsin(sd)
    # 2. quasar redshifts
    zq = rng.uniform(2.1, 3.5, n)
    # 3. pixel windows on the wavelength grid
    lam_grid = _grid_lambda(spec.grid, RF_MAX * (1.0 + 3.5))
    d_grid = comoving_distance(lam_grid / LYA_REST_A - 1.0, spec.omega_m)
    lo = np.searchsorted(lam_grid, RF_MIN * (1.0 + zq), side="left")
    hi = np.searchsorted(lam_grid, RF_MAX * (1.0 + zq), side="right")
    n_nat = hi - lo
    if spec.length_range is not None:
        lmin, lmax = int(spec.length_range[0]), int(spec.length_range[1])
        lq = rng.integers(lmin, lmax + 1, n)
        u = rng.random(n)
        length = np.minimum(lq, n_nat)
        start = lo + np.floor(u * (n_nat - length + 1)).astype(np.int64)
    else:
        length = n_nat
        start = lo
    length = length.astype(np.int64)
    offsets = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(length, out=offsets[1:])
    n_pix = int(offsets[-1])
    forest_of_pix = np.repeat(np.arange(n, dtype=np.int64), length)
    kidx = start[forest_of_pix] + (np.arange(n_pix, dtype=np.int64) - offsets[forest_of_pix])
    lam = lam_grid[kidx]
    dist = d_grid[kidx]
    loglam = np.log(lam)
    # 4-5. per-pixel noise and deltas
    sigma = np.exp(rng.normal(math.log(0.15), 0.3, n_pix))
    weight = (1.0 / sigma ** 2).astype(np.float32)
    delta = rng.normal(0.0, spec.delta_sigma, n_pix)
    # 6. per-forest continuum tilt
    if spec.tilt:
        a = rng.normal(0.0, 0.1, n)
        bslope = rng.normal(0.0, 1.0, n)
        lam_c = np.log(0.5 * (RF_MIN + RF_MAX) * (1.0 + zq))
        delta = delta + a[forest_of_pix] + bslope[forest_of_pix] * (loglam - lam_c[forest_of_pix])
    return Catalog(ra=ra, dec=dec, offsets=offsets, dist=dist, loglam=loglam,
                   delta=delta.astype(np.float32), weight=weight, name=name, zq=zq)


@dataclasses.dataclass
class Quasars:
    """Point tracers for the forest x quasar cross-correlation."""

    ra: np.ndarray        # [n] float64, radians
    dec: np.ndarray       # [n] float64, radians
    dist: np.ndarray      # [n] float64, comoving distance, Mpc/h
    weight: np.ndarray    # [n] float32
    z: np.ndarray         # [n] float64

    @property
    def n(self) -> int:
        return int(self.ra.shape[0])


def quasars(spec: Spec, cat: Catalog, extra_fraction: float = 0.5, z_extra=(1.8, 3.5)):
    """Quasar catalogue of a forest catalogue drawn from ``spec``.

    Quasar a (a < n_forests) is the source of forest a: its line of sight and
    redshift z_q.  ``round(extra_fraction * n_forests)`` further quasars
    without a forest follow, drawn from ``default_rng([spec.seed, 7])`` in this
    order: positions uniform in area over the same region, then
    z ~ U[z_extra].  Weights w_q = ((1 + z) / 3.25)^0.44, the redshift
    evolution of the quasar weights of the eBOSS DR16 analysis
    (du Mas des Bourboux et al. 2020).  Returns (quasars, forest_qso) with
    forest_qso[a] = a, the index of each forest's own quasar."""
    if cat.zq is None:
        raise ValueError("catalogue has no quasar redshifts")
    n = cat.n_forests
    n_extra = int(round(extra_fraction * n))
    rng = np.random.default_rng([spec.seed, 7])
    if spec.region == "box":
        b = math.radians(spec.box_deg)
        ra_x = rng.uniform(0.0, b, n_extra)
        sd_x = rng.uniform(math.sin(-0.5 * b), math.sin(0.5 * b), n_extra)
    else:
        th = math.radians(cap_half_angle_deg(spec.area_deg2))
        ra_x = rng.uniform(0.0, 2.0 * math.pi, n_extra)
        sd_x = rng.uniform(math.cos(th), 1.0, n_extra)
    z_x = rng.uniform(z_extra[0], z_extra[1], n_extra)
    z = np.concatenate([np.asarray(cat.zq, dtype=np.float64), z_x])
    q = Quasars(ra=np.concatenate([cat.ra, ra_x]), dec=np.concatenate([cat.dec, np.arcsin(sd_x)]),
                dist=comoving_distance(z, spec.omega_m),
                weight=(((1.0 + z) / 3.25) ** 0.44).astype(np.float32), z=z)
    return q, np.arange(n, dtype=np.int64)


# ----------------------------------------------------------------------------
# the five workloads
# ----------------------------------------------------------------------------
def spec_for(config: int, seed: Optional[int] = None, n_forests: Optional[int] = None) -> Spec:
    """Generator settings of the five workloads.

    0: 200 forests, 3 x 3 deg box, log10 grid, delta sigma 0.2 (tiny, plain FP64)
    1: 60,000 forests, 2,500 deg^2 cap, log10 grid (SDSS-DR16-like)
    2: 600,000 forests, 10,000 deg^2, linear 0.8 A grid, 100-600 px, tilt (DESI-Y5-like)
    3: 20,000 forests, 800 deg^2, linear grid, 100-600 px (differentiable xi)
    4: one mock of 15,000 forests, 600 deg^2, linear grid, 100-600 px (seed = mock id)
    """
    if config == 0:
        s = Spec(n_forests=200, seed=0, region="box", box_deg=3.0, grid="log10", delta_sigma=0.2)
    elif config == 1:
        s = Spec(n_forests=60_000, seed=1, area_deg2=2500.0, grid="log10", delta_sigma=0.2)
    elif config == 2:
        s = Spec(n_forests=600_000, seed=2, area_deg2=10_000.0, grid="linear", delta_sigma=0.25,
                 length_range=(100, 600), tilt=True)
    elif config == 3:
        s = Spec(n_forests=20_000, seed=3, area_deg2=800.0, grid="linear", delta_sigma=0.25,
                 length_range=(100, 600))
    elif config == 4:
        s = Spec(n_forests=15_000, seed=0, area_deg2=600.0, grid="linear", delta_sigma=0.25,
                 length_range=(100, 600))
    else:
        raise ValueError(config)
    if seed is not None:
        s.seed = seed
    if n_forests is not None:
        s.n_forests = n_forests
    return s


def bins_for(config: int) -> Bins:
    """Bin grids: 25 x 25 of 4 Mpc/h for workload 0, 50 x 50 of 4 Mpc/h otherwise."""
    if config == 0:
        return Bins(25, 25, 100.0, 100.0)
    return Bins(50, 50, 200.0, 200.0)


def dm_fraction_for(config: int) -> float:
    """Forest-pair subsample fraction used for the distortion matrix."""
    return {0: 1.0, 1: 0.05, 4: 0.02}.get(config, 0.05)


def make(config: int, seed: Optional[int] = None, n_forests: Optional[int] = None) -> Catalog:
    return generate(spec_for(config, seed, n_forests), name=f"workload{config}")


def concat(cats: Sequence[Catalog]) -> Catalog:
    """Stack independent catalogues (mocks) into one flat catalogue."""
    offs = [np.zeros(1, dtype=np.int64)]
    base = 0
    for c in cats:
        offs.append(c.offsets[1:] + base)
        base += c.n_pix
    return Catalog(
        ra=np.concatenate([c.ra for c in cats]), dec=np.concatenate([c.dec for c in cats]),
        offsets=np.concatenate(offs), dist=np.concatenate([c.dist for c in cats]),
        loglam=np.concatenate([c.loglam for c in cats]),
        delta=np.concatenate([c.delta for c in cats]), weight=np.concatenate([c.weight for c in cats]),
        name="+".join(c.name for c in cats),
        zq=np.concatenate([c.zq for c in cats]) if all(c.zq is not None for c in cats) else None)


def subset(cat: Catalog, forests: np.ndarray) -> Catalog:
    """Catalogue restricted to the given forests (in the given order)."""
    forests = np.asarray(forests, dtype=np.int64)
    lens = cat.lengths()[forests]
    offs = np.zeros(len(forests) + 1, dtype=np.int64)
    np.cumsum(lens, out=offs[1:])
    idx = np.concatenate([np.arange(cat.offsets[f], cat.offsets[f + 1]) for f in forests]) \
        if len(forests) else np.zeros(0, dtype=np.int64)
    return Catalog(ra=cat.ra[forests], dec=cat.dec[forests], offsets=offs, dist=cat.dist[idx],
                   loglam=cat.loglam[idx], delta=cat.delta[idx], weight=cat.weight[idx],
                   name=cat.name + "[subset]", zq=None if cat.zq is None else cat.zq[forests])
