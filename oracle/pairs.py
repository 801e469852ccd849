"""Forest-pair set (Section 2.1: only pairs of different forests, restricted to
a neighbourhood defined by the maximum separation).

Readings:

* every unordered pair of distinct forests is counted once (a < b); counting
  both orders would double W and leave xi unchanged;
* a pair can hold an in-grid pixel pair only if
  (d_min,a + d_min,b) sin(theta/2) < r_perp_max, since r_perp >= (d_i + d_j) sin(theta/2)
  and d_i >= d_min of its forest.  ``forest_pairs`` returns exactly the pairs
  passing that test.  The test drops no in-grid pixel pair, so the xi, W and D
  sums over it equal the sums over all forest pairs (checked in the tests);
* forests with no pixels never pair.

The search is brute force for small catalogues and a k-d tree on the unit
vectors (chord radius of the catalogue-wide angle bound) otherwise -- a
method independent of the HEALPix cells the CUDA library uses.
"""
from __future__ import annotations

import math

import numpy as np

from .geometry import unit_vectors, half_angle


def forest_dmin(cat) -> np.ndarray:
    """Smallest pixel distance of each forest (+inf for empty forests)."""
    n = cat.n_forests
    out = np.full(n, np.inf)
    lens = np.diff(cat.offsets)
    nz = lens > 0
    out[nz] = cat.dist[cat.offsets[:-1][nz]]  # distances increase within a forest
    return out


def theta_max(cat, bins) -> float:
    """Catalogue-wide angle bound 2 asin(r_perp_max / (2 d_min))."""
    dmin = float(np.min(cat.dist)) if cat.n_pix else 1.0
    return 2.0 * math.asin(min(1.0, bins.r_perp_max / (2.0 * dmin)))


def _exact_keep(na, nb, dmin_a, dmin_b, r_perp_max):
    _, s = half_angle(na, nb)
    return (dmin_a + dmin_b) * s < r_perp_max


def all_pairs(n: int):
    """Every unordered pair a < b of n forests (no cut)."""
    a, b = np.triu_indices(n, k=1)
    return a.astype(np.int64), b.astype(np.int64)


def forest_pairs(cat, bins, method: str = "auto"):
    """Pairs (a, b), a < b, sorted by (a, b), that can hold an in-grid pixel pair."""
    n = cat.n_forests
    nvec = unit_vectors(cat.ra, cat.dec)
    dmin = forest_dmin(cat)
    if method == "auto":
        method = "brute" if n <= 2000 else "kdtree"
    if method == "brute":
        a, b = all_pairs(n)
    elif method == "kdtree":
        from scipy.spatial import cKDTree
        th = theta_max(cat, bins)
        chord = 2.0 * math.sin(0.5 * th) * (1.0 + 1e-9)
        tree = cKDTree(nvec)
        pr = tree.query_pairs(chord, output_type="ndarray")
        if len(pr) == 0:
            return np.zeros(0, np.int64), np.zeros(0, np.int64)
        a = np.minimum(pr[:, 0], pr[:, 1]).astype(np.int64)
        b = np.maximum(pr[:, 0], pr[:, 1]).astype(np.int64)
    else:
        raise ValueError(method)
    ok = np.isfinite(dmin[a]) & np.isfinite(dmin[b])
    a, b = a[ok], b[ok]
    keep = _exact_keep(nvec[a], nvec[b], dmin[a], dmin[b], bins.r_perp_max)
    a, b = a[keep], b[keep]
    order = np.lexsort((b, a))
    return a[order], b[order]
