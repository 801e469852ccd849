"""Pair geometry (Section 2.1, text after Eq. 2.4).

The paper bins each pixel pair by its separation (r_perp, r_par) "in comoving
coordinates" without defining the split.  Reading used here (the standard one
of the Lyman-alpha literature the paper follows): with theta the angle between
the two lines of sight,

    r_par  = |d_i - d_j| cos(theta/2)
    r_perp = (d_i + d_j) sin(theta/2)

so that r_par^2 + r_perp^2 = d_i^2 + d_j^2 - 2 d_i d_j cos(theta), the squared
3-D distance.  r_par is taken as an absolute value (auto-correlation).

cos(theta/2) and sin(theta/2) come from the chord lengths |n_a +- n_b| / 2,
which stay accurate at the small angles involved (no arccos of a dot product).
"""
from __future__ import annotations

import numpy as np


def unit_vectors(ra: np.ndarray, dec: np.ndarray) -> np.ndarray:
    """Line-of-sight unit vectors (cos dec cos ra, cos dec sin ra, sin dec)."""
    ra = np.asarray(ra, dtype=np.float64)
    dec = np.asarray(dec, dtype=np.float64)
    cd = np.cos(dec)
    return np.stack([cd * np.cos(ra), cd * np.sin(ra), np.sin(dec)], axis=-1)


def half_angle(n_a: np.ndarray, n_b: np.ndarray):
    """(cos(theta/2), sin(theta/2)) of the angle between unit vectors n_a, n_b."""
    c = 0.5 * np.linalg.norm(np.asarray(n_a) + np.asarray(n_b), axis=-1)
    s = 0.5 * np.linalg.norm(np.asarray(n_a) - np.asarray(n_b), axis=-1)
    return c, s


def separations(d_a: np.ndarray, d_b: np.ndarray, c: float, s: float):
    """(r_par, r_perp) for every pixel pair (i in a, j in b), shape (n_a, n_b)."""
    d_a = np.asarray(d_a, dtype=np.float64)[:, None]
    d_b = np.asarray(d_b, dtype=np.float64)[None, :]
    r_par = np.abs(d_a - d_b) * c
    r_perp = (d_a + d_b) * s
    return r_par, r_perp
