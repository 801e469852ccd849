"""Covariance of xi from HEALPix sub-samples.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper obtains the uncertainty of its correlations by sub-sampling the
forests' data in HEALPix pixels (Sections 3.2 and 3.4), and builds the
covariance from the two-point sums in post-processing (Appendix A).  It gives
no formula.  Readings:

* a forest pair (a < b) belongs to the sub-sample of its first forest a: the
  HEALPix pixel, at resolution nside in the nested numbering, that contains
  a's line of sight;
* per sub-sample s, N^s_A and W^s_A are the sums of Eq. (2.4) over its pairs,
  so that sum_s N^s = N and sum_s W^s = W;
* the covariance is the weighted sub-sample covariance
      C_AB = sum_s W^s_A W^s_B (xi^s_A - xi_A)(xi^s_B - xi_B) / (W_A W_B),
  xi^s = N^s / W^s, xi = N / W (the full-sample values); with
  a^s_A = W^s_A (xi^s_A - xi_A) = N^s_A - W^s_A xi_A this is
  C = a^T a / (W W^T); rows and columns with W_A = 0 are zero.

HEALPix pixel numbering (nested scheme) follows the definition of the grid in
Gorski et al. 2005 (ApJ 622, 759): twelve base pixels, four around each pole
and four on the equator, each split into nside x nside pixels whose (x, y)
indices are interleaved bit by bit.
"""
from __future__ import annotations

import math

import numpy as np

from . import pairs as _pairs
from . import xi as _xi


def _interleave(ix: np.ndarray, iy: np.ndarray) -> np.ndarray:
    """Morton number with the bits of ix on even and of iy on odd positions."""
    out = np.zeros_like(ix, dtype=np.int64)
    for bit in range(32):
        out |= ((ix >> bit) & 1) << (2 * bit)
        out |= ((iy >> bit) & 1) << (2 * bit + 1)
    return out


def ang2pix_nest(nside: int, z: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """Nested HEALPix pixel of points with cos(colatitude) z and longitude phi.

    Equatorial zone |z| <= 2/3: the pixel boundaries are the lines
    nside (1/2 + t) -+ 3 nside z / 4 = const (t = 2 phi / pi); polar caps: the
    boundaries are nside t' sqrt(3 (1 - |z|)) = const and
    nside (1 - t') sqrt(3 (1 - |z|)) = const within each quarter (t' the
    fractional part of t)."""
    if nside < 1 or nside & (nside - 1):
        raise ValueError("nside must be a power of two")
    z = np.asarray(z, dtype=np.float64)
    phi = np.mod(np.asarray(phi, dtype=np.float64), 2.0 * math.pi)
    t = phi * (2.0 / math.pi)
    za = np.abs(z)
    n = nside
    face = np.zeros(z.shape, dtype=np.int64)
    ix = np.zeros(z.shape, dtype=np.int64)
    iy = np.zeros(z.shape, dtype=np.int64)
    eq = za <= 2.0 / 3.0
    # equatorial zone
    if np.any(eq):
        a = n * (0.5 + t[eq])
        b = n * 0.75 * z[eq]
        up = np.floor(a - b).astype(np.int64)     # index of the ascending edge line
        dn = np.floor(a + b).astype(np.int64)     # index of the descending edge line
        fu, fd = up // n, dn // n
        f = np.where(fu == fd, fu % 4 + 4, np.where(fu < fd, fu % 4, fd % 4 + 8))
        face[eq] = f
        ix[eq] = dn % n
        iy[eq] = n - 1 - (up % n)
    pol = ~eq
    if np.any(pol):
        q = np.minimum(np.floor(t[pol]).astype(np.int64), 3)
        tf = t[pol] - q
        r = n * np.sqrt(3.0 * (1.0 - za[pol]))
        u = np.minimum(np.floor(tf * r).astype(np.int64), n - 1)
        v = np.minimum(np.floor((1.0 - tf) * r).astype(np.int64), n - 1)
        north = z[pol] > 0
        face[pol] = np.where(north, q, q + 8)
        ix[pol] = np.where(north, n - 1 - v, u)
        iy[pol] = np.where(north, n - 1 - u, v)
    return face * n * n + _interleave(ix, iy)


def subsample_ids(cat, nside: int) -> np.ndarray:
    """Sub-sample (nested pixel at nside) of every forest's line of sight."""
    return ang2pix_nest(nside, np.sin(cat.dec), cat.ra)


def subsample_sums(cat, bins, nside: int, pair_list=None, eps_edge: float = 0.0):
    """Per sub-sample sums of Eq. (2.4): dict of arrays [12 nside^2, nb]
    (num, wsum, edge_w, edge_n) over the pairs of each sub-sample."""
    if pair_list is None:
        pair_list = _pairs.forest_pairs(cat, bins)
    a, b = (np.asarray(x, dtype=np.int64) for x in pair_list)
    first = np.minimum(a, b)
    sid = subsample_ids(cat, nside)[first] if len(first) else np.zeros(0, np.int64)
    ns = 12 * nside * nside
    out = {k: np.zeros((ns, bins.nbins)) for k in ("num", "wsum", "edge_w", "edge_n")}
    for s in np.unique(sid):
        m = sid == s
        r = _xi.xi_sums(cat, bins, (a[m], b[m]), eps_edge=eps_edge)
        for k in out:
            out[k][s] = r[k]
    return out


def covariance(num_s: np.ndarray, wsum_s: np.ndarray) -> np.ndarray:
    """Weighted sub-sample covariance from per sub-sample sums [n_sub, nb]."""
    num_s = np.asarray(num_s, dtype=np.float64)
    wsum_s = np.asarray(wsum_s, dtype=np.float64)
    W = wsum_s.sum(axis=0)
    N = num_s.sum(axis=0)
    xi = np.divide(N, W, out=np.zeros_like(W), where=W != 0)
    a = num_s - wsum_s * xi[None, :]
    C = a.T @ a
    den = np.outer(W, W)
    return np.divide(C, den, out=np.zeros_like(C), where=den != 0)
