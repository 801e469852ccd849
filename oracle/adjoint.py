"""Gradient of L = sum_A c_A xi_A with respect to delta and w.

Not in the paper; it is the chain rule applied to Eq. (2.4).  With
N_A = sum_A (w d)_i (w d)_j, W_A = sum_A w_i w_j, xi_A = N_A / W_A,
gamma_A = c_A / W_A and rho_A = gamma_A xi_A (both 0 where W_A = 0):

    dL/d delta_i = w_i      sum_{j paired with i in grid} gamma_A (w d)_j
    dL/d w_i     = delta_i  sum_j gamma_A (w d)_j  -  sum_j rho_A w_j

where A is the bin of the pair (i, j) and j runs over pixels of the other
forest of every forest pair containing i.
"""
from __future__ import annotations

import numpy as np

from .geometry import unit_vectors, half_angle
from .xi import pixel_pair_bins, xi_sums
from . import pairs as _pairs


def xi_grad(cat, bins, grad_xi, pair_list=None, delta=None):
    """(dL/d delta, dL/d w, forward sums) for L = sum_A grad_xi[A] xi_A."""
    if pair_list is None:
        pair_list = _pairs.forest_pairs(cat, bins)
    d = np.asarray(cat.delta if delta is None else delta, dtype=np.float64)
    fwd = xi_sums(cat, bins, pair_list, delta=d)
    W = fwd["wsum"]
    g = np.asarray(grad_xi, dtype=np.float64)
    gamma = np.divide(g, W, out=np.zeros_like(W), where=W != 0)
    rho = gamma * fwd["xi"]
    gd = np.zeros(cat.n_pix)
    gw = np.zeros(cat.n_pix)
    w_all = cat.weight.astype(np.float64)
    nvec = unit_vectors(cat.ra, cat.dec)
    for a, b in zip(*pair_list):
        sa, sb = cat.forest(a), cat.forest(b)
        if sa.stop == sa.start or sb.stop == sb.start:
            continue
        c, s = half_angle(nvec[a], nvec[b])
        A, ok, _, _ = pixel_pair_bins(cat.dist[sa], cat.dist[sb], c, s, bins)
        G = np.where(ok, gamma[np.maximum(A, 0)], 0.0)
        R = np.where(ok, rho[np.maximum(A, 0)], 0.0)
        wa, wb = w_all[sa], w_all[sb]
        da, db = d[sa], d[sb]
        wda, wdb = wa * da, wb * db
        ga = G @ wdb            # sum_j gamma (w d)_j, per i
        gb = G.T @ wda          # sum_i gamma (w d)_i, per j
        ra = R @ wb             # sum_j rho w_j
        rb = R.T @ wa
        gd[sa] += wa * ga
        gd[sb] += wb * gb
        gw[sa] += da * ga - ra
        gw[sb] += db * gb - rb
    return gd, gw, fwd


def loss(cat, bins, grad_xi, pair_list=None, delta=None, weight=None) -> float:
    """L = sum_A c_A xi_A, with optional replacement delta / weight arrays."""
    if weight is not None:
        import copy
        cat = copy.copy(cat)
        cat.weight = np.asarray(weight)
    out = xi_sums(cat, bins, pair_list, delta=delta)
    return float(np.dot(np.asarray(grad_xi, dtype=np.float64), out["xi"]))
