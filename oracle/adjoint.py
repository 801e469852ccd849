"""Gradient of L = sum_A c_A xi_A + sum_A e_A W_A with respect to delta and w.

Not in the paper; it is the chain rule applied to Eq. (2.4).  With
N_A = sum_A (w d)_i (w d)_j, W_A = sum_A w_i w_j, xi_A = N_A / W_A,
gamma_A = c_A / W_A and rho_A = gamma_A xi_A - e_A (gamma and gamma xi are 0
where W_A = 0):

    dL/d delta_i = w_i      sum_{j paired with i in grid} gamma_A (w d)_j
    dL/d w_i     = delta_i  sum_j gamma_A (w d)_j  -  sum_j rho_A w_j

where A is the bin of the pair (i, j) and j runs over pixels of the other
forest of every forest pair containing i.  The e_A term is dW_A/dw_i =
sum_{j in A} w_j, the weight sum's own dependence on w.
"""
from __future__ import annotations

import numpy as np

from .geometry import unit_vectors, half_angle
from .xi import pixel_pair_bins, xi_sums
from . import pairs as _pairs


def xi_grad(cat, bins, grad_xi, pair_list=None, delta=None, absolute: bool = False,
            eps_edge: float = 0.0, fwd=None, grad_wsum=None):
    """(dL/d delta, dL/d w, forward sums) for
    L = sum_A grad_xi[A] xi_A + sum_A grad_wsum[A] W_A (grad_wsum default 0).

    With ``absolute`` the forward dict also holds the same sums taken over the
    absolute values of the terms (the scale of rounding effects).  With
    ``eps_edge`` > 0 it holds, per pixel, the largest change of each gradient
    that moving the pixel pairs whose scaled separations lie within eps_edge
    of a bin edge into a neighbouring candidate bin can cause (the same
    candidate bins as ``oracle.xi``).  ``fwd`` may pass precomputed forward
    sums (num, wsum, xi) to use for gamma and rho."""
    if pair_list is None:
        pair_list = _pairs.forest_pairs(cat, bins)
    d = np.asarray(cat.delta if delta is None else delta, dtype=np.float64)
    if fwd is None:
        fwd = xi_sums(cat, bins, pair_list, delta=d)
    fwd = dict(fwd)
    W = fwd["wsum"]
    g = np.asarray(grad_xi, dtype=np.float64)
    gamma = np.divide(g, W, out=np.zeros_like(W), where=W != 0)
    rho = gamma * fwd["xi"]
    if grad_wsum is not None:
        rho = rho - np.asarray(grad_wsum, dtype=np.float64)
    gd = np.zeros(cat.n_pix)
    gw = np.zeros(cat.n_pix)
    gda = np.zeros(cat.n_pix)
    gwa = np.zeros(cat.n_pix)
    ega = np.zeros(cat.n_pix)
    ewa = np.zeros(cat.n_pix)
    w_all = cat.weight.astype(np.float64)
    nvec = unit_vectors(cat.ra, cat.dec)
    for a, b in zip(*pair_list):
        sa, sb = cat.forest(a), cat.forest(b)
        if sa.stop == sa.start or sb.stop == sb.start:
            continue
        c, s = half_angle(nvec[a], nvec[b])
        A, ok, x, y = pixel_pair_bins(cat.dist[sa], cat.dist[sb], c, s, bins)
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
        if eps_edge > 0.0:
            # largest |gamma'-gamma|, |rho'-rho| over the candidate bins of each ambiguous pair
            p_lo = np.floor(np.maximum(x - eps_edge, 0.0))
            p_hi = np.floor(x + eps_edge)
            t_lo = np.floor(np.maximum(y - eps_edge, 0.0))
            t_hi = np.floor(y + eps_edge)
            amb = (p_lo != p_hi) | (t_lo != t_hi)
            dG = np.zeros_like(G)
            dR = np.zeros_like(R)
            if np.any(amb):
                for pp, tt in ((p_lo, t_lo), (p_hi, t_lo), (p_lo, t_hi), (p_hi, t_hi)):
                    inside = (pp < bins.n_par) & (tt < bins.n_perp)
                    idx = np.where(inside, pp * bins.n_perp + tt, 0).astype(np.int64)
                    gc = np.where(inside, gamma[idx], 0.0)
                    rc = np.where(inside, rho[idx], 0.0)
                    dG = np.where(amb, np.maximum(dG, np.abs(gc - G)), dG)
                    dR = np.where(amb, np.maximum(dR, np.abs(rc - R)), dR)
            ega[sa] += np.abs(wa) * (dG @ np.abs(wdb))
            ega[sb] += np.abs(wb) * (dG.T @ np.abs(wda))
            ewa[sa] += np.abs(da) * (dG @ np.abs(wdb)) + dR @ np.abs(wb)
            ewa[sb] += np.abs(db) * (dG.T @ np.abs(wda)) + dR.T @ np.abs(wa)
        if absolute:
            Ga, Ra = np.abs(G), np.abs(R)
            gda[sa] += np.abs(wa) * (Ga @ np.abs(wdb))
            gda[sb] += np.abs(wb) * (Ga.T @ np.abs(wda))
            gwa[sa] += np.abs(da) * (Ga @ np.abs(wdb)) + Ra @ np.abs(wb)
            gwa[sb] += np.abs(db) * (Ga.T @ np.abs(wda)) + Ra.T @ np.abs(wa)
    if absolute:
        fwd["grad_delta_abs"] = gda
        fwd["grad_weight_abs"] = gwa
    if eps_edge > 0.0:
        fwd["grad_delta_edge"] = ega
        fwd["grad_weight_edge"] = ewa
    return gd, gw, fwd


def loss(cat, bins, grad_xi, pair_list=None, delta=None, weight=None, grad_wsum=None) -> float:
    """L = sum_A c_A xi_A (+ sum_A e_A W_A with e = grad_wsum), with optional
    replacement delta / weight arrays."""
    if weight is not None:
        import copy
        cat = copy.copy(cat)
        cat.weight = np.asarray(weight)
    out = xi_sums(cat, bins, pair_list, delta=delta)
    L = float(np.dot(np.asarray(grad_xi, dtype=np.float64), out["xi"]))
    if grad_wsum is not None:
        L += float(np.dot(np.asarray(grad_wsum, dtype=np.float64), out["wsum"]))
    return L
