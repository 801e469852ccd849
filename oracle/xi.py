"""Two-point estimator, Eq. (2.4):  xi_A = sum_A (d_i w_i)(d_j w_j) / sum_A w_i w_j.

The sums run over pixel pairs (i, j) of different forests whose separation
lies in bin A (Section 2.1): the rectangle r_par in [p D_par, (p+1) D_par),
r_perp in [t D_perp, (t+1) D_perp), with D = r_max / n and A = p * n_perp + t.

Readings:

* the paper writes the rectangle with open ends; a value exactly on an edge
  goes to the upper bin (half-open intervals), in-grid iff p < n_par and
  t < n_perp (separations are non-negative);
* a bin with W_A = 0 has xi_A = 0;
* every unordered forest pair is counted once (``oracle.pairs``).

Alongside N_A and W_A the oracle returns per bin: the in-grid pixel-pair
count, sum of squared numerator terms (for the noise floor sigma_A =
sqrt(sum t^2) / W_A) and, for a given edge width eps (in bin units), the
absolute numerator and weight mass of pixel pairs whose scaled separation lies
within eps of a bin edge -- the mass that a separation computed with error
below eps could move between bins.
"""
from __future__ import annotations

import numpy as np

from .geometry import unit_vectors, half_angle, separations
from ._pool import map_pairs
from . import pairs as _pairs


def pixel_pair_bins(d_a, d_b, c, s, bins):
    """Scaled separations and bin of every pixel pair of one forest pair.

    Returns (A, in_grid, x, y) with x = r_par / D_par, y = r_perp / D_perp.
    """
    r_par, r_perp = separations(d_a, d_b, c, s)
    x = r_par / (bins.r_par_max / bins.n_par)
    y = r_perp / (bins.r_perp_max / bins.n_perp)
    p = np.floor(x)
    t = np.floor(y)
    ok = (p < bins.n_par) & (t < bins.n_perp)
    A = (p * bins.n_perp + t)
    A = np.where(ok, A, -1).astype(np.int64)
    return A, ok, x, y


def _xi_chunk(cat, bins, a_arr, b_arr, extra):
    eps = extra.get("eps_edge", 0.0)
    delta = extra["delta"]
    nb = bins.nbins
    num = np.zeros(nb)
    wsum = np.zeros(nb)
    cnt = np.zeros(nb)
    sq = np.zeros(nb)
    ew = np.zeros(nb)
    en = np.zeros(nb)
    cand = 0.0
    nvec = unit_vectors(cat.ra, cat.dec)
    for a, b in zip(a_arr, b_arr):
        sa, sb = cat.forest(a), cat.forest(b)
        if sa.stop == sa.start or sb.stop == sb.start:
            continue
        c, s = half_angle(nvec[a], nvec[b])
        A, ok, x, y = pixel_pair_bins(cat.dist[sa], cat.dist[sb], c, s, bins)
        wa = cat.weight[sa].astype(np.float64)
        wb = cat.weight[sb].astype(np.float64)
        wda = wa * delta[sa].astype(np.float64)
        wdb = wb * delta[sb].astype(np.float64)
        tw = wa[:, None] * wb[None, :]
        tn = wda[:, None] * wdb[None, :]
        cand += A.size
        Ai = A[ok]
        num += np.bincount(Ai, weights=tn[ok], minlength=nb)
        wsum += np.bincount(Ai, weights=tw[ok], minlength=nb)
        cnt += np.bincount(Ai, minlength=nb)
        sq += np.bincount(Ai, weights=tn[ok] ** 2, minlength=nb)
        if eps > 0.0:
            p_lo = np.floor(np.maximum(x - eps, 0.0))
            p_hi = np.floor(x + eps)
            t_lo = np.floor(np.maximum(y - eps, 0.0))
            t_hi = np.floor(y + eps)
            amb = (p_lo != p_hi) | (t_lo != t_hi)
            if np.any(amb):
                pl, ph, tl, th = p_lo[amb], p_hi[amb], t_lo[amb], t_hi[amb]
                aw, an = np.abs(tw[amb]), np.abs(tn[amb])
                combos = [(pl, tl, np.ones_like(pl, dtype=bool)),
                          (ph, tl, ph != pl),
                          (pl, th, th != tl),
                          (ph, th, (ph != pl) & (th != tl))]
                for pp, tt, use in combos:
                    m = use & (pp < bins.n_par) & (tt < bins.n_perp)
                    idx = (pp[m] * bins.n_perp + tt[m]).astype(np.int64)
                    ew += np.bincount(idx, weights=aw[m], minlength=nb)
                    en += np.bincount(idx, weights=an[m], minlength=nb)
    return {"num": num, "wsum": wsum, "count": cnt, "num_sq": sq, "edge_w": ew,
            "edge_n": en, "candidates": cand}


def xi_sums(cat, bins, pair_list=None, delta=None, eps_edge: float = 0.0,
            processes: int = 1):
    """N_A, W_A, xi_A and diagnostics over the given forest pairs (default:
    ``oracle.pairs.forest_pairs``).  ``delta`` overrides ``cat.delta``."""
    if pair_list is None:
        pair_list = _pairs.forest_pairs(cat, bins)
    a, b = pair_list
    extra = {"eps_edge": float(eps_edge),
             "delta": np.asarray(cat.delta if delta is None else delta)}
    out = map_pairs(_xi_chunk, cat, bins, a, b, extra, processes=processes)
    w = out["wsum"]
    out["xi"] = np.divide(out["num"], w, out=np.zeros_like(w), where=w != 0)
    out["sigma"] = np.divide(np.sqrt(out["num_sq"]), w, out=np.zeros_like(w), where=w != 0)
    out["pairs"] = len(a)
    return out


def _means_chunk(cat, bins, a_arr, b_arr, extra):
    eps_edge = extra.get("eps_edge", 0.0)
    zpix = extra.get("z")
    nb = bins.nbins
    W, WP, WT, WD, WZ, cnt, ew, ec = (np.zeros(nb) for _ in range(8))
    nvec = unit_vectors(cat.ra, cat.dec)
    for a, b in zip(a_arr, b_arr):
        sa, sb = cat.forest(a), cat.forest(b)
        if sa.stop == sa.start or sb.stop == sb.start:
            continue
        c, s = half_angle(nvec[a], nvec[b])
        r_par, r_perp = separations(cat.dist[sa], cat.dist[sb], c, s)
        A, ok, x, y = pixel_pair_bins(cat.dist[sa], cat.dist[sb], c, s, bins)
        tw = cat.weight[sa].astype(np.float64)[:, None] * cat.weight[sb].astype(np.float64)[None, :]
        dm = 0.5 * (np.asarray(cat.dist[sa], dtype=np.float64)[:, None] + np.asarray(cat.dist[sb], dtype=np.float64)[None, :])
        Ai = A[ok]
        W += np.bincount(Ai, weights=tw[ok], minlength=nb)
        WP += np.bincount(Ai, weights=(tw * r_par)[ok], minlength=nb)
        WT += np.bincount(Ai, weights=(tw * r_perp)[ok], minlength=nb)
        WD += np.bincount(Ai, weights=(tw * dm)[ok], minlength=nb)
        if zpix is not None:
            zm = 0.5 * (np.asarray(zpix[sa], dtype=np.float64)[:, None] + np.asarray(zpix[sb], dtype=np.float64)[None, :])
            WZ += np.bincount(Ai, weights=(tw * zm)[ok], minlength=nb)
        cnt += np.bincount(Ai, minlength=nb)
        if eps_edge > 0.0:
            p_lo = np.floor(np.maximum(x - eps_edge, 0.0))
            p_hi = np.floor(x + eps_edge)
            t_lo = np.floor(np.maximum(y - eps_edge, 0.0))
            t_hi = np.floor(y + eps_edge)
            amb = (p_lo != p_hi) | (t_lo != t_hi)
            if np.any(amb):
                pl, ph, tl, th = p_lo[amb], p_hi[amb], t_lo[amb], t_hi[amb]
                aw = np.abs(tw[amb])
                for pp, tt, use in ((pl, tl, np.ones_like(pl, dtype=bool)), (ph, tl, ph != pl),
                                    (pl, th, th != tl), (ph, th, (ph != pl) & (th != tl))):
                    m = use & (pp < bins.n_par) & (tt < bins.n_perp)
                    idx = (pp[m] * bins.n_perp + tt[m]).astype(np.int64)
                    ew += np.bincount(idx, weights=aw[m], minlength=nb)
                    ec += np.bincount(idx, minlength=nb)
    return {"W": W, "WP": WP, "WT": WT, "WD": WD, "WZ": WZ, "count": cnt, "edge_w": ew, "edge_c": ec}


def bin_means(cat, bins, pair_list=None, eps_edge: float = 0.0, processes: int = 1, z=None):
    """Per-bin weighted means of the separations and of the pair distance, and
    pixel-pair counts, over the pixel pairs of Eq. (2.4):

        rpar_mean_A  = sum_A w_i w_j r_par / W_A,   rperp_mean_A = sum_A w_i w_j r_perp / W_A,
        dist_mean_A  = sum_A w_i w_j (d_i + d_j) / 2 / W_A,   count_A = number of pairs in A,

    0 where W_A = 0.  These are the per-bin columns a PICCA/Vega fit reads next
    to xi (the paper exports its results for Vega, Appendix A).  With ``z``, a
    per-pixel redshift array of the catalogue's pixels, also the bin's mean
    redshift  z_mean_A = sum_A w_i w_j (z_i + z_j) / 2 / W_A  (the redshift of a
    pixel pair is the mean of its two pixels' redshifts).  With eps_edge > 0
    also ``edge_c``, the number of pairs within eps of an edge per candidate
    bin (as ``edge_w`` counts their weight)."""
    if pair_list is None:
        pair_list = _pairs.forest_pairs(cat, bins)
    a, b = pair_list
    extra = {"eps_edge": float(eps_edge)}
    if z is not None:
        extra["z"] = np.asarray(z, dtype=np.float64)
    t = map_pairs(_means_chunk, cat, bins, a, b, extra, processes=processes)
    W = t["W"]
    div = lambda v: np.divide(v, W, out=np.zeros_like(W), where=W != 0)
    out = {"wsum": W, "rpar_mean": div(t["WP"]), "rperp_mean": div(t["WT"]), "dist_mean": div(t["WD"]),
           "count": t["count"], "edge_w": t["edge_w"], "edge_c": t["edge_c"]}
    if z is not None:
        out["z_mean"] = div(t["WZ"])
    return out
