"""Forest x quasar cross-correlation and its distortion matrix.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper lists the cross-correlation of forests with quasars as future work
of its pipeline (Section 4) and gives no formula for it.  Readings, taken
from the two-point machinery of Sections 2.1-2.2 with a quasar q (position
d_q n_q, weight w_q, no delta) in place of the second pixel:

* estimator (Eq. 2.4 with the quasar as second point):
      xi_A = sum_{(i,q) in A} w_i delta_i w_q / sum_{(i,q) in A} w_i w_q;
* separations (the bisector split of Section 2.1, signed along the line of
  sight because the two tracers differ):
      r_par  = (d_i - d_q) cos(theta/2),   r_perp = (d_i + d_q) sin(theta/2);
* bins: n_par rectangles of width D_par = 2 r_par_max / n_par over
  [-r_par_max, r_par_max), n_perp of width D_perp = r_perp_max / n_perp over
  [0, r_perp_max), half-open, p = floor((r_par + r_par_max) / D_par),
  t = floor(r_perp / D_perp), A = p n_perp + t;
* pairs: every pixel of every forest with every quasar except the forest's
  own quasar (``forest_qso[a]``, -1 for none);
* distortion matrix (Eq. 2.6 with the projection eta of Eq. 2.7 acting on the
  forest only):
      D_AB = W_A^-1 sum_{(a,q)} sum_{i: (i,q) in A} w_i w_q sum_{k: (k,q) in B} eta_ik,
  W_A the weight sum over the same (forest, quasar) pairs, which are a seeded
  Bernoulli(p) subsample: keep (a, q) iff SplitMix64(seed XOR (a 2^32 + q))
  < floor(p 2^64) (the rule of ``oracle.subsample`` on the ordered pair).

With eta = I - 1 u^T - x v^T (u = w / W_a, v = w x / S_a, x = Lambda - Lbar)
the inner sum is [bin(i,q) = B] - alpha_q[B] / W_a - x_i beta_q[B] / S_a with
the histograms alpha_q[B] = sum_{k: (k,q) in B} w_k and
beta_q[B] = sum_{k: (k,q) in B} w_k x_k, so one (forest, quasar) pair adds

    w_q (diag(alpha_q) - alpha_q alpha_q^T / W_a - beta_q beta_q^T / S_a)

to D~ = W D (terms of eta that ``oracle.project`` drops are absent here too).
``xdmat_literal`` sums the definition term by term; the tests check the two.

Edge allowance (``eps_edge`` > 0, bin units): a pixel whose scaled
separations lie within eps of an edge may land in any candidate bin.  Moving
pixel k of pair (a, q) to B changes column B of D~ by
v_k[A] = sum_{i: (i,q) in A} w_i w_q eta_ik and, because w_i eta_ik =
w_k eta_ki, row B by its transpose; two moved pixels i, k change entry
(cand(i), cand(k)) by w_i w_q eta_ik.  ``edge_d`` is the sum of these bounds.
"""
from __future__ import annotations

import numpy as np

from .geometry import unit_vectors, half_angle
from .project import eta_matrix, forest_moments
from .subsample import splitmix64, threshold


def pixel_bins(d_pix, d_q, c, s, bins):
    """Scaled separations and bin of every pixel of one forest with one quasar.

    Returns (A, in_grid, x, y), x = (r_par + r_par_max) / D_par,
    y = r_perp / D_perp; A = -1 outside the grid."""
    d_pix = np.asarray(d_pix, dtype=np.float64)
    r_par = (d_pix - d_q) * c
    r_perp = (d_pix + d_q) * s
    x = (r_par + bins.r_par_max) / (2.0 * bins.r_par_max / bins.n_par)
    y = r_perp / (bins.r_perp_max / bins.n_perp)
    p = np.floor(x)
    t = np.floor(y)
    ok = (p >= 0) & (p < bins.n_par) & (t < bins.n_perp)
    A = np.where(ok, p * bins.n_perp + t, -1).astype(np.int64)
    return A, ok, x, y


def keep_xpairs(a, q, seed: int, p: float) -> np.ndarray:
    """Subsample mask of ordered (forest, quasar) pairs."""
    a = np.asarray(a, dtype=np.int64)
    q = np.asarray(q, dtype=np.int64)
    if p >= 1.0:
        return np.ones(a.shape, dtype=bool)
    if p <= 0.0:
        return np.zeros(a.shape, dtype=bool)
    key = (a.astype(np.uint64) << np.uint64(32)) | q.astype(np.uint64)
    return splitmix64(np.uint64(seed) ^ key) < np.uint64(threshold(p))


def forest_quasar_pairs(cat, qso, bins, forest_qso=None, margin: float = 1e-3):
    """(a, q) pairs that can hold an in-grid (or edge-ambiguous) pixel:
    (d_first,a + d_q) sin(theta/2) < r_perp_max (1 + margin), own quasar
    excluded.  Brute force over all quasars; a prefilter only (r_perp of every
    pixel is at least that bound)."""
    nf = unit_vectors(cat.ra, cat.dec)
    nq = unit_vectors(qso.ra, qso.dec)
    lens = cat.lengths()
    A, Q = [], []
    for a in range(cat.n_forests):
        if lens[a] == 0:
            continue
        d0 = cat.dist[cat.offsets[a]]
        s = 0.5 * np.linalg.norm(nq - nf[a][None, :], axis=1)
        keep = (d0 + qso.dist) * s < bins.r_perp_max * (1.0 + margin)
        if forest_qso is not None and forest_qso[a] >= 0:
            keep[forest_qso[a]] = False
        qs = np.nonzero(keep)[0]
        A.append(np.full(len(qs), a, dtype=np.int64))
        Q.append(qs.astype(np.int64))
    if not A:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    return np.concatenate(A), np.concatenate(Q)


def _edge_candidates(x, y, eps, bins):
    """Candidate bins (up to 4 per pixel, -1 unused) of the pixels within eps of
    an edge, and the mask of those pixels."""
    p_lo = np.floor(x - eps)
    p_hi = np.floor(x + eps)
    t_lo = np.floor(np.maximum(y - eps, 0.0))
    t_hi = np.floor(y + eps)
    amb = (p_lo != p_hi) | (t_lo != t_hi)
    cands = np.full((len(x), 4), -1, dtype=np.int64)
    for k, (pp, tt) in enumerate(((p_lo, t_lo), (p_hi, t_lo), (p_lo, t_hi), (p_hi, t_hi))):
        inside = (pp >= 0) & (pp < bins.n_par) & (tt < bins.n_perp)
        cands[:, k] = np.where(inside, pp * bins.n_perp + tt, -1)
    for k in range(1, 4):
        dup = np.any(cands[:, :k] == cands[:, k:k + 1], axis=1)
        cands[dup, k] = -1
    return cands, amb


def xcf_sums(cat, qso, bins, pair_list=None, forest_qso=None, delta=None, eps_edge: float = 0.0):
    """N_A, W_A, xi_A and diagnostics over the (forest, quasar) pairs (default:
    ``forest_quasar_pairs``)."""
    if pair_list is None:
        pair_list = forest_quasar_pairs(cat, qso, bins, forest_qso)
    delta = np.asarray(cat.delta if delta is None else delta)
    nb = bins.nbins
    num, wsum, cnt, sq = np.zeros(nb), np.zeros(nb), np.zeros(nb), np.zeros(nb)
    ew, en = np.zeros(nb), np.zeros(nb)
    nf = unit_vectors(cat.ra, cat.dec)
    nq = unit_vectors(qso.ra, qso.dec)
    wq_all = qso.weight.astype(np.float64)
    for a, q in zip(*pair_list):
        sl = cat.forest(a)
        if sl.stop == sl.start:
            continue
        c, s = half_angle(nf[a], nq[q])
        A, ok, x, y = pixel_bins(cat.dist[sl], qso.dist[q], c, s, bins)
        w = cat.weight[sl].astype(np.float64)
        tw = w * wq_all[q]
        tn = w * delta[sl].astype(np.float64) * wq_all[q]
        Ai = A[ok]
        num += np.bincount(Ai, weights=tn[ok], minlength=nb)
        wsum += np.bincount(Ai, weights=tw[ok], minlength=nb)
        cnt += np.bincount(Ai, minlength=nb)
        sq += np.bincount(Ai, weights=tn[ok] ** 2, minlength=nb)
        if eps_edge > 0.0:
            cands, amb = _edge_candidates(x, y, eps_edge, bins)
            for k in range(4):
                m = amb & (cands[:, k] >= 0)
                ew += np.bincount(cands[m, k], weights=np.abs(tw[m]), minlength=nb)
                en += np.bincount(cands[m, k], weights=np.abs(tn[m]), minlength=nb)
    xi = np.divide(num, wsum, out=np.zeros_like(wsum), where=wsum != 0)
    sigma = np.divide(np.sqrt(sq), wsum, out=np.zeros_like(wsum), where=wsum != 0)
    return {"num": num, "wsum": wsum, "xi": xi, "count": cnt, "num_sq": sq, "sigma": sigma,
            "edge_w": ew, "edge_n": en, "pairs": len(pair_list[0])}


def _forest_eta(cat, a, eta_identity):
    sl = cat.forest(a)
    w = cat.weight[sl].astype(np.float64)
    return np.eye(len(w)) if eta_identity else eta_matrix(w, cat.loglam[sl])


def xdmat_literal(cat, qso, bins, pair_list, eta_identity: bool = False):
    """Distortion matrix summed term by term (tiny catalogues only)."""
    nb = bins.nbins
    dt = np.zeros((nb, nb))
    wdm = np.zeros(nb)
    nf = unit_vectors(cat.ra, cat.dec)
    nq = unit_vectors(qso.ra, qso.dec)
    for a, q in zip(*pair_list):
        sl = cat.forest(a)
        if sl.stop == sl.start:
            continue
        c, s = half_angle(nf[a], nq[q])
        A, ok, _, _ = pixel_bins(cat.dist[sl], qso.dist[q], c, s, bins)
        w = cat.weight[sl].astype(np.float64)
        wq = float(qso.weight[q])
        eta = _forest_eta(cat, a, eta_identity)
        idx = np.nonzero(ok)[0]
        for i in idx:
            wdm[A[i]] += w[i] * wq
            for k in idx:
                dt[A[i], A[k]] += w[i] * wq * eta[i, k]
    D = np.divide(dt, wdm[:, None], out=np.zeros_like(dt), where=wdm[:, None] != 0)
    return {"dmat": D, "dtilde": dt, "wsum": wdm}


def xdmat(cat, qso, bins, pair_list, eta_identity: bool = False, eps_edge: float = 0.0):
    """Distortion matrix via the expanded eta (module docstring).  Returns
    dict(dmat, dtilde, wsum) and, with eps_edge > 0, edge_d and edge_w (the
    weight that could move between bins of W_A)."""
    nb = bins.nbins
    dt = np.zeros((nb, nb))
    wdm = np.zeros(nb)
    E = np.zeros((nb + 1, nb + 1)) if eps_edge > 0 else None
    E2 = np.zeros((nb + 1, nb + 1)) if eps_edge > 0 else None
    ew = np.zeros(nb + 1)
    nf = unit_vectors(cat.ra, cat.dec)
    nq = unit_vectors(qso.ra, qso.dec)
    for a, q in zip(*pair_list):
        sl = cat.forest(a)
        if sl.stop == sl.start:
            continue
        c, s = half_angle(nf[a], nq[q])
        A, ok, x, y = pixel_bins(cat.dist[sl], qso.dist[q], c, s, bins)
        w = cat.weight[sl].astype(np.float64)
        wq = float(qso.weight[q])
        if E is not None:
            cands, amb = _edge_candidates(x, y, eps_edge, bins)
            ks = np.nonzero(amb)[0]
            if len(ks):
                eta = _forest_eta(cat, a, eta_identity)
                ii = np.nonzero(ok)[0]
                cc = np.where(cands[ks] >= 0, cands[ks], nb)
                for r, k in enumerate(ks):
                    v = np.abs(np.bincount(A[ii], weights=w[ii] * wq * eta[ii, k], minlength=nb + 1))
                    for B in cc[r]:
                        E[:, B] += v
                        ew[B] += abs(w[k] * wq)
                T = np.abs(w[ks][:, None] * wq * eta[np.ix_(ks, ks)])
                for s1 in range(4):
                    for s2 in range(4):
                        np.add.at(E2, (cc[:, s1][:, None], cc[:, s2][None, :]), T)
        if not np.any(ok):
            continue
        idx = np.nonzero(ok)[0]
        uniq, loc = np.unique(A[idx], return_inverse=True)
        L = len(uniq)
        alpha = np.bincount(loc, weights=w[idx], minlength=L)
        upd = np.diag(alpha)
        if not eta_identity:
            Wa, _, Sa, xa = forest_moments(w, cat.loglam[sl])
            if Wa > 0:
                upd -= np.outer(alpha, alpha) / Wa
                if Sa > 0:
                    beta = np.bincount(loc, weights=w[idx] * xa[idx], minlength=L)
                    upd -= np.outer(beta, beta) / Sa
        dt[np.ix_(uniq, uniq)] += wq * upd
        wdm[uniq] += wq * alpha
    D = np.divide(dt, wdm[:, None], out=np.zeros_like(dt), where=wdm[:, None] != 0)
    out = {"dmat": D, "dtilde": dt, "wsum": wdm}
    if E is not None:
        E, E2 = E[:nb, :nb], E2[:nb, :nb]
        out["edge_d"] = E + E.T + E2
        out["edge_w"] = ew[:nb]
    return out
