"""Distortion matrix, Eq. (2.6) (Section 2.2):

    D_AB = W_A^-1 sum_{(i,j) in A} w_i w_j sum_{(k,l) in B} eta_ik eta_jl,
    W_A  = sum_{(i,j) in A} w_i w_j

with eta of Eq. (2.7), non-zero only inside a forest: for a pixel pair (i, j)
of forests (a, b) the inner sum runs over pixel pairs (k, l) of the same
forests, k in a, l in b.

Readings:

* W_A is the weight sum over the pairs that enter D (the subsample), so that
  eta = identity gives D = identity exactly;
* a bin with W_A = 0 has a zero row;
* the subsample is ``oracle.subsample``.

Two forms:

``dmat_literal`` -- the quadruple sum as written (tiny forests only).

``dmat`` -- the same sum with eta = I - 1 u^T - x v^T (u = w/W, v = w x / S,
x = Lambda - Lbar) multiplied out.  With, for one forest pair,

    T1[A]  = sum_A w_i w_j,      Tx[A] = sum_A w_i w_j x_i,
    Ty[A]  = sum_A w_i w_j y_j,  Txy[A] = sum_A w_i w_j x_i y_j,
    alpha_j[A]  = sum_{i: (i,j) in A} w_i,  beta_j[A]  = sum_{i: (i,j) in A} w_i x_i,
    alpha'_i[A] = sum_{j: (i,j) in A} w_j,  beta'_i[A] = sum_{j: (i,j) in A} w_j y_j,

(x for forest a, y for forest b) the pair adds to  sum_{(i,j) in A} w_i w_j sum_B eta eta

    diag(T1)
    - sum_j w_j (alpha_j alpha_j^T / W_a + beta_j beta_j^T / S_a)
    - sum_i w_i (alpha'_i alpha'_i^T / W_b + beta'_i beta'_i^T / S_b)
    + T1 T1^T / (W_a W_b) + Ty Ty^T / (W_a S_b) + Tx Tx^T / (S_a W_b) + Txy Txy^T / (S_a S_b)

where each term whose forest term of eta is dropped (W = 0 or S = 0, see
``oracle.project``) is absent.  W_a and S_a run over all pixels of forest a.
The tests check the two forms against each other.

Edge allowance (``eps_edge`` > 0).  A pixel pair (k, l) whose scaled
separation lies within eps of a bin edge may be binned in any of its candidate
bins (the same candidates as ``oracle.xi``) by a separation computed with an
error below eps.  Moving it changes column B of D~ by
v_kl[A] = sum_{(i,j) in A} w_i w_j eta_ik eta_jl in every row A, and, since
w_i eta_ik = w_k eta_ki, row B by the transpose.  ``edge_d[A, B]`` bounds
|change of D~_AB| for any such rebinning of the ambiguous pairs: the sum of
|v_kl[A]| over ambiguous (k, l) with candidate B, the same transposed, and
|w_i w_j eta_ik eta_jl| for every two ambiguous pairs (i, j), (k, l) of a
forest pair whose candidates include A and B (both moved).
"""
from __future__ import annotations

import numpy as np

from .geometry import unit_vectors, half_angle
from .project import eta_matrix, forest_moments
from .xi import pixel_pair_bins
from ._pool import map_pairs
from . import pairs as _pairs


def dmat_literal(cat, bins, pair_list=None, eta_identity: bool = False):
    """Eq. (2.6) summed term by term.  Returns dict(dmat, dtilde, wsum)."""
    if pair_list is None:
        pair_list = _pairs.forest_pairs(cat, bins)
    nb = bins.nbins
    dt = np.zeros((nb, nb))
    wdm = np.zeros(nb)
    nvec = unit_vectors(cat.ra, cat.dec)
    for a, b in zip(*pair_list):
        sa, sb = cat.forest(a), cat.forest(b)
        c, s = half_angle(nvec[a], nvec[b])
        A, ok, _, _ = pixel_pair_bins(cat.dist[sa], cat.dist[sb], c, s, bins)
        wa = cat.weight[sa].astype(np.float64)
        wb = cat.weight[sb].astype(np.float64)
        if eta_identity:
            ea, eb = np.eye(len(wa)), np.eye(len(wb))
        else:
            ea, eb = eta_matrix(wa, cat.loglam[sa]), eta_matrix(wb, cat.loglam[sb])
        ij = list(zip(*np.nonzero(ok)))
        for (i, j) in ij:
            wdm[A[i, j]] += wa[i] * wb[j]
            for (k, l) in ij:
                dt[A[i, j], A[k, l]] += wa[i] * wb[j] * ea[i, k] * eb[j, l]
    D = np.divide(dt, wdm[:, None], out=np.zeros_like(dt), where=wdm[:, None] != 0)
    return {"dmat": D, "dtilde": dt, "wsum": wdm}


def _edge_terms(A, x, y, ii, jj, wa, wb, ea, eb, eps, bins, E, E2):
    """Edge allowance of one forest pair (see the module docstring).

    For every pixel pair (k, l) within eps of a bin edge, |v_kl| is added to
    column B of E for each candidate bin B; for every two such pairs (i, j),
    (k, l) (the same pair included), |w_i w_j eta_ik eta_jl| is added to E2 at
    every (candidate of (i, j), candidate of (k, l)).  Index nb is a dummy
    row / column for the unused candidate slots."""
    nb = bins.nbins
    p_lo = np.floor(np.maximum(x - eps, 0.0))
    p_hi = np.floor(x + eps)
    t_lo = np.floor(np.maximum(y - eps, 0.0))
    t_hi = np.floor(y + eps)
    amb = (p_lo != p_hi) | (t_lo != t_hi)
    ka, la = np.nonzero(amb)
    if len(ka) == 0:
        return
    cands = np.full((len(ka), 4), nb, dtype=np.int64)
    for s_, (pp, tt) in enumerate(((p_lo, t_lo), (p_hi, t_lo), (p_lo, t_hi), (p_hi, t_hi))):
        pv, tv = pp[ka, la], tt[ka, la]
        inside = (pv < bins.n_par) & (tv < bins.n_perp)
        cands[:, s_] = np.where(inside, (pv * bins.n_perp + tv).astype(np.int64), nb)
    # the same bin may appear in several slots: keep the first
    for s_ in range(1, 4):
        dup = np.any(cands[:, :s_] == cands[:, s_:s_ + 1], axis=1)
        cands[dup, s_] = nb
    rows = A[ii, jj]
    for q, (k, l) in enumerate(zip(ka, la)):
        v = np.abs(np.bincount(rows, weights=(wa[ii] * ea[ii, k]) * (wb[jj] * eb[jj, l]), minlength=nb + 1))
        for B in cands[q]:
            E[:, B] += v
    T = np.abs((wa[ka][:, None] * ea[np.ix_(ka, ka)]) * (wb[la][:, None] * eb[np.ix_(la, la)]))
    for s1 in range(4):
        for s2 in range(4):
            np.add.at(E2, (cands[:, s1][:, None], cands[:, s2][None, :]), T)


def _dm_chunk(cat, bins, a_arr, b_arr, extra):
    eta_identity = extra["eta_identity"]
    eps = extra.get("eps_edge", 0.0)
    nb = bins.nbins
    dt = np.zeros((nb, nb))
    wdm = np.zeros(nb)
    E = np.zeros((nb + 1, nb + 1)) if eps > 0.0 else None
    E2 = np.zeros((nb + 1, nb + 1)) if eps > 0.0 else None
    nvec = unit_vectors(cat.ra, cat.dec)
    for a, b in zip(a_arr, b_arr):
        sa, sb = cat.forest(a), cat.forest(b)
        na, nbp = sa.stop - sa.start, sb.stop - sb.start
        if na == 0 or nbp == 0:
            continue
        c, s = half_angle(nvec[a], nvec[b])
        A, ok, x, y = pixel_pair_bins(cat.dist[sa], cat.dist[sb], c, s, bins)
        if not np.any(ok):
            continue
        ii, jj = np.nonzero(ok)
        if E is not None:
            w_a = cat.weight[sa].astype(np.float64)
            w_b = cat.weight[sb].astype(np.float64)
            if eta_identity:
                ea, eb = np.eye(na), np.eye(nbp)
            else:
                ea, eb = eta_matrix(w_a, cat.loglam[sa]), eta_matrix(w_b, cat.loglam[sb])
            _edge_terms(A, x, y, ii, jj, w_a, w_b, ea, eb, eps, bins, E, E2)
        uniq, loc = np.unique(A[ii, jj], return_inverse=True)
        L = len(uniq)
        wa = cat.weight[sa].astype(np.float64)
        wb = cat.weight[sb].astype(np.float64)
        Wa, _, Sa, xa = forest_moments(wa, cat.loglam[sa])
        Wb, _, Sb, yb = forest_moments(wb, cat.loglam[sb])
        tw = wa[ii] * wb[jj]
        T1 = np.bincount(loc, weights=tw, minlength=L)
        D = np.diag(T1)
        if not eta_identity:
            Tx = np.bincount(loc, weights=tw * xa[ii], minlength=L)
            Ty = np.bincount(loc, weights=tw * yb[jj], minlength=L)
            Txy = np.bincount(loc, weights=tw * xa[ii] * yb[jj], minlength=L)
            col = jj * L + loc
            row = ii * L + loc
            alpha = np.bincount(col, weights=wa[ii], minlength=nbp * L).reshape(nbp, L)
            beta = np.bincount(col, weights=wa[ii] * xa[ii], minlength=nbp * L).reshape(nbp, L)
            alphap = np.bincount(row, weights=wb[jj], minlength=na * L).reshape(na, L)
            betap = np.bincount(row, weights=wb[jj] * yb[jj], minlength=na * L).reshape(na, L)
            if Wa > 0:
                D -= (alpha.T * wb[None, :]) @ alpha / Wa
            if Sa > 0:
                D -= (beta.T * wb[None, :]) @ beta / Sa
            if Wb > 0:
                D -= (alphap.T * wa[None, :]) @ alphap / Wb
            if Sb > 0:
                D -= (betap.T * wa[None, :]) @ betap / Sb
            if Wa > 0 and Wb > 0:
                D += np.outer(T1, T1) / (Wa * Wb)
            if Wa > 0 and Sb > 0:
                D += np.outer(Ty, Ty) / (Wa * Sb)
            if Sa > 0 and Wb > 0:
                D += np.outer(Tx, Tx) / (Sa * Wb)
            if Sa > 0 and Sb > 0:
                D += np.outer(Txy, Txy) / (Sa * Sb)
        dt[np.ix_(uniq, uniq)] += D
        wdm[uniq] += T1
    out = {"dtilde": dt, "wsum": wdm}
    if E is not None:
        E, E2 = E[:nb, :nb], E2[:nb, :nb]
        out["edge_d"] = E + E.T + E2
    return out


def dmat(cat, bins, pair_list=None, eta_identity: bool = False, processes: int = 1,
         eps_edge: float = 0.0):
    """Eq. (2.6) via the expanded eta.  Returns dict(dmat, dtilde, wsum) and,
    with eps_edge > 0, the column edge allowance edge_d (module docstring)."""
    if pair_list is None:
        pair_list = _pairs.forest_pairs(cat, bins)
    a, b = pair_list
    out = map_pairs(_dm_chunk, cat, bins, a, b,
                    {"eta_identity": bool(eta_identity), "eps_edge": float(eps_edge)},
                    processes=processes, chunk=200)
    w = out["wsum"]
    out["dmat"] = np.divide(out["dtilde"], w[:, None], out=np.zeros_like(out["dtilde"]),
                            where=w[:, None] != 0)
    return out


def pair_pairs(cat, bins, pair_list) -> float:
    """Number of terms of the quadruple sum of Eq. (2.6): sum over forest pairs
    of (in-grid pixel pairs)^2."""
    nvec = unit_vectors(cat.ra, cat.dec)
    tot = 0.0
    for a, b in zip(*pair_list):
        sa, sb = cat.forest(a), cat.forest(b)
        c, s = half_angle(nvec[a], nvec[b])
        _, ok, _, _ = pixel_pair_bins(cat.dist[sa], cat.dist[sb], c, s, bins)
        k = float(np.count_nonzero(ok))
        tot += k * k
    return tot


def closed_form_work(cat, bins, pair_list) -> dict:
    """Work counts of the closed form above, per forest pair of ``pair_list``:
    the in-grid pixel pairs, the sum over rank-1 vectors (each column j of b,
    a histogram over i of a, and each row i of a) of |S_v|^2 with |S_v| the
    number of distinct bins the vector's pixel pairs fall in, and the sum of
    |S_pair|^2 over pairs with |S_pair| the distinct bins of the pair.  The
    algorithmic flops of the closed form are about 20 per in-grid pixel pair
    plus 4 sum |S_v|^2 (two rank-1 outer products per vector) plus
    8 sum |S_pair|^2 (four T outer products)."""
    nvec = unit_vectors(cat.ra, cat.dec)
    pix = 0
    sv2 = 0.0
    sp2 = 0.0
    for a, b in zip(*pair_list):
        sa, sb = cat.forest(a), cat.forest(b)
        if sa.stop == sa.start or sb.stop == sb.start:
            continue
        c, s = half_angle(nvec[a], nvec[b])
        A, ok, _, _ = pixel_pair_bins(cat.dist[sa], cat.dist[sb], c, s, bins)
        if not np.any(ok):
            continue
        pix += int(np.count_nonzero(ok))
        for j in range(A.shape[1]):
            sv2 += float(len(np.unique(A[ok[:, j], j]))) ** 2
        for i in range(A.shape[0]):
            sv2 += float(len(np.unique(A[i, ok[i, :]]))) ** 2
        sp2 += float(len(np.unique(A[ok]))) ** 2
    return {"pixel_pairs": pix, "sum_vec_support_sq": sv2, "sum_pair_support_sq": sp2,
            "flops": 20.0 * pix + 4.0 * sv2 + 8.0 * sp2}
