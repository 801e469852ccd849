"""Three-point estimator, Eq. (2.8) (Section 2.3):

    xi3_A = sum_A (w d)_i (w d)_j (w d)_k / sum_A w_i w_j w_k

over pixel triplets (i, j, k) of three distinct forests (quasars).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

A triangle is a main vertex i with the displacement vectors r1 = x_j - x_i and
r2 = x_k - x_i, x = d n the comoving position of a pixel (distance d along its
forest's unit vector n).  It is binned in five variables (Section 2.3 and the
caption of the 3PCF figure): the side lengths r1, r2 (n_r bins over
[0, r_max)), the inner angle alpha between r1 and r2 (n_alpha bins of cos alpha
over [-1, 1]) and the angles theta1, theta2 of r1, r2 to the line of sight
(n_theta bins over [0, pi]), flattened in that order into the triangle index

    A = (((i_r1 n_r + i_r2) n_alpha + i_alpha) n_theta + i_theta1) n_theta + i_theta2.

Readings (the paper leaves these open):

* every triplet is recorded once with each of its pixels as main vertex (the
  figure caption: the same triangle is recorded depending on which point is
  the main vertex), and, for a given vertex, with both assignments of the
  other two pixels to (r1, r2) -- so the estimator is symmetric under
  (r1, theta1) <-> (r2, theta2);
* a record enters the grid iff |r1| < r_max and |r2| < r_max (the third side
  is not restricted);
* the line of sight of a record is the main vertex's (its forest's unit
  vector);
* bins are half-open; cos alpha = 1 and theta = pi (values on the last edge)
  go to the last bin;
* the figure's grid is r in [0, 80) Mpc/h in 20 bins, theta in 10 bins and
  cos alpha in 20 bins; the timings use r_max = 40 Mpc/h.

Edge allowance: a record is ambiguous if r/Delta_r lies within eps_r of an
integer, or cos theta or cos alpha lies within eps_c of a bin edge (the
quantities a single-precision computation compares); its absolute terms are
added to every bin reachable by moving each ambiguous variable across the
nearby edge (the record's own bin included).
"""
from __future__ import annotations

import dataclasses
import itertools
import math

import numpy as np

from .geometry import unit_vectors


@dataclasses.dataclass
class Grid3:
    n_r: int
    n_theta: int
    n_alpha: int
    r_max: float

    @property
    def nbins(self) -> int:
        return self.n_r * self.n_r * self.n_alpha * self.n_theta * self.n_theta


def triangle_index(grid: Grid3, ir1, ir2, ia, it1, it2):
    return (((ir1 * grid.n_r + ir2) * grid.n_alpha + ia) * grid.n_theta + it1) * grid.n_theta + it2


def _r_bin(r, grid):
    return np.minimum(np.floor(r / (grid.r_max / grid.n_r)).astype(np.int64), grid.n_r - 1)


def _theta_bin(cos_t, grid):
    th = np.arccos(np.clip(cos_t, -1.0, 1.0))
    return np.minimum(np.floor(th / (math.pi / grid.n_theta)).astype(np.int64), grid.n_theta - 1)


def _alpha_bin(cos_a, grid):
    return np.minimum(np.floor((np.clip(cos_a, -1.0, 1.0) + 1.0) / (2.0 / grid.n_alpha)).astype(np.int64),
                      grid.n_alpha - 1)


def _alts(idx, near_lo, near_hi, n):
    """Candidate indices: idx, idx-1 if near the lower edge, idx+1 if near the upper edge."""
    lo = np.where(near_lo, np.maximum(idx - 1, 0), idx)
    hi = np.where(near_hi, np.minimum(idx + 1, n - 1), idx)
    return lo, hi


def xi3_sums(cat, grid: Grid3, eps_r: float = 0.0, eps_c: float = 0.0, max_vertices=None):
    """N_A, W_A, xi3_A, the in-grid record count, sum of squared numerator
    terms and (with eps > 0) the edge masses, over all main vertices (or the
    first ``max_vertices`` pixels)."""
    nb = grid.nbins
    num = np.zeros(nb)
    wsum = np.zeros(nb)
    cnt = np.zeros(nb)
    sq = np.zeros(nb)
    ew = np.zeros(nb)
    en = np.zeros(nb)
    nvec = unit_vectors(cat.ra, cat.dec)
    lens = np.diff(cat.offsets)
    forest = np.repeat(np.arange(cat.n_forests), lens)
    pos = cat.dist[:, None] * nvec[forest]
    w = cat.weight.astype(np.float64)
    wd = w * cat.delta.astype(np.float64)
    dr = grid.r_max / grid.n_r
    th_edges = np.cos(np.arange(1, grid.n_theta) * (math.pi / grid.n_theta))      # decreasing
    a_edges = -1.0 + np.arange(1, grid.n_alpha) * (2.0 / grid.n_alpha)
    nv = cat.n_pix if max_vertices is None else min(cat.n_pix, max_vertices)
    for i in range(nv):
        fi = forest[i]
        R = pos - pos[i]
        dist = np.sqrt(np.einsum("ij,ij->i", R, R))
        cand = np.nonzero((forest != fi) & (dist < grid.r_max))[0]
        if len(cand) < 2:
            continue
        Rc, dc, fc = R[cand], dist[cand], forest[cand]
        ni = nvec[fi]
        cth = (Rc @ ni) / dc
        ir = _r_bin(dc, grid)
        it = _theta_bin(cth, grid)
        p, q = np.nonzero(fc[:, None] != fc[None, :])          # ordered pairs of distinct forests
        if len(p) == 0:
            continue
        ca = np.einsum("ij,ij->i", Rc[p], Rc[q]) / (dc[p] * dc[q])
        ia = _alpha_bin(ca, grid)
        A = triangle_index(grid, ir[p], ir[q], ia, it[p], it[q])
        tw = w[i] * w[cand][p] * w[cand][q]
        tn = wd[i] * wd[cand][p] * wd[cand][q]
        num += np.bincount(A, weights=tn, minlength=nb)
        wsum += np.bincount(A, weights=tw, minlength=nb)
        cnt += np.bincount(A, minlength=nb)
        sq += np.bincount(A, weights=tn * tn, minlength=nb)
        if eps_r > 0.0 or eps_c > 0.0:
            x = dc / dr
            # r: near an integer (the upper edge of bin ir or the lower one)
            r_lo = (x - np.floor(x)) < eps_r
            r_hi = (np.ceil(x) - x) < eps_r
            # cos theta: bins decrease in cos; edge k (k = 1..n-1) is the upper edge of bin k-1 in theta
            dth = np.abs(cth[:, None] - th_edges[None, :]) < eps_c
            t_lo = np.zeros(len(cand), bool)
            t_hi = np.zeros(len(cand), bool)
            if dth.any():
                k = np.arange(1, grid.n_theta)[None, :]
                t_lo = np.any(dth & (k == it[:, None]), axis=1)        # edge between it-1 and it
                t_hi = np.any(dth & (k == it[:, None] + 1), axis=1)    # edge between it and it+1
            da = np.abs(ca[:, None] - a_edges[None, :]) < eps_c
            a_lo = np.zeros(len(p), bool)
            a_hi = np.zeros(len(p), bool)
            if da.any():
                k = np.arange(1, grid.n_alpha)[None, :]
                a_lo = np.any(da & (k == ia[:, None]), axis=1)
                a_hi = np.any(da & (k == ia[:, None] + 1), axis=1)
            amb = r_lo[p] | r_hi[p] | r_lo[q] | r_hi[q] | t_lo[p] | t_hi[p] | t_lo[q] | t_hi[q] | a_lo | a_hi
            if np.any(amb):
                sel = np.nonzero(amb)[0]
                opts = []
                for idx, lo, hi, n in ((ir[p][sel], r_lo[p][sel], r_hi[p][sel], grid.n_r),
                                       (ir[q][sel], r_lo[q][sel], r_hi[q][sel], grid.n_r),
                                       (ia[sel], a_lo[sel], a_hi[sel], grid.n_alpha),
                                       (it[p][sel], t_lo[p][sel], t_hi[p][sel], grid.n_theta),
                                       (it[q][sel], t_lo[q][sel], t_hi[q][sel], grid.n_theta)):
                    opts.append(_alts(idx, lo, hi, n))
                for combo in itertools.product(*[(0, 1, 2)] * 5):
                    # 0: own index, 1: lower alternative, 2: upper alternative
                    vals = []
                    use = np.ones(len(sel), bool)
                    for c, (idx, (lo, hi)) in zip(combo, zip((ir[p][sel], ir[q][sel], ia[sel], it[p][sel], it[q][sel]),
                                                             opts)):
                        v = idx if c == 0 else (lo if c == 1 else hi)
                        use &= (v != idx) if c != 0 else True
                        vals.append(v)
                    if not use.any():
                        continue
                    B = triangle_index(grid, *vals)
                    ew += np.bincount(B[use], weights=np.abs(tw[sel][use]), minlength=nb)
                    en += np.bincount(B[use], weights=np.abs(tn[sel][use]), minlength=nb)
    xi = np.divide(num, wsum, out=np.zeros_like(wsum), where=wsum != 0)
    sigma = np.divide(np.sqrt(sq), wsum, out=np.zeros_like(wsum), where=wsum != 0)
    return {"num": num, "wsum": wsum, "xi": xi, "count": cnt, "num_sq": sq, "sigma": sigma,
            "edge_w": ew, "edge_n": en}
