"""Pins of the oracle's three-point estimator (Eq. 2.8, Section 2.3)."""
import math

import numpy as np
import pytest

from conftest import line_catalog
from oracle import xi3 as ox3
from paper_2507_00129_gb300 import synth


def _points_catalog(points, deltas, weights):
    """One single-pixel forest per 3-D point (its line of sight through the point)."""
    fs = []
    for (x, y, z), dl, w in zip(points, deltas, weights):
        d = math.sqrt(x * x + y * y + z * z)
        fs.append((math.atan2(y, x) % (2 * math.pi), math.asin(z / d), [d], [8.2], [dl], [w]))
    return line_catalog(fs)


def test_hand_built_triangle():
    """Vertex on the z axis at 1000, r1 = (3, 0, 2), r2 = (0, 4, 1):
    |r1| = sqrt(13) = 3.61 (bin 1 of width 2), |r2| = sqrt(17) = 4.12 (bin 2),
    cos alpha = 2 / sqrt(221) = 0.1345 (bin 11 of 20 over [-1, 1]),
    theta1 = acos(2 / sqrt(13)) = 56.3 deg (bin 3 of 18 deg), theta2 = acos(1 / sqrt(17)) = 76.0 deg (bin 4)."""
    g = ox3.Grid3(n_r=5, n_theta=10, n_alpha=20, r_max=10.0)
    xi = (0.0, 0.0, 1000.0)
    pts = [xi, (3.0, 0.0, 1002.0), (0.0, 4.0, 1001.0)]
    cat = _points_catalog(pts, [0.5, -0.25, 0.4], [2.0, 3.0, 0.5])
    out = ox3.xi3_sums(cat, g)
    A = (((1 * 5 + 2) * 20 + 11) * 10 + 3) * 10 + 4
    A_swap = (((2 * 5 + 1) * 20 + 11) * 10 + 4) * 10 + 3
    w3 = 2.0 * 3.0 * 0.5
    n3 = (2.0 * 0.5) * (3.0 * -0.25) * (0.5 * 0.4)
    assert out["wsum"][A] == pytest.approx(w3) and out["wsum"][A_swap] == pytest.approx(w3)
    assert out["num"][A] == pytest.approx(n3)
    # every pixel is a main vertex once, with both orders: six records in all
    assert out["count"].sum() == 6
    assert out["wsum"].sum() == pytest.approx(6 * w3)
    assert out["xi"][A] == pytest.approx(n3 / w3)


def test_records_equal_brute_force_count():
    """The number of in-grid records is the count, over main vertices i, of
    ordered pairs (j, k) of pixels of two other, distinct forests with
    |x_j - x_i| < r_max and |x_k - x_i| < r_max (explicit loops)."""
    rng = np.random.default_rng(2)
    pts = [(rng.uniform(-6, 6), rng.uniform(-6, 6), 1000 + rng.uniform(-6, 6)) for _ in range(9)]
    cat = _points_catalog(pts, rng.normal(0, 1, 9), rng.uniform(0.5, 2, 9))
    g = ox3.Grid3(n_r=4, n_theta=10, n_alpha=20, r_max=8.0)
    out = ox3.xi3_sums(cat, g)
    P = np.array(pts)
    cnt = 0
    for i in range(9):
        for j in range(9):
            for k in range(9):
                if len({i, j, k}) == 3 and np.linalg.norm(P[j] - P[i]) < 8.0 and np.linalg.norm(P[k] - P[i]) < 8.0:
                    cnt += 1
    assert cnt > 20
    assert out["count"].sum() == cnt


def _small3():
    spec = synth.Spec(n_forests=30, seed=8, region="box", box_deg=0.6, grid="log10", delta_sigma=0.2)
    cat = synth.generate(spec)
    return synth.subset(cat, np.arange(30))


def test_symmetric_under_side_swap():
    cat = _small3()
    g = ox3.Grid3(n_r=5, n_theta=10, n_alpha=20, r_max=20.0)
    out = ox3.xi3_sums(cat, g, max_vertices=400)
    W = out["wsum"].reshape(g.n_r, g.n_r, g.n_alpha, g.n_theta, g.n_theta)
    np.testing.assert_allclose(W, W.transpose(1, 0, 2, 4, 3), rtol=1e-12)
    assert out["count"].sum() > 1000


def test_invariant_under_forest_order():
    cat = _small3()
    g = ox3.Grid3(n_r=5, n_theta=10, n_alpha=20, r_max=20.0)
    perm = np.random.default_rng(4).permutation(cat.n_forests)
    a = ox3.xi3_sums(cat, g)
    b = ox3.xi3_sums(synth.subset(cat, perm), g)
    np.testing.assert_allclose(b["wsum"], a["wsum"], rtol=1e-12)
    np.testing.assert_allclose(b["num"], a["num"], rtol=1e-9, atol=1e-12 * np.abs(a["num"]).max())


def test_edge_mass_brackets_rescaled_radius_bins():
    """Rescaling r_max (hence Delta_r) by less than eps_r bin units moves at
    most the edge mass."""
    cat = _small3()
    g = ox3.Grid3(n_r=5, n_theta=10, n_alpha=20, r_max=20.0)
    eps = 2e-3
    base = ox3.xi3_sums(cat, g, eps_r=eps, eps_c=1e-12, max_vertices=300)
    moved_any = False
    for scale in (1 + 0.9 * eps / g.n_r, 1 - 0.9 * eps / g.n_r):
        g2 = ox3.Grid3(n_r=5, n_theta=10, n_alpha=20, r_max=20.0 * scale)
        m = ox3.xi3_sums(cat, g2, max_vertices=300)
        # records with |r| within the rescaled r_max only: compare bins that stay inside both grids
        d = np.abs(m["wsum"] - base["wsum"])
        moved_any |= bool(np.any(d > 1e-9))
        assert np.all(d <= base["edge_w"] * (1 + 1e-12) + 1e-9 + _outer_edge(base, g, m))
    assert moved_any


def _outer_edge(base, g, m):
    """Records crossing r_max itself (in or out of the grid) are not bin flips;
    allow the full weight of the outermost r bins for them."""
    W = np.zeros_like(base["wsum"]).reshape(g.n_r, g.n_r, g.n_alpha, g.n_theta, g.n_theta)
    W[g.n_r - 1] = np.inf
    W[:, g.n_r - 1] = np.inf
    return W.reshape(-1)
