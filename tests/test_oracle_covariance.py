"""Pins of the oracle's HEALPix sub-samples and sub-sample covariance."""
import math

import numpy as np
import pytest

from oracle import covariance as ocov, pairs, xi as oxi
from paper_2507_00129_gb300 import synth


def test_base_pixels_at_nside_1():
    """Near the centres of the twelve base pixels: four around the north pole at
    longitudes pi/4 + k pi/2, four on the equator at k pi/2, four in the south."""
    k = np.arange(4)
    z = np.concatenate([np.full(4, 0.6), np.zeros(4), np.full(4, -0.6)])
    phi = np.concatenate([math.pi / 4 + k * math.pi / 2, k * math.pi / 2, math.pi / 4 + k * math.pi / 2])
    np.testing.assert_array_equal(ocov.ang2pix_nest(1, z, phi), np.arange(12))
    # the poles belong to the first pixel of the polar base pixels' quarter
    assert ocov.ang2pix_nest(1, np.array([1.0]), np.array([0.1]))[0] == 0
    assert ocov.ang2pix_nest(1, np.array([-1.0]), np.array([0.1]))[0] == 8


def test_face_orientation_of_the_nested_numbering():
    """Within a base pixel the nested index interleaves x (even bits) and y
    (odd bits), x counting from the pixel's southern corner toward its eastern
    corner and y toward its western corner (the HEALPix grid of Gorski et al.
    2005).  At nside 2 the four sub-pixels of a base pixel f are 4f (south),
    4f+1 (east), 4f+2 (west) and 4f+3 (north).  Base pixel 4 spans longitudes
    -pi/4 .. pi/4 on the equator, so its east and west sub-pixels have their
    centres at longitudes +pi/8 and -pi/8; base pixel 0 has its western corner
    at (z = 2/3, phi = 0) and its eastern corner at (z = 2/3, phi = pi/2).
    Swapping x and y exchanges 4f+1 and 4f+2, which these points tell apart."""
    eq = ocov.ang2pix_nest(2, np.zeros(4), np.array([math.pi / 8, -math.pi / 8, 0.01, -0.01]))
    np.testing.assert_array_equal(eq, [17, 18, 17, 18])
    # equator, just above and below phi = 0 on the south / north halves
    assert ocov.ang2pix_nest(2, np.array([-0.3]), np.array([0.0]))[0] == 16
    assert ocov.ang2pix_nest(2, np.array([0.3]), np.array([0.0]))[0] == 19
    # polar base pixel 0 near its east and west corners (z just below 2/3)
    pol = ocov.ang2pix_nest(2, np.full(2, 0.66), np.array([math.pi / 2 - 0.02, 0.02]))
    np.testing.assert_array_equal(pol, [1, 2])
    # and near its north corner, the pole
    assert ocov.ang2pix_nest(2, np.array([0.999]), np.array([math.pi / 4]))[0] == 3


@pytest.mark.parametrize("nside", [1, 2, 4, 8, 16, 32, 64])
def test_nested_hierarchy(nside):
    """In the nested scheme pixel p at nside splits into 4p .. 4p+3 at 2 nside."""
    rng = np.random.default_rng(nside)
    z = rng.uniform(-1, 1, 20000)
    phi = rng.uniform(0, 2 * math.pi, 20000)
    np.testing.assert_array_equal(ocov.ang2pix_nest(2 * nside, z, phi) // 4, ocov.ang2pix_nest(nside, z, phi))


def test_equal_area_pixels():
    """Points uniform on the sphere fill the 192 pixels of nside 4 evenly."""
    rng = np.random.default_rng(3)
    n = 400000
    p = ocov.ang2pix_nest(4, rng.uniform(-1, 1, n), rng.uniform(0, 2 * math.pi, n))
    counts = np.bincount(p, minlength=192)
    assert counts.shape == (192,) and counts.min() > 0
    mean = n / 192
    assert np.max(np.abs(counts - mean)) < 5 * math.sqrt(mean)


def test_covariance_hand_example():
    """Two sub-samples, one bin: W = (1, 3), N = (2, 0): xi = 2/4, and
    C = (1^2 (2 - 0.5)^2 + 3^2 (0 - 0.5)^2) / 4^2 = 0.28125."""
    C = ocov.covariance(np.array([[2.0], [0.0]]), np.array([[1.0], [3.0]]))
    assert C.shape == (1, 1) and C[0, 0] == pytest.approx(0.28125, rel=1e-15)


def test_covariance_properties():
    rng = np.random.default_rng(5)
    W = rng.uniform(0.5, 2.0, (40, 30))
    N = rng.normal(0, 1, (40, 30))
    W[:, 7] = 0.0                      # an empty bin
    N[:, 7] = 0.0
    C = ocov.covariance(N, W)
    np.testing.assert_allclose(C, C.T, rtol=1e-13, atol=1e-15)
    assert np.all(C[7] == 0) and np.all(C[:, 7] == 0)
    assert np.linalg.eigvalsh(C).min() > -1e-12 * np.abs(C).max()
    # one sub-sample: no scatter
    assert np.abs(ocov.covariance(N[:1], W[:1])).max() < 1e-28
    # sub-samples with identical xi: no scatter
    C0 = ocov.covariance(W * 0.3, W)
    assert np.abs(C0).max() < 1e-15


def test_subsample_sums_add_up(cat0, bins0):
    pr = pairs.forest_pairs(cat0, bins0)
    s = ocov.subsample_sums(cat0, bins0, 64, pr)
    full = oxi.xi_sums(cat0, bins0, pr)
    assert np.count_nonzero(s["wsum"].sum(axis=1)) > 1
    np.testing.assert_allclose(s["wsum"].sum(axis=0), full["wsum"], rtol=1e-12)
    np.testing.assert_allclose(s["num"].sum(axis=0), full["num"], rtol=1e-10, atol=1e-9)
