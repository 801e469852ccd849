"""The seeded input generator: cosmology closed forms and catalogue shape."""
import math

import numpy as np
import pytest

from paper_2507_00129_gb300 import synth


def test_distance_einstein_de_sitter_closed_form():
    z = np.array([0.5, 1.96, 2.5, 3.44])
    d = synth.comoving_distance(z, omega_m=1.0)
    np.testing.assert_allclose(d, 2 * synth.C_OVER_H0 * (1 - 1 / np.sqrt(1 + z)), rtol=1e-14)


def test_distance_empty_universe_is_linear():
    z = np.array([0.1, 2.0, 3.5])
    np.testing.assert_allclose(synth.comoving_distance(z, omega_m=0.0), synth.C_OVER_H0 * z, rtol=1e-14)


@pytest.mark.parametrize("cfg", [0, 3])
def test_catalogue_shape(cfg):
    cat = synth.make(cfg, n_forests=300)
    L = cat.lengths()
    assert cat.offsets[0] == 0 and cat.offsets[-1] == cat.n_pix
    for f in range(0, cat.n_forests, 17):
        d = cat.dist[cat.forest(f)]
        assert np.all(np.diff(d) > 0)
    lam = np.exp(cat.loglam)
    assert lam.min() > 3600.0
    assert np.all(cat.weight > 0)
    if cfg == 0:
        assert 40 <= L.min() and L.max() <= 210
    else:
        assert L.min() >= 100 and L.max() <= 600
    again = synth.make(cfg, n_forests=300)
    np.testing.assert_array_equal(cat.delta, again.delta)


def test_cap_area():
    th = synth.cap_half_angle_deg(2500.0)
    area = 2 * math.pi * (1 - math.cos(math.radians(th))) * (180 / math.pi) ** 2
    assert area == pytest.approx(2500.0)
