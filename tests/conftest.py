import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")
    config.addinivalue_line("markers", "slow: larger CPU case")


from paper_2507_00129_gb300 import synth  # noqa: E402


def line_catalog(forests, region_deg=0.2, seed=0):
    """Small catalogue from explicit per-forest (ra, dec, dist, loglam, delta, weight)."""
    ra = np.array([f[0] for f in forests], dtype=np.float64)
    dec = np.array([f[1] for f in forests], dtype=np.float64)
    lens = [len(f[2]) for f in forests]
    offs = np.zeros(len(forests) + 1, dtype=np.int64)
    np.cumsum(lens, out=offs[1:])
    cat_ = lambda k, dt: np.concatenate([np.asarray(f[k], dtype=dt) for f in forests]) \
        if sum(lens) else np.zeros(0, dt)
    return synth.Catalog(ra=ra, dec=dec, offsets=offs, dist=cat_(2, np.float64),
                         loglam=cat_(3, np.float64), delta=cat_(4, np.float32),
                         weight=cat_(5, np.float32), name="hand")


def random_small(n_forests=12, max_len=8, patch_deg=0.05, seed=0, d0=1000.0, spread=30.0,
                 zero_weight_forest=False, single_pixel_forest=False):
    """Tiny random catalogue in a small patch (for O(n^4) checks)."""
    rng = np.random.default_rng(seed)
    forests = []
    for f in range(n_forests):
        n = int(rng.integers(2, max_len + 1))
        if single_pixel_forest and f == 1:
            n = 1
        d = np.sort(d0 + rng.uniform(0, spread, n))
        d = d + np.arange(n) * 1e-3  # strictly increasing
        L = np.log(3600.0 + rng.uniform(0, 400, n))
        L.sort()
        w = rng.uniform(0.5, 2.0, n)
        if zero_weight_forest and f == 2:
            w = np.zeros(n)
        forests.append((rng.uniform(0, np.radians(patch_deg)), rng.uniform(0, np.radians(patch_deg)),
                        d, L, rng.normal(0, 0.3, n), w))
    return line_catalog(forests)


@pytest.fixture(scope="session")
def cat0():
    return synth.make(0)


@pytest.fixture(scope="session")
def bins0():
    return synth.bins_for(0)
