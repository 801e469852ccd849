"""Three-point estimator (lya_xi3) against the oracle (oracle.xi3).

Tolerance: |dW_A| <= 1e-6 W_A + E^W_A and |dN_A| <= 1e-5 sqrt(sum t^2) + E^N_A,
E the oracle's edge mass for records within eps of a bin edge: eps_r = 1e-9
bin units (the library bins |r| in FP64), eps_c = 2e-6 in cos theta and
cos alpha (cos alpha is FP32 in the library: three roundings of unit-scale
products)."""
import numpy as np
import pytest
import torch

from oracle import xi3 as ox3
from paper_2507_00129_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_00129_gb300 import build, api as _api
    build.build()
    return _api


@pytest.fixture(scope="module")
def handle(api):
    h = api.Handle()
    yield h
    h.close()


def _np(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("nf,box,rmax", [(14, 0.3, 15.0), (24, 0.5, 20.0)])
def test_xi3_matches_oracle(api, handle, nf, box, rmax):
    spec = synth.Spec(n_forests=nf, seed=8, region="box", box_deg=box, grid="log10", delta_sigma=0.2)
    cat = synth.generate(spec)
    g = ox3.Grid3(n_r=5, n_theta=10, n_alpha=20, r_max=rmax)
    num, wsum, xi = api.lya_xi3(handle, api.DeviceCatalog.from_host(cat), g)
    api.lya_sync_status(handle)
    ref = ox3.xi3_sums(cat, g, eps_r=1e-9, eps_c=2e-6)
    W, N = _np(wsum), _np(num)
    assert ref["count"].sum() > 1e6
    assert np.all(np.abs(W - ref["wsum"]) <= 1e-6 * ref["wsum"] + ref["edge_w"] + 1e-9)
    assert np.all(np.abs(N - ref["num"]) <= 1e-5 * np.sqrt(ref["num_sq"]) + ref["edge_n"] + 1e-12)
    # mirror symmetry of the grid (sides swapped) holds exactly
    Wr = W.reshape(g.n_r, g.n_r, g.n_alpha, g.n_theta, g.n_theta)
    np.testing.assert_array_equal(Wr, Wr.transpose(1, 0, 2, 4, 3))
    on = ref["wsum"] > 0
    np.testing.assert_allclose(_np(xi)[~on], 0.0)


def test_xi3_unit_weights_count_records(api, handle):
    """With w = 1 the weight sum of a bin is its number of records."""
    spec = synth.Spec(n_forests=14, seed=8, region="box", box_deg=0.3, grid="log10", delta_sigma=0.2)
    cat = synth.generate(spec)
    cat.weight[:] = 1.0
    g = ox3.Grid3(n_r=5, n_theta=10, n_alpha=20, r_max=15.0)
    _, wsum, _ = api.lya_xi3(handle, api.DeviceCatalog.from_host(cat), g)
    ref = ox3.xi3_sums(cat, g, eps_r=1e-9, eps_c=2e-6)
    W = _np(wsum)
    assert np.all(np.abs(W - ref["count"]) <= ref["edge_w"] + 1e-9)
    assert abs(W.sum() - ref["count"].sum()) <= ref["edge_w"].sum() + 0.5


def test_xi3_argument_errors(api, handle):
    from paper_2507_00129_gb300._lib import LyaError
    cat = synth.subset(synth.make(0), np.arange(10))
    dc = api.DeviceCatalog.from_host(cat)
    with pytest.raises(LyaError) as e:
        api.lya_xi3(handle, dc, ox3.Grid3(n_r=0, n_theta=10, n_alpha=20, r_max=10.0))
    assert e.value.code == -8
    with pytest.raises(LyaError) as e:
        api.lya_xi3(handle, dc, ox3.Grid3(n_r=5, n_theta=10, n_alpha=20, r_max=-1.0))
    assert e.value.code == -1


def test_xi3_dense_forests_use_a_larger_capacity(api, handle):
    """DESI-like pixel density (0.57 Mpc/h spacing) at r_max = 40 Mpc/h puts
    thousands of pixels around a vertex; the call sizes its capacity to the
    largest list and counts every record: with unit weights the total weight
    equals, summed over vertices, (sum_f c_f)^2 - sum_f c_f^2, c_f the vertex's
    in-range pixels of forest f (ordered pairs from distinct forests)."""
    spec = synth.Spec(n_forests=80, seed=12, region="box", box_deg=0.8, grid="linear", delta_sigma=0.25,
                      length_range=(300, 600))
    cat = synth.generate(spec)
    cat.weight[:] = 1.0
    g = ox3.Grid3(n_r=10, n_theta=10, n_alpha=20, r_max=40.0)
    _, wsum, _ = api.lya_xi3(handle, api.DeviceCatalog.from_host(cat), g)
    api.lya_sync_status(handle)
    from oracle.geometry import unit_vectors
    n = unit_vectors(cat.ra, cat.dec)
    forest = np.repeat(np.arange(cat.n_forests), np.diff(cat.offsets))
    pos = cat.dist[:, None] * n[forest]
    total, most = 0.0, 0
    for i in range(cat.n_pix):
        d2 = np.einsum("ij,ij->i", pos - pos[i], pos - pos[i])
        m = (forest != forest[i]) & (d2 < 40.0 ** 2)
        c = np.bincount(forest[m], minlength=cat.n_forests).astype(np.float64)
        total += c.sum() ** 2 - (c * c).sum()
        most = max(most, int(m.sum()))
    assert most > 2200          # beyond three blocks' shared memory per SM
    W = _np(wsum)
    assert abs(W.sum() - total) <= 1e-9 * total + 10
    Wr = W.reshape(g.n_r, g.n_r, g.n_alpha, g.n_theta, g.n_theta)
    np.testing.assert_array_equal(Wr, Wr.transpose(1, 0, 2, 4, 3))
