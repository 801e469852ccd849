"""Degenerate inputs of the extension entry points (lya_xcf, lya_xdmat,
lya_xi1d, lya_xi_bin_means) against the oracle, and their refusal inside a
graph capture."""
import numpy as np
import pytest
import torch

import oracle
from conftest import line_catalog
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


def _degenerate():
    # single-pixel forests, a zero-weight forest, an empty forest, an isolated forest
    fs = [(0.0, 0.0, [1000.0], [8.2], [0.5], [1.0]),
          (1e-4, 0.0, [1001.0], [8.2], [-0.5], [2.0]),
          (2e-4, 0.0, [1000.5, 1002.0], [8.2, 8.3], [0.1, 0.2], [0.0, 0.0]),
          (3e-4, 0.0, [], [], [], []),
          (1.0, 0.5, [1000.0, 1003.0, 1009.0], [8.2, 8.3, 8.4], [0.3, 0.1, -0.2], [1.0, 2.0, 1.5])]
    return line_catalog(fs)


def _quasars(ra, dec, dist, w):
    return synth.Quasars(ra=np.asarray(ra, float), dec=np.asarray(dec, float), dist=np.asarray(dist, float),
                         weight=np.asarray(w, np.float32), z=np.zeros(len(ra)))


def test_xcf_degenerate_inputs(api, handle):
    cat = _degenerate()
    q = _quasars([5e-5, 1.0, 2.0], [0.0, 0.5, 0.0], [1004.3, 1002.0, 1000.0], [1.0, 0.5, 2.0])
    bins = synth.Bins(8, 4, 16.0, 16.0)
    dc, dq = api.DeviceCatalog.from_host(cat), api.DeviceQuasars.from_host(q)
    num, wsum, xi = api.lya_xcf(handle, dc, dq, bins)
    api.lya_sync_status(handle)
    ref = oracle.xcf.xcf_sums(cat, q, bins, eps_edge=6e-5)
    assert ref["count"].sum() > 0
    np.testing.assert_allclose(_np(wsum), ref["wsum"], rtol=1e-6, atol=1e-12)
    np.testing.assert_allclose(_np(num), ref["num"], rtol=1e-5, atol=1e-12)
    D, W = api.lya_xdmat(handle, dc, dq, bins, 1.0, 0)
    rd = oracle.xcf.xdmat(cat, q, bins, oracle.xcf.forest_quasar_pairs(cat, q, bins))
    np.testing.assert_allclose(_np(D), rd["dmat"], rtol=1e-5, atol=1e-6)
    # no quasars at all: zero sums, zero D
    none = _quasars([], [], [], [])
    num0, wsum0, xi0 = api.lya_xcf(handle, dc, api.DeviceQuasars.from_host(none), bins)
    assert float(wsum0.abs().sum()) == 0 and float(xi0.abs().sum()) == 0
    D0, W0 = api.lya_xdmat(handle, dc, api.DeviceQuasars.from_host(none), bins, 1.0, 0)
    assert float(D0.abs().sum()) == 0 and float(W0.abs().sum()) == 0


def test_xi1d_and_means_degenerate_inputs(api, handle):
    cat = _degenerate()
    dc = api.DeviceCatalog.from_host(cat)
    num, wsum, xi = api.lya_xi1d(handle, dc, 4, 12.0)
    ref = oracle.xi1d.xi1d_sums(cat, 4, 12.0)
    assert ref["count"].sum() == 3 + 1    # the isolated forest's 3 pairs, the zero-weight forest's 1
    np.testing.assert_allclose(_np(wsum), ref["wsum"], rtol=1e-12)
    np.testing.assert_allclose(_np(num), ref["num"], rtol=1e-12, atol=1e-15)
    bins = synth.Bins(4, 4, 16.0, 16.0)
    out = api.lya_xi_bin_means(handle, dc, bins)
    api.lya_sync_status(handle)
    rm = oracle.xi.bin_means(cat, bins, oracle.pairs.all_pairs(cat.n_forests))
    np.testing.assert_array_equal(_np(out["count"]), rm["count"])
    np.testing.assert_allclose(_np(out["wsum"]), rm["wsum"], rtol=1e-6, atol=1e-12)
    on = rm["wsum"] > 0
    np.testing.assert_allclose(_np(out["rpar_mean"])[on], rm["rpar_mean"][on], rtol=1e-5, atol=1e-5)
    # one forest: no pairs
    one = line_catalog([(0.0, 0.0, [1000.0, 1001.0], [8.2, 8.3], [0.5, 0.1], [1.0, 1.0])])
    out1 = api.lya_xi_bin_means(handle, api.DeviceCatalog.from_host(one), bins)
    assert int(out1["count"].sum()) == 0 and float(out1["rpar_mean"].abs().sum()) == 0


def test_extension_calls_are_refused_during_capture(api):
    from paper_2507_00129_gb300._lib import LyaError
    cat = synth.make(0, n_forests=30)
    spec = synth.spec_for(0, n_forests=30)
    q, own = synth.quasars(spec, cat)
    bins = synth.bins_for(0)
    dc, dq = api.DeviceCatalog.from_host(cat), api.DeviceQuasars.from_host(q)
    h = api.Handle()
    s = torch.cuda.Stream()
    try:
        with torch.cuda.stream(s):
            api.lya_xi(h, dc, bins, "mixed", stream=s)
            api.lya_sync_status(h, s)
            calls = (lambda: api.lya_xcf(h, dc, dq, bins, stream=s),
                     lambda: api.lya_xdmat(h, dc, dq, bins, 1.0, 0, stream=s),
                     lambda: api.lya_xi1d(h, dc, 10, 50.0, stream=s),
                     lambda: api.lya_xi_bin_means(h, dc, bins, stream=s))
            for call in calls:      # outside a capture first (the binding's output tensors come from the cache)
                call()
            api.lya_sync_status(h, s)
            for call in calls:
                api.lya_capture_begin(h, s)
                with pytest.raises(LyaError):
                    call()
                with pytest.raises(LyaError):
                    api.lya_capture_end(h)
            # the handle still works
            num, wsum, _ = api.lya_xcf(h, dc, dq, bins, forest_qso=own, stream=s)
            assert float(wsum.sum()) > 0
    finally:
        h.close()
