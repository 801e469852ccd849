"""CUDA-graph capture of a call sequence (lya_capture_begin / _end,
lya_graph_launch): a replay with new deltas equals the same calls run eagerly,
and the library refuses what a graph cannot do (synchronise, allocate, run on
freed buffers)."""
import numpy as np
import pytest
import torch

from paper_2507_00129_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_00129_gb300 import build, api as _api
    build.build()
    return _api


def _setup(api, n_forests=120):
    cat = synth.subset(synth.make(0), np.arange(n_forests))
    bins = synth.bins_for(0)
    dc = api.DeviceCatalog.from_host(cat)
    nb = bins.nbins
    o = {
        "dp": torch.empty_like(dc.delta),
        "num": torch.empty(nb, dtype=torch.float64, device="cuda"),
        "wsum": torch.empty(nb, dtype=torch.float64, device="cuda"),
        "xi": torch.empty(nb, dtype=torch.float64, device="cuda"),
        "gd": torch.empty_like(dc.delta),
        "gw": torch.empty_like(dc.weight),
        "D": torch.empty((nb, nb), dtype=torch.float64, device="cuda"),
        "Wd": torch.empty(nb, dtype=torch.float64, device="cuda"),
    }
    g = torch.from_numpy(np.random.default_rng(303).normal(size=nb)).cuda()
    return cat, bins, dc, o, g


def _calls(api, h, dc, bins, o, g, stream):
    dcp = dc.with_(delta=o["dp"])
    api.lya_project(h, dc, out=o["dp"], stream=stream)
    api.lya_xi(h, dcp, bins, "mixed", o["num"], o["wsum"], o["xi"], stream=stream)
    api.lya_xi_backward(h, dcp, bins, g, o["xi"], o["wsum"], stream=stream, grad_delta=o["gd"],
                        grad_weight=o["gw"])
    api.lya_dmat(h, dcp, bins, 1.0, 3, stream=stream, D=o["D"], W=o["Wd"])


def test_replay_equals_eager_with_new_deltas(api):
    cat, bins, dc, o, g = _setup(api)
    h = api.Handle()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        _calls(api, h, dc, bins, o, g, s)          # eager once: pair list, buffer sizes
        api.lya_sync_status(h, s)
        api.lya_capture_begin(h, s)
        _calls(api, h, dc, bins, o, g, s)
        graph = api.lya_capture_end(h)
        n0 = api.lya_kernel_launches()
        rng = np.random.default_rng(9)
        for rep in range(2):
            dc.delta.copy_(torch.from_numpy(rng.normal(0, 0.2, cat.n_pix).astype(np.float32)).cuda())
            graph.launch(s)
            api.lya_sync_status(h, s)
            got = {k: v.clone() for k, v in o.items()}
            _calls(api, h, dc, bins, o, g, s)
            api.lya_sync_status(h, s)
            np.testing.assert_array_equal(got["dp"].cpu().numpy(), o["dp"].cpu().numpy())
            for k in ("num", "wsum", "xi"):
                np.testing.assert_allclose(got[k].cpu().numpy(), o[k].cpu().numpy(), rtol=1e-9,
                                           atol=1e-12 * float(o[k].abs().max()))
            # D sums each chunk of pairs in FP32 in an order set by atomic
            # scatter, so two runs agree to the D tolerance, not bit for bit
            for k in ("D", "Wd"):
                np.testing.assert_allclose(got[k].cpu().numpy(), o[k].cpu().numpy(), rtol=1e-5,
                                           atol=1e-5 * float(o[k].abs().max()))
            for k in ("gd", "gw"):
                np.testing.assert_allclose(got[k].cpu().numpy(), o[k].cpu().numpy(), rtol=1e-5,
                                           atol=1e-6 * float(o[k].abs().max()))
        assert api.lya_kernel_launches() > n0
    graph.close()
    h.close()


def test_capture_refuses_sync_default_stream_and_stale_graph(api):
    from paper_2507_00129_gb300._lib import LyaError
    cat, bins, dc, o, g = _setup(api, n_forests=60)
    h = api.Handle()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        _calls(api, h, dc, bins, o, g, s)
        api.lya_sync_status(h, s)
        # the legacy default stream cannot be captured
        with pytest.raises(LyaError) as e:
            api.lya_capture_begin(h, torch.cuda.default_stream())
        assert e.value.code == -1
        # a synchronising call inside the capture fails, and so does the capture
        api.lya_capture_begin(h, s)
        with pytest.raises(LyaError):
            api.lya_sync_status(h, s)
        with pytest.raises(LyaError):
            api.lya_capture_end(h)
        # the handle works afterwards; capture again
        _calls(api, h, dc, bins, o, g, s)
        api.lya_sync_status(h, s)
        api.lya_capture_begin(h, s)
        _calls(api, h, dc, bins, o, g, s)
        graph = api.lya_capture_end(h)
        graph.launch(s)
        api.lya_sync_status(h, s)
        # a call on a larger catalogue reallocates the handle's buffers: the graph refuses to run
        big = synth.make(0)
        api.lya_xi(h, api.DeviceCatalog.from_host(big), bins, "mixed", stream=s)
        api.lya_sync_status(h, s)
        with pytest.raises(LyaError) as e:
            graph.launch(s)
        assert e.value.code == -1
        graph.close()
    h.close()
