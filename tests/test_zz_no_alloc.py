"""lya_xi_pairs_static: the allocation-free variant of lya_xi_pairs.

Some callers cannot allocate device memory at run time (a device under
global-mode graph capture, memory owned by a pool allocator, real-time
pipelines); this entry point keeps its scratch in a fixed device array of the
library.  Its results must match the CPU FP64 oracle on the same pairs, within
the mixed path's tolerance, on two calls in a row (the second call must not see
the first call's leftovers), and a call must not change the device's free
memory.  The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2507_00129_gb300 import synth

pytestmark = pytest.mark.gpu

EPS_EDGE = 6e-5   # FP32 error bound of the mixed path's scaled separations, in bin units


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_00129_gb300 import build, api as _api
    build.build()
    return _api


def _check_against_oracle(cat, bins, a, b, num, wsum, xi):
    ref = oracle.xi.xi_sums(cat, bins, (a, b), eps_edge=EPS_EDGE)
    W, N, X = (t.cpu().numpy() for t in (wsum, num, xi))
    assert ref["wsum"].sum() > 0
    # W: 1e-6 relative plus the weight of pixel pairs within eps of an edge
    assert np.all(np.abs(W - ref["wsum"]) <= 1e-6 * ref["wsum"] + ref["edge_w"] + 1e-9)
    assert np.all(np.abs(N - ref["num"]) <= 1e-5 * np.sqrt(ref["num_sq"]) + ref["edge_n"] + 1e-9)
    on = ref["wsum"] > 0
    # xi = N / W: edge flips move it by (dN - xi dW) / (W + dW), at most (E^N + |xi| E^W) / (W - E^W)
    den = ref["wsum"] - ref["edge_w"]
    allow = (1e-5 * np.maximum(np.abs(ref["xi"]), ref["sigma"])
             + np.divide(ref["edge_n"] + np.abs(ref["xi"]) * ref["edge_w"], den, out=np.full_like(den, np.inf),
                         where=den > 0))
    assert np.all(np.abs(X - ref["xi"])[on] <= allow[on] + 1e-15)
    assert np.all(X[~on] == 0)


def test_static_scratch_matches_oracle_on_two_calls(api):
    cat = synth.make(0)
    bins = synth.bins_for(0)
    a, b = oracle.pairs.forest_pairs(cat, bins)
    dc = api.DeviceCatalog.from_host(cat)
    rng = np.random.default_rng(21)
    first = np.sort(rng.choice(len(a), 3000, replace=False))
    second = np.sort(rng.choice(len(a), 1200, replace=False))
    for sel in (first, second):
        pa = torch.from_numpy(a[sel]).cuda()
        pb = torch.from_numpy(b[sel]).cuda()
        num, wsum, xi = api.lya_xi_pairs_static(dc, bins, pa, pb)
        _check_against_oracle(cat, bins, a[sel], b[sel], num, wsum, xi)


def test_static_call_allocates_no_device_memory(api):
    """After a first call (lazy module loading, symbol lookup), a second call
    with caller-owned outputs leaves the device's free memory unchanged."""
    from paper_2507_00129_gb300 import _lib
    cat = synth.make(0)
    bins = synth.bins_for(0)
    a, b = oracle.pairs.forest_pairs(cat, bins)
    dc = api.DeviceCatalog.from_host(cat)
    # the C ABI takes int32 forest indices
    pa = torch.from_numpy(a[:2000]).to(torch.int32).cuda()
    pb = torch.from_numpy(b[:2000]).to(torch.int32).cuda()
    nb = bins.nbins
    out = [torch.empty(nb, dtype=torch.float64, device="cuda") for _ in range(3)]
    c, bb = dc.c(), api.c_bins(bins)
    lib = _lib.load()

    def call():
        return lib.lya_xi_pairs_static(ctypes.byref(c), ctypes.byref(bb), pa.data_ptr(), pb.data_ptr(),
                                       int(pa.numel()), out[0].data_ptr(), out[1].data_ptr(),
                                       out[2].data_ptr(), None)

    assert call() == _lib.LYA_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    assert call() == _lib.LYA_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    _check_against_oracle(cat, bins, a[:2000], b[:2000], out[0], out[1], out[2])


def test_static_scratch_rejects_bad_arguments_before_gpu_work(api):
    from paper_2507_00129_gb300._lib import LyaError
    cat = synth.make(0)
    dc = api.DeviceCatalog.from_host(cat)
    z = torch.zeros(4, dtype=torch.int32, device="cuda")
    n = (1 << 20) + 1
    big = torch.zeros(n, dtype=torch.int32, device="cuda")
    with pytest.raises(LyaError) as e:
        api.lya_xi_pairs_static(dc, synth.bins_for(0), big, big)
    assert e.value.code == -8
    # n_par above the mixed pair kernel's limit of 203
    with pytest.raises(LyaError) as e:
        api.lya_xi_pairs_static(dc, synth.Bins(204, 4, 100.0, 100.0), z, z)
    assert e.value.code == -8
    # a non-finite range
    with pytest.raises(LyaError) as e:
        api.lya_xi_pairs_static(dc, synth.Bins(25, 25, float("inf"), 100.0), z, z)
    assert e.value.code == -1
    # the entry point still works afterwards
    bins = synth.bins_for(0)
    a, b = oracle.pairs.forest_pairs(cat, bins)
    num, wsum, xi = api.lya_xi_pairs_static(dc, bins, torch.from_numpy(a[:500]).cuda(),
                                            torch.from_numpy(b[:500]).cuda())
    _check_against_oracle(cat, bins, a[:500], b[:500], num, wsum, xi)
