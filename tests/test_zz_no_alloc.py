"""lya_xi_pairs_static: the allocation-free variant of lya_xi_pairs.

Some callers cannot allocate device memory at run time (a device under
global-mode graph capture, memory owned by a pool allocator, real-time
pipelines); this entry point keeps its scratch in a fixed device array of the
library.  Its results must match lya_xi_pairs on the same pairs, on two calls
in a row (the second call must not see the first call's leftovers).  The file
is named so that pytest collects it last.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2507_00129_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_00129_gb300 import build, api as _api
    build.build()
    return _api


def test_static_scratch_matches_allocating_entry_point(api):
    cat = synth.make(0)
    bins = synth.bins_for(0)
    a, b = oracle.pairs.forest_pairs(cat, bins)
    dc = api.DeviceCatalog.from_host(cat)
    rng = np.random.default_rng(21)
    first = rng.choice(len(a), 6000, replace=False)
    second = rng.choice(len(a), 2500, replace=False)
    with api.Handle() as h:
        for sel in (first, second):
            pa = torch.from_numpy(a[sel]).cuda()
            pb = torch.from_numpy(b[sel]).cuda()
            n_ref, w_ref, x_ref = api.lya_xi_pairs(h, dc, bins, pa, pb, "mixed")
            n_s, w_s, x_s = api.lya_xi_pairs_static(dc, bins, pa, pb)
            W, Wr = w_s.cpu().numpy(), w_ref.cpu().numpy()
            assert Wr.sum() > 0
            # the mixed-path tolerance of the parity tests: 1e-6 relative on W
            np.testing.assert_allclose(W, Wr, rtol=1e-6, atol=1e-9)
            N, Nr = n_s.cpu().numpy(), n_ref.cpu().numpy()
            np.testing.assert_allclose(N, Nr, rtol=1e-6, atol=1e-6 * np.abs(Nr).max())
            X, Xr = x_s.cpu().numpy(), x_ref.cpu().numpy()
            np.testing.assert_allclose(X, Xr, rtol=1e-5, atol=1e-12)


def test_static_scratch_rejects_oversize(api):
    from paper_2507_00129_gb300._lib import LyaError
    cat = synth.make(0)
    dc = api.DeviceCatalog.from_host(cat)
    n = (1 << 20) + 1
    z = torch.zeros(n, dtype=torch.int32, device="cuda")
    with pytest.raises(LyaError) as e:
        api.lya_xi_pairs_static(dc, synth.bins_for(0), z, z)
    assert e.value.code == -8
