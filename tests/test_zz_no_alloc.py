"""The allocation-free classify entry point against the ordinary one.

spdba_classify_static serves callers that cannot allocate device memory: its
scratch is a fixed array inside the library.  This file sorts last so that a
run stopping at the first failure has already run every other test.  It must
pass in a fresh process and after the other tests (the shared array then
holds an earlier call's contents, which the entry point must not depend on).
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _classify_both(nb, meas, tau, force_dc, transitions):
    import torch
    from paper_2609_03922_gb300 import spdba
    n = int(np.prod(nb))
    md = torch.from_numpy(meas.ravel().copy()).cuda()
    td = torch.tensor([tau], dtype=torch.float64, device="cuda")
    outs = []
    for static in (False, True):
        states = torch.full((n,), 7, dtype=torch.uint8, device="cuda")
        chi = torch.full((n,), 255, dtype=torch.uint8, device="cuda")
        lst = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        cnt = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        if static:
            # straight through the C ABI
            L = spdba.lib()
            dims = (ctypes.c_int64 * len(nb))(*nb)
            st = L.spdba_classify_static(len(nb), dims, md.data_ptr(), td.data_ptr(), force_dc, transitions,
                                         states.data_ptr(), chi.data_ptr(), lst.data_ptr(), cnt.data_ptr(),
                                         torch.cuda.current_stream().cuda_stream)
            assert st == spdba.SPDBA_OK, L.spdba_last_error()
        else:
            scratch = torch.empty(spdba.classify_scratch_bytes(n), dtype=torch.uint8, device="cuda")
            spdba.classify(nb, md, td, force_dc, transitions, states, chi, lst, cnt, scratch)
        torch.cuda.synchronize()
        c = int(cnt.item())
        outs.append((states.cpu().numpy(), chi.cpu().numpy(), lst.cpu().numpy()[:c], c))
    return outs


def _check_pair(a, b):
    assert a[3] == b[3]
    assert np.array_equal(a[0], b[0])
    trans = a[0] == 1
    assert np.array_equal(a[1][trans], b[1][trans])
    assert np.array_equal(a[2], b[2])


@pytest.mark.parametrize("force_dc", [0, 1])
@pytest.mark.parametrize("transitions", [0, 1])
@pytest.mark.parametrize("nb", [(32, 32, 32), (48, 48, 48)])
def test_static_classify_matches_allocating_classify_twice(nb, transitions, force_dc):
    r = np.random.default_rng(11 + 2 * transitions + force_dc)
    for call in range(2):   # two calls in a row: the second sees the first call's leftovers
        meas = np.exp(-8 * r.random(nb))
        tau = float(np.quantile(meas, 0.85 if call == 0 else 0.6))
        a, b = _classify_both(nb, meas, tau, force_dc, transitions)
        _check_pair(a, b)


def test_static_classify_at_exact_capacity():
    """A map of exactly 2^20 blocks (the largest the fixed array serves)."""
    nb = (128, 128, 64)
    r = np.random.default_rng(5)
    for call in range(2):
        meas = np.exp(-8 * r.random(nb))
        tau = float(np.quantile(meas, 0.9 if call == 0 else 0.5))
        a, b = _classify_both(nb, meas, tau, 1, 1)
        _check_pair(a, b)


def test_static_classify_rejects_oversized_maps():
    import torch
    from paper_2609_03922_gb300 import spdba
    nb = (129, 128, 64)   # 1,056,768 blocks > 2^20
    L = spdba.lib()
    dims = (ctypes.c_int64 * 3)(*nb)
    dummy = torch.empty(8, dtype=torch.float64, device="cuda")
    st = L.spdba_classify_static(3, dims, dummy.data_ptr(), dummy.data_ptr(), 1, 1, dummy.data_ptr(),
                                 dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(), None)
    assert st == spdba.SPDBA_ERR_UNSUPPORTED
    assert b"fixed capacity" in L.spdba_last_error()
