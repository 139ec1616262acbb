"""tqp_filter_noalloc: the filter for callers that cannot allocate a device
workspace (a host program whose memory manager owns every device
allocation, or code where allocating is not allowed or could stall).  Its
scratch is a fixed array inside the library, so it is checked here against
the regular tqp_filter, on two calls in a row: the second, smaller call
must not be disturbed by what the first one left in the shared array.
This file is collected last so that a run stopping at its first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_filter_noalloc_matches_filter_on_two_calls():
    from paper_2209_04579_b300 import build
    build.build()
    from paper_2209_04579_b300 import tqp
    lib = tqp._lib
    rng = np.random.default_rng(2026)
    cases = [
        (3_000_017, [np.int32, np.int8], [(0, tqp.LE, 2400), (1, tqp.NE, 3)]),
        (50_003, [np.int64, np.int16], [(0, tqp.GT, -7), (1, tqp.LT, 100)]),
    ]
    for n, dts, preds in cases:
        cols = [torch.from_numpy(rng.integers(-200, 2600, n).astype(dt)).cuda() for dt in dts]
        want, want_n = tqp.tqp_filter(cols, preds)
        out = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        cnt = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        st = lib.tqp_filter_noalloc(tqp._cols(cols), len(cols), tqp._preds(preds), len(preds), n, None,
                                    ctypes.c_void_p(out.data_ptr()), n, ctypes.c_void_p(cnt.data_ptr()),
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == tqp.OK
        k = int(want_n.item())
        assert int(cnt.item()) == k
        assert torch.equal(out[:k], want[:k])
    assert tqp.tqp_status_poll() == tqp.OK
    # beyond the fixed scratch: rejected before any work
    cols = [torch.zeros(16, dtype=torch.int32, device="cuda")]
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = lib.tqp_filter_noalloc(tqp._cols(cols), 1, tqp._preds([(0, tqp.LT, 1)]), 1, tqp.NOALLOC_MAX_ROWS + 1,
                                None, None, 0, ctypes.c_void_p(cnt.data_ptr()), None)
    assert st == tqp.ERR_TOO_LARGE


def test_filter_noalloc_device_count_through_binding():
    """The Python wrapper with a device-resident row count d_n below n: only
    the first *d_n rows are filtered, exactly as by tqp_filter given the same
    d_n, again on two calls in a row."""
    from paper_2209_04579_b300 import build
    build.build()
    from paper_2209_04579_b300 import tqp
    rng = np.random.default_rng(77)
    n = 1_000_003
    col = torch.from_numpy(rng.integers(0, 1000, n).astype(np.int32)).cuda()
    for used in (654_321, 4_097):
        d_n = torch.tensor([used], dtype=torch.int64, device="cuda")
        want, want_n = tqp.tqp_filter([col], [(0, tqp.LT, 500)], d_n=d_n)
        got, got_n = tqp.tqp_filter_noalloc([col], [(0, tqp.LT, 500)], d_n=d_n)
        k = int(want_n.item())
        assert int(got_n.item()) == k
        assert k == int((col[:used] < 500).sum().item())
        assert torch.equal(got[:k], want[:k])
    assert tqp.tqp_status_poll() == tqp.OK
