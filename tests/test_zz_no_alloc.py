"""The allocation-free sort entry point (gs_sort_pairs_u32_noalloc).

It exists for callers that cannot allocate device memory: plug-ins whose
host framework owns every byte of device memory, code under a fixed
device-memory budget, and loops that cannot afford cudaMalloc's implicit
device synchronisation.  These tests call it through the C ABI and check that it
returns exactly what the scratch-taking gs_sort_pairs_u32 returns, and the
stable sort by the key bits, on two calls in a row (the second call reuses
the static scratch the first one left behind), and that it refuses sizes
beyond its stated maximum.

The file is named so pytest collects it last.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _sort_with_scratch(lib, keys, vals, begin, end):
    kt = torch.from_numpy(keys.view(np.int32)).cuda()
    vt = torch.from_numpy(vals.view(np.int32)).cuda()
    ko, vo = torch.empty_like(kt), torch.empty_like(vt)
    scratch = torch.empty(int(lib.gs_sort_scratch_bytes(keys.size)), dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert lib.gs_sort_pairs_u32(kt.data_ptr(), vt.data_ptr(), ko.data_ptr(), vo.data_ptr(), keys.size,
                                 begin, end, scratch.data_ptr(), s) == 0
    torch.cuda.synchronize()
    return ko.cpu().numpy().view(np.uint32), vo.cpu().numpy().view(np.uint32)


def _sort_noalloc(lib, keys, vals, begin, end):
    kt = torch.from_numpy(keys.view(np.int32)).cuda()
    vt = torch.from_numpy(vals.view(np.int32)).cuda()
    ko, vo = torch.empty_like(kt), torch.empty_like(vt)
    s = torch.cuda.current_stream().cuda_stream
    assert lib.gs_sort_pairs_u32_noalloc(kt.data_ptr(), vt.data_ptr(), ko.data_ptr(), vo.data_ptr(), keys.size,
                                         begin, end, s) == 0
    torch.cuda.synchronize()
    return ko.cpu().numpy().view(np.uint32), vo.cpu().numpy().view(np.uint32)


def test_noalloc_sort_matches_the_scratch_sort_on_two_calls():
    from paper_2601_19489_gb300 import _lib

    lib = _lib.load()
    # two calls in a row with different sizes, bit ranges and key patterns
    for call, (n, begin, end) in enumerate([(300007, 0, 32), (70001, 4, 17)]):
        rng = np.random.default_rng(1234 + call)
        keys = rng.integers(0, 1 << 32, size=n, dtype=np.uint64).astype(np.uint32)
        keys[: n // 4] = keys[7]  # a long run of equal keys exercises stability
        vals = np.arange(n, dtype=np.uint32)
        want_k, want_v = _sort_with_scratch(lib, keys, vals, begin, end)
        got_k, got_v = _sort_noalloc(lib, keys, vals, begin, end)
        np.testing.assert_array_equal(got_k, want_k)
        np.testing.assert_array_equal(got_v, want_v)
        # and both are the stable sort by the key bits [begin, end)
        digit = (keys.astype(np.uint64) >> np.uint64(begin)) & np.uint64((1 << (end - begin)) - 1)
        order = np.argsort(digit, kind="stable")
        np.testing.assert_array_equal(got_v, vals[order])
        np.testing.assert_array_equal(got_k, keys[order])


def test_noalloc_sort_refuses_sizes_beyond_its_maximum():
    from paper_2601_19489_gb300 import _lib

    lib = _lib.load()
    # rejected on the host before anything is enqueued, so no buffers are needed
    assert lib.gs_sort_pairs_u32_noalloc(None, None, None, None, 1 << 31, 0, 32, None) == _lib.GS_ERR_ARG
    assert lib.gs_sort_pairs_u32_noalloc(None, None, None, None, 0, 0, 32, None) == 0
