"""The allocation-free sort entry point (gs_sort_pairs_noalloc) against the
context-based gs_sort_pairs, through the C ABI, on two calls in a row.

This file is named so that pytest collects it last: a run that stops at the
first failure has already run every other test. It also passes on its own in
a fresh process."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _keys(rng, n, bits):
    k = rng.integers(0, 2 ** 62, n, dtype=np.int64).view(np.uint64)
    k &= np.uint64((1 << bits) - 1)
    k[: n // 4] &= np.uint64(0xFFF)  # duplicates, so stability is exercised
    return k


def test_noalloc_sort_matches_context_sort():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_15951_gb300 import build
    build.build()
    import paper_2607_15951_gb300 as gs
    from paper_2607_15951_gb300 import _native as N

    lib = N.load()
    ctx = gs.Context(0)
    rng = np.random.default_rng(2024)
    stream = torch.cuda.current_stream().cuda_stream
    # Calls in a row: each must not see the previous call's leftovers. An odd
    # number of 8-bit passes (17 bits: 3, 40 bits: 5) leaves the result in the
    # library's array, from where it is copied back; an even number (45 bits:
    # 6, 64 bits: 8) leaves it in the caller's buffers. The last case fills
    # the array to its stated maximum.
    for n, bits in [(200_003, 45), (5_001, 64), (131_071, 17), (77_777, 40),
                    (N.NOALLOC_SORT_MAX_PAIRS, 64)]:
        keys = _keys(rng, n, bits)
        vals = rng.permutation(n).astype(np.uint32)
        k_ref = torch.from_numpy(keys.view(np.int64)).cuda()
        v_ref = torch.from_numpy(vals.view(np.int32)).cuda()
        k_new, v_new = k_ref.clone(), v_ref.clone()
        gs.gs_sort_pairs(ctx, k_ref, v_ref, n, bits)
        st = lib.gs_sort_pairs_noalloc(ctypes.c_void_p(k_new.data_ptr()),
                                       ctypes.c_void_p(v_new.data_ptr()), n, bits,
                                       ctypes.c_void_p(stream))
        assert st == N.GS_OK
        torch.cuda.synchronize()
        gs.gs_sync_status(ctx)
        # Integer results: the tolerance is exact equality.
        assert torch.equal(k_new, k_ref)
        assert torch.equal(v_new, v_ref)
        order = np.argsort(keys, kind="stable")
        assert np.array_equal(k_new.cpu().numpy().view(np.uint64), keys[order])
    # Above the stated maximum the call is refused before any launch.
    big = N.NOALLOC_SORT_MAX_PAIRS + 1
    st = lib.gs_sort_pairs_noalloc(ctypes.c_void_p(k_new.data_ptr()),
                                   ctypes.c_void_p(v_new.data_ptr()), big, 45,
                                   ctypes.c_void_p(stream))
    assert st == N.GS_ERR_CAPACITY
    ctx.close()
