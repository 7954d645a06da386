"""The allocation-free sort entry point (drk_sort_pairs_static).

It serves callers that cannot allocate device memory while they sort: an
embedder whose device memory is fixed at start-up, a loop that must not
meet an allocation's latency or implicit synchronisation, or code inside
an allocator's own bookkeeping.  Its working memory is a fixed array inside
the library.  Here it must give exactly what drk_sort_pairs (which
allocates from the context's pool) gives, twice in a row on the shared
array, and refuse bad arguments and sizes above its limit before launching
anything.  This file is collected last so that a run stopping at the first
failure has run every other test first.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MAX_PAIRS = 1 << 20
INVALID_ARG, CAPACITY = 1, 4


@pytest.fixture(scope="module")
def drk():
    from paper_2412_11752_gb300 import drk as D
    D.lib()
    return D


def _pairs(n, bits, seed):
    rng = np.random.default_rng(seed)
    keys = rng.integers(0, 2 ** bits, size=n, dtype=np.uint64).astype(np.uint32)
    keys[: n // 4] = keys[0]          # long runs of equal keys: stability is visible
    vals = rng.permutation(n).astype(np.uint32)
    k = torch.from_numpy(keys.view(np.int32).copy()).cuda()
    v = torch.from_numpy(vals.view(np.int32).copy()).cuda()
    return k, v


def _raw_call(drk, k, v, n, bits):
    """The C entry point itself (no wrapper checks), on the current stream."""
    return drk.lib().drk_sort_pairs_static(C.c_void_p(k.data_ptr()), C.c_void_p(v.data_ptr()), n, bits,
                                           C.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_static_sort_matches_pool_sort_twice(drk):
    # two calls in a row on the shared array, then an 8-bit (one pass) sort
    for n, bits, seed in ((MAX_PAIRS, 32, 11), (123457, 20, 12), (5000, 8, 13)):
        k1, v1 = _pairs(n, bits, seed)
        k0, v0 = k1.cpu().numpy().view(np.uint32), v1.cpu().numpy().view(np.uint32)
        k2, v2 = k1.clone(), v1.clone()
        drk.drk_sort_pairs(k1, v1, bits)
        drk.drk_sort_pairs_static(k2, v2, bits)
        torch.cuda.synchronize()
        assert torch.equal(k1, k2) and torch.equal(v1, v2), (n, bits)
        # and both are the stable order
        order = np.argsort(k0, kind="stable")
        assert np.array_equal(k2.cpu().numpy().view(np.uint32), k0[order])
        assert np.array_equal(v2.cpu().numpy().view(np.uint32), v0[order])


def test_static_sort_trivial_sizes(drk):
    for n in (0, 1):
        k, v = _pairs(max(n, 1), 32, 14)
        k0, v0 = k.clone(), v.clone()
        drk.drk_sort_pairs_static(k[:n], v[:n], 32)
        torch.cuda.synchronize()
        assert torch.equal(k, k0) and torch.equal(v, v0)


def test_static_sort_rejects_bad_arguments(drk):
    k = torch.zeros(MAX_PAIRS + 1, dtype=torch.int32, device="cuda")
    v = torch.zeros_like(k)
    with pytest.raises(drk.DrkError) as e:
        drk.drk_sort_pairs_static(k, v, 32)
    assert e.value.code == CAPACITY          # nothing launched
    for bits in (0, 33):
        assert _raw_call(drk, k, v, 16, bits) == INVALID_ARG
        assert b"key_bits" in drk.lib().drk_last_error()
    # a pinned host array: refused before any launch (the kernel never sees it)
    hk = torch.zeros(64, dtype=torch.int32).pin_memory()
    hv = torch.zeros_like(hk).pin_memory()
    assert _raw_call(drk, hk, hv, 64, 32) == INVALID_ARG
    assert b"not device memory" in drk.lib().drk_last_error()
    assert _raw_call(drk, k, hv, 64, 32) == INVALID_ARG
    torch.cuda.synchronize()
