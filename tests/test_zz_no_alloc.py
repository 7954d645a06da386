"""The allocation-free sort entry point (drk_sort_pairs_static).

It serves callers that cannot allocate device memory while they sort, e.g.
code recording a CUDA graph that must not contain allocation nodes: its
working memory is a fixed array inside the library.  Here it must give
exactly what drk_sort_pairs (which allocates from the context's pool)
gives, twice in a row on the shared array, and refuse sizes above its
limit before launching anything.  This file is collected last so that a
run stopping at the first failure has run every other test first.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MAX_PAIRS = 1 << 20


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


def test_static_sort_matches_pool_sort_twice(drk):
    for n, bits, seed in ((MAX_PAIRS, 32, 11), (123457, 20, 12)):
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


def test_static_sort_rejects_too_many_pairs(drk):
    k = torch.zeros(MAX_PAIRS + 1, dtype=torch.int32, device="cuda")
    v = torch.zeros_like(k)
    with pytest.raises(drk.DrkError) as e:
        drk.drk_sort_pairs_static(k, v, 32)
    assert e.value.code == 4          # DRK_ERR_CAPACITY, nothing launched
