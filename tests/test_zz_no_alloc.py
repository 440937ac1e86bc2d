"""The allocation-free sort entry point against the allocating one.

hm_radix_sort_pairs_noalloc exists for callers that cannot allocate device
memory while they run (a program whose free device memory belongs to its own
pool, a loop that must not block on an allocation). It must sort exactly like
hm_radix_sort_pairs. This file is collected last so that a run stopping at the
first failure has already run every other test; it also passes on its own in
a fresh process.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1708_09707_gb300 import build, hm
    build.build()
    return hm.lib()


def _sorted_both(L, keys, vals, bits):
    import torch
    ka = torch.from_numpy(keys.view(np.int64).copy()).cuda()
    va = torch.from_numpy(vals.view(np.int32).copy()).cuda()
    kb, vb = ka.clone(), va.clone()
    n = keys.size
    assert L.hm_radix_sort_pairs(ctypes.c_void_p(ka.data_ptr()), ctypes.c_void_p(va.data_ptr()),
                                 n, bits, None) == 0
    rc = L.hm_radix_sort_pairs_noalloc(ctypes.c_void_p(kb.data_ptr()),
                                       ctypes.c_void_p(vb.data_ptr()), n, bits, None)
    assert rc == 0, L.hm_last_error()
    torch.cuda.synchronize()
    return (ka.cpu().numpy().view(np.uint64), va.cpu().numpy().view(np.uint32),
            kb.cpu().numpy().view(np.uint64), vb.cpu().numpy().view(np.uint32))


def test_noalloc_sort_matches_allocating_sort_twice(lib):
    L = lib
    nmax = 262144
    rng = np.random.default_rng(13)
    # calls in a row: each one fills the shared scratch, the next must not
    # see anything of it (different size, ties, different key width)
    # keys are drawn over the full 64 bits, so the last radix pass sorts on
    # the top bits; one case sets the top bit of every other key, one is a
    # single pair
    cases = [(nmax, 64, False, False), (100003, 40, True, False), (77777, 64, False, True),
             (1, 64, False, True)]
    for n, bits, ties, high in cases:
        keys = rng.integers(0, 2 ** 64, size=n, dtype=np.uint64)
        if bits < 64:
            keys &= np.uint64((1 << bits) - 1)
        if ties:
            keys %= np.uint64(997)
        if high:
            keys[::2] |= np.uint64(1 << 63)
        vals = np.arange(n, dtype=np.uint32)
        ka, va, kb, vb = _sorted_both(L, keys, vals, bits)
        assert np.array_equal(ka, kb) and np.array_equal(va, vb)
        order = np.argsort(keys, kind="stable")
        assert np.array_equal(kb, keys[order]) and np.array_equal(vb, vals[order])


def test_noalloc_sort_rejects_oversized_input(lib):
    import torch
    L = lib
    n = 262145
    k = torch.arange(n, 0, -1, dtype=torch.int64, device="cuda")
    v = torch.zeros(n, dtype=torch.int32, device="cuda")
    before = k.clone()
    rc = L.hm_radix_sort_pairs_noalloc(ctypes.c_void_p(k.data_ptr()), ctypes.c_void_p(v.data_ptr()),
                                       n, 32, None)
    assert rc == -1
    assert b"262144" in L.hm_last_error()
    torch.cuda.synchronize()
    assert torch.equal(k, before)
