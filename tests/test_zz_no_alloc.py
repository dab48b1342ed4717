"""r4g_sort_pairs_noalloc -- the radix sort for callers that cannot allocate
device memory (it keeps its scratch in a fixed device array inside the
library instead of a caller buffer) -- gives exactly the result of
r4g_sort_pairs, call after call, and refuses sizes beyond its limit.

The file name sorts last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process."""
import ctypes as C

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def r4g():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2402_03307_gb300 as m
    return m


def _noalloc(lib, keys, vals, b0, b1):
    ko = torch.empty_like(keys)
    vo = torch.empty_like(vals)
    st = lib.r4g_sort_pairs_noalloc(keys.data_ptr(), vals.data_ptr(), ko.data_ptr(), vo.data_ptr(),
                                    keys.numel(), b0, b1, torch.cuda.current_stream().cuda_stream)
    assert st == 0, lib.r4g_last_error(None)
    return ko, vo


@pytest.mark.parametrize("cases", [((300_001, 0, 45), (4_099, 3, 40)), ((1_048_576, 0, 64), (777, 32, 45))])
def test_matches_the_allocating_sort_twice_in_a_row(r4g, cases):
    from paper_2402_03307_gb300 import abi
    lib = abi.lib()
    for k, (n, b0, b1) in enumerate(cases):
        keys, vals = synth.random_keys(seed=1000 + n + k, n=n, high_bits=13)
        kd = torch.as_tensor(keys.view(np.int64)).cuda()
        vd = torch.as_tensor(vals.view(np.int32)).cuda()
        ko, vo = _noalloc(lib, kd, vd, b0, b1)
        rk, rv = r4g.sort_pairs(kd, vd, b0, b1)
        torch.cuda.synchronize()
        assert torch.equal(ko, rk) and torch.equal(vo, rv), (n, b0, b1)
        assert torch.equal(kd.cpu(), torch.as_tensor(keys.view(np.int64)))  # inputs untouched
        # and against a CPU stable sort on the same key bits
        mask = np.uint64((1 << (b1 - b0)) - 1) if b1 - b0 < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
        order = np.argsort((keys >> np.uint64(b0)) & mask, kind="stable")
        assert np.array_equal(ko.cpu().numpy().view(np.uint64), keys[order]), (n, b0, b1)
        assert np.array_equal(vo.cpu().numpy().view(np.uint32), vals[order]), (n, b0, b1)


def test_allocates_no_device_memory(r4g):
    """After a warm call, further calls change neither the device's free
    memory nor what PyTorch's allocator holds."""
    from paper_2402_03307_gb300 import abi
    lib = abi.lib()
    keys, vals = synth.random_keys(seed=77, n=500_000, high_bits=13)
    kd = torch.as_tensor(keys.view(np.int64)).cuda()
    vd = torch.as_tensor(vals.view(np.int32)).cuda()
    ko = torch.empty_like(kd)
    vo = torch.empty_like(vd)
    s = torch.cuda.current_stream().cuda_stream

    def call():
        st = lib.r4g_sort_pairs_noalloc(kd.data_ptr(), vd.data_ptr(), ko.data_ptr(), vo.data_ptr(),
                                        kd.numel(), 0, 45, s)
        assert st == 0, lib.r4g_last_error(None)

    call()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    held0 = torch.cuda.memory_allocated()
    for _ in range(3):
        call()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0 and torch.cuda.memory_allocated() == held0


def test_rejects_sizes_beyond_the_limit(r4g):
    from paper_2402_03307_gb300 import abi
    lib = abi.lib()
    n = 1_048_577
    st = lib.r4g_sort_pairs_noalloc(C.c_void_p(256), C.c_void_p(512), C.c_void_p(1024), C.c_void_p(2048),
                                    n, 0, 64, None)
    assert st == abi.R4G_EINVAL
    assert b"R4G_SORT_NOALLOC_MAX_PAIRS" in lib.r4g_last_error(None)
