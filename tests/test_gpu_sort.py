"""The radix sort entry point (r4g_sort_pairs) is bit-exact against a CPU
stable sort of the same seeded keys: sizes that span several tiles and CTAs
with ragged tails, heavy duplicate keys (stability), partial bit ranges."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def _cpu_sort(keys: np.ndarray, vals: np.ndarray, b0: int, b1: int):
    width = b1 - b0
    mask = np.uint64((1 << width) - 1) if width < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
    digit = (keys >> np.uint64(b0)) & mask
    order = np.argsort(digit, kind="stable")
    return keys[order], vals[order]


@pytest.mark.parametrize("n", [1, 7, 2047, 2048, 2049, 100_003, 1_000_000])
@pytest.mark.parametrize("bits", [(0, 64), (0, 45), (32, 45), (3, 17)])
def test_sort_pairs_bit_exact(n, bits):
    import paper_2402_03307_gb300 as r4g
    keys, vals = synth.random_keys(seed=n, n=n, high_bits=13)
    kd = torch.as_tensor(keys.view(np.int64)).cuda()
    vd = torch.as_tensor(vals.view(np.int32)).cuda()
    ko, vo = r4g.sort_pairs(kd, vd, *bits)
    torch.cuda.synchronize()
    rk, rv = _cpu_sort(keys, vals, *bits)
    assert np.array_equal(ko.cpu().numpy().view(np.uint64), rk)
    assert np.array_equal(vo.cpu().numpy().view(np.uint32), rv)
    # inputs untouched
    assert np.array_equal(kd.cpu().numpy().view(np.uint64), keys)


def test_sort_large_full_width():
    """8M pairs on the 45 bits the 1352x1014 render sorts (tile id below 2^13)."""
    import paper_2402_03307_gb300 as r4g
    n = 8_000_000
    keys, vals = synth.random_keys(seed=99, n=n, high_bits=13)
    ko, vo = r4g.sort_pairs(torch.as_tensor(keys.view(np.int64)).cuda(),
                            torch.as_tensor(vals.view(np.int32)).cuda(), 0, 45)
    rk, rv = _cpu_sort(keys, vals, 0, 45)
    assert np.array_equal(ko.cpu().numpy().view(np.uint64), rk)
    assert np.array_equal(vo.cpu().numpy().view(np.uint32), rv)


def test_sort_empty():
    import paper_2402_03307_gb300 as r4g
    ko, vo = r4g.sort_pairs(torch.zeros(0, dtype=torch.int64, device="cuda"),
                            torch.zeros(0, dtype=torch.int32, device="cuda"))
    assert ko.numel() == 0 and vo.numel() == 0
