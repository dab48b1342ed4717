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


def _depth_like_keys(seed: int, n: int, bits: int) -> np.ndarray:
    """Seeded uint32 keys: IEEE bits of positive depths in (0.2, 20) for 32 bits
    (a quarter of them duplicated, as tied depths), uniform tile ids below 2^bits
    otherwise."""
    rng = np.random.default_rng(seed)
    if bits == 32:
        z = rng.uniform(0.2, 20.0, n).astype(np.float32)
        z[rng.integers(0, n, n // 4)] = z[rng.integers(0, n, n // 4)]
        return z.view(np.uint32)
    return rng.integers(0, 1 << bits, n, dtype=np.uint64).astype(np.uint32)


@pytest.mark.parametrize("n,bits", [(1, 32), (2047, 32), (2049, 13), (300_001, 32), (3_000_000, 13),
                                    (3_000_000, 32), (12_000_000, 13)])
def test_render_sort_bit_exact(n, bits):
    """The render's own sort kernels (r4g_sort32) against a CPU stable sort:
    depth-like 32-bit keys (four passes) and tile ids of the 1352x1014 view
    (13 bits, two passes), up to 12M pairs."""
    import paper_2402_03307_gb300 as r4g
    keys = _depth_like_keys(n + bits, n, bits)
    vals = np.random.default_rng(n).permutation(n).astype(np.uint32)
    ko, vo = r4g.sort32(torch.as_tensor(keys.view(np.int32)).cuda(), torch.as_tensor(vals.view(np.int32)).cuda(),
                        bits)
    order = np.argsort(keys & np.uint32((1 << bits) - 1 if bits < 32 else 0xFFFFFFFF), kind="stable")
    assert np.array_equal(ko.cpu().numpy().view(np.uint32), keys[order])
    assert np.array_equal(vo.cpu().numpy().view(np.uint32), vals[order])
    # values omitted: the positions are sorted
    _, po = r4g.sort32(torch.as_tensor(keys.view(np.int32)).cuda(), None, bits)
    assert np.array_equal(po.cpu().numpy(), order.astype(np.int32))


def test_render_sort_bounded_wait_runs_out():
    """The failure path of the look-back wait (a tile that never publishes):
    the call completes, its status reads R4G_ETIMEOUT, nothing hangs or
    faults, and the next call on the same scratch is correct. The wait is the
    sort's only wait; its limit is 2^22 rounds in the render and 1000 here."""
    from paper_2402_03307_gb300 import abi
    n, bits = 20 * 2048 + 5, 32
    keys = _depth_like_keys(5, n, bits)
    kd = torch.as_tensor(keys.view(np.int32)).cuda()
    ko = torch.empty_like(kd)
    vo = torch.empty_like(kd)
    nb = abi.r4g_sort32_scratch_bytes(n, bits)
    scratch = torch.empty(nb, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    lib = abi.lib()
    st = lib.r4g_sort32_wait_test(kd.data_ptr(), None, ko.data_ptr(), vo.data_ptr(), n, bits, scratch.data_ptr(),
                                  nb, s, 3, 1000)
    assert st == abi.R4G_OK
    assert lib.r4g_sort32_status(scratch.data_ptr(), s) == abi.R4G_ETIMEOUT
    assert b"look-back" in lib.r4g_last_error(None)
    # the context and the scratch stay usable
    abi.r4g_sort32(kd.data_ptr(), None, ko.data_ptr(), vo.data_ptr(), n, bits, scratch.data_ptr(), nb, s)
    assert lib.r4g_sort32_status(scratch.data_ptr(), s) == abi.R4G_OK
    order = np.argsort(keys, kind="stable")
    assert np.array_equal(ko.cpu().numpy().view(np.uint32), keys[order])
    assert np.array_equal(vo.cpu().numpy(), order.astype(np.int32))
    # the hook refuses a limit that would make the test wait long
    assert lib.r4g_sort32_wait_test(kd.data_ptr(), None, ko.data_ptr(), vo.data_ptr(), n, bits,
                                    scratch.data_ptr(), nb, s, 3, 1 << 20) == abi.R4G_EINVAL
