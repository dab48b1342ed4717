"""The C ABI library builds for sm_103a, loads without a GPU and exports every
entry point include/r4g.h declares; host-side argument checks return their
error codes without touching a device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "r4g.h")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2402_03307_gb300 import abi
    return abi.lib()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(r4g_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_the_header(lib):
    from paper_2402_03307_gb300 import abi
    bound = {s[0] for s in abi.SIGNATURES}
    assert set(declared_functions()) <= bound


def test_version(lib):
    assert lib.r4g_version() == 10000


def test_create_rejects_bad_config(lib):
    from paper_2402_03307_gb300 import abi
    cfg = abi.r4g_config()
    cfg.tile_w, cfg.tile_h, cfg.sh_degree = 12, 12, 3
    h = C.c_void_p()
    assert lib.r4g_create(C.byref(h), C.byref(cfg)) == abi.R4G_EINVAL
    cfg.tile_w, cfg.tile_h, cfg.sh_degree = 16, 16, 4
    assert lib.r4g_create(C.byref(h), C.byref(cfg)) == abi.R4G_EINVAL
    cfg.sh_degree, cfg.flags = 3, 0x100
    assert lib.r4g_create(C.byref(h), C.byref(cfg)) == abi.R4G_EINVAL
    assert b"flag" in lib.r4g_last_error(None)


def test_frame_bytes_and_argument_checks(lib):
    from paper_2402_03307_gb300 import abi
    ctx = abi.r4g_create()
    try:
        a = abi.r4g_frame_bytes(ctx, 1000, 128, 128, 1 << 16)
        b = abi.r4g_frame_bytes(ctx, 1000, 128, 128, 1 << 17)
        assert b - a >= 16 * (1 << 16)  # two (tile key, value) buffers per extra key
        assert a % 256 == 0
        out = C.c_size_t()
        assert lib.r4g_frame_bytes(ctx, -1, 128, 128, 10, C.byref(out)) == abi.R4G_EINVAL
        assert lib.r4g_frame_bytes(ctx, 10, 0, 128, 10, C.byref(out)) == abi.R4G_EINVAL
        # render with a NULL gaussian struct / camera is rejected on the host
        cam = abi.r4g_camera()
        cam.width, cam.height, cam.fx, cam.fy = 16, 16, 10.0, 10.0
        g = abi.r4g_gaussians()
        g.n = 0
        assert lib.r4g_render(ctx, None, C.byref(cam), 0.5, None, None, None, None, 0, 0, None) == abi.R4G_EINVAL
        assert lib.r4g_render(ctx, C.byref(g), None, 0.5, None, None, None, None, 0, 0, None) == abi.R4G_EINVAL
        # n > 0 with NULL parameter pointers
        g.n = 5
        assert lib.r4g_render(ctx, C.byref(g), C.byref(cam), 0.5, 1, None, None, 256, 1 << 20, 16,
                              None) == abi.R4G_EINVAL
        # an undersized frame is refused before any launch
        g.n = 0
        need = abi.r4g_frame_bytes(ctx, 0, 16, 16, 16)
        assert lib.r4g_render(ctx, C.byref(g), C.byref(cam), 0.5, 256, None, None, 256, need - 256, 16,
                              None) == abi.R4G_EWORKSPACE
        # non-finite t
        assert lib.r4g_render(ctx, C.byref(g), C.byref(cam), float("nan"), 256, None, None, 256, need, 16,
                              None) == abi.R4G_EINVAL
    finally:
        abi.r4g_destroy(ctx)


def test_sort_argument_checks(lib):
    from paper_2402_03307_gb300 import abi
    out = C.c_size_t()
    assert lib.r4g_sort_scratch_bytes(1000, C.byref(out)) == abi.R4G_OK and out.value >= 12000
    assert lib.r4g_sort_pairs(None, None, None, None, 10, 0, 70, None, 0, None) == abi.R4G_EINVAL
    assert lib.r4g_sort_pairs(None, None, None, None, 10, 8, 8, None, 0, None) == abi.R4G_EINVAL
    assert lib.r4g_sort_pairs(None, None, None, None, 0, 0, 64, None, 0, None) == abi.R4G_OK
    assert lib.r4g_sort_pairs(256, 512, 1024, 2048, 10, 0, 64, 4096, 1, None) == abi.R4G_EWORKSPACE
    assert lib.r4g_sort_pairs(256, 512, 256, 2048, 10, 0, 64, 4096, 1 << 20, None) == abi.R4G_EINVAL


def test_density_argument_checks(lib):
    from paper_2402_03307_gb300 import abi
    out = C.c_size_t()
    assert lib.r4g_densify_scratch_bytes(1000, C.byref(out)) == abi.R4G_OK and out.value >= 5000
    assert lib.r4g_densify_scratch_bytes(-1, C.byref(out)) == abi.R4G_EINVAL
    g = abi.r4g_gaussians()
    g.n = 10
    g.mean = g.rotor = g.logscale = g.sh = 256
    g.logit = 256
    cfg = abi.r4g_densify_config(2e-4, 0.06, 1.6, 0.005, 0.0, 0.0)
    nb = out.value
    # each bad configuration field is refused before any launch
    for field, value in (("grad_threshold", -1.0), ("dense_scale", 0.0), ("split_divisor", 1.0),
                         ("min_opacity", 1.0), ("max_scale", -1.0), ("max_screen_radius", float("inf"))):
        bad = abi.r4g_densify_config(2e-4, 0.06, 1.6, 0.005, 0.0, 0.0)
        setattr(bad, field, value)
        assert lib.r4g_densify_plan(C.byref(g), 256, 512, None, C.byref(bad), 4096, 1 << 20, 8, None) \
            == abi.R4G_EINVAL, field
    # missing statistics, misaligned scratch, undersized scratch, BF16 storage
    assert lib.r4g_densify_plan(C.byref(g), None, 512, None, C.byref(cfg), 4096, 1 << 20, 8, None) == abi.R4G_EINVAL
    assert lib.r4g_densify_plan(C.byref(g), 256, 512, None, C.byref(cfg), 4100, 1 << 20, 8, None) == abi.R4G_EINVAL
    assert lib.r4g_densify_plan(C.byref(g), 256, 512, None, C.byref(cfg), 4096, 16, 8, None) == abi.R4G_EWORKSPACE
    g.sh_dtype = abi.R4G_BF16
    assert lib.r4g_densify_plan(C.byref(g), 256, 512, None, C.byref(cfg), 4096, nb, 8, None) == abi.R4G_EINVAL
    g.sh_dtype = abi.R4G_F32
    o = abi.r4g_params_out()
    assert lib.r4g_densify_apply(C.byref(g), 256, C.byref(cfg), 4096, nb, C.byref(o), 5, None, None) \
        == abi.R4G_EINVAL  # NULL output rows
    assert lib.r4g_densify_apply(C.byref(g), 256, C.byref(cfg), 4096, nb, C.byref(o), -1, None, None) \
        == abi.R4G_EINVAL
    assert lib.r4g_opacity_reset(256, 10, 1.0, None) == abi.R4G_EINVAL
    assert lib.r4g_opacity_reset(None, 10, 0.01, None) == abi.R4G_EINVAL
    assert lib.r4g_opacity_reset(None, 0, 0.01, None) == abi.R4G_OK


def test_frame_status_decode(lib):
    """r4g_frame_status_decode is host logic: the three status words of a frame
    (status bits, key count, keys needed) to the r4g_frame_status result."""
    from paper_2402_03307_gb300 import abi
    words = (C.c_uint32 * 3)(0, 1000, 1000)
    need = C.c_int64()
    assert lib.r4g_frame_status_decode(words, C.byref(need)) == abi.R4G_OK and need.value == 1000
    words[0], words[2] = 1, 5000
    assert lib.r4g_frame_status_decode(words, C.byref(need)) == abi.R4G_EOVERFLOW and need.value == 5000
    assert b"capacity" in lib.r4g_last_error(None)
    words[0] = 2
    assert lib.r4g_frame_status_decode(words, None) == abi.R4G_ETIMEOUT
    words[0] = 4
    assert lib.r4g_frame_status_decode(words, None) == abi.R4G_EDEVICE
    assert lib.r4g_frame_status_decode(None, None) == abi.R4G_EINVAL
    assert lib.r4g_frame_status_async(None, 1 << 20, 256, None) == abi.R4G_EINVAL
    assert lib.r4g_frame_status_async(256, 16, 256, None) == abi.R4G_EWORKSPACE
