"""ctypes binding of the r4g C ABI (include/r4g.h): the same names, argument
marshalling only. Importing this module loads ``libr4g.so`` from the package
directory and raises if it is missing -- there is no fallback path."""
from __future__ import annotations

import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libr4g.so")

R4G_OK, R4G_EINVAL, R4G_ENOMEM, R4G_EWORKSPACE, R4G_ECUDA, R4G_ETIMEOUT, R4G_EDEVICE, R4G_EOVERFLOW = range(8)
R4G_F32, R4G_BF16 = 0, 1
R4G_FLAG_FP64_SLICE = 0x1
R4G_FLAG_NO_TEMPORAL_CULL = 0x2
R4G_FLAG_COUNT_PAIRS = 0x4
R4G_FLAG_FLOW = 0x8
STATUS_NAMES = {0: "R4G_OK", 1: "R4G_EINVAL", 2: "R4G_ENOMEM", 3: "R4G_EWORKSPACE", 4: "R4G_ECUDA",
                5: "R4G_ETIMEOUT", 6: "R4G_EDEVICE", 7: "R4G_EOVERFLOW"}


class r4g_config(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("bg", C.c_float * 3),
                ("sh_degree", C.c_int32), ("flags", C.c_uint32)]


class r4g_gaussians(C.Structure):
    _fields_ = [("mean", C.c_void_p), ("rotor", C.c_void_p), ("logscale", C.c_void_p),
                ("logit", C.c_void_p), ("sh", C.c_void_p), ("n", C.c_int64),
                ("scale_dtype", C.c_int32), ("sh_dtype", C.c_int32)]


class r4g_camera(C.Structure):
    _fields_ = [("world_to_cam", C.c_float * 12), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32)]


class r4g_grads(C.Structure):
    _fields_ = [("mean", C.c_void_p), ("rotor", C.c_void_p), ("logscale", C.c_void_p),
                ("logit", C.c_void_p), ("sh", C.c_void_p), ("vs_grad", C.c_void_p),
                ("vs_count", C.c_void_p), ("max_radius", C.c_void_p)]


class r4g_densify_config(C.Structure):
    _fields_ = [("grad_threshold", C.c_float), ("dense_scale", C.c_float), ("split_divisor", C.c_float),
                ("min_opacity", C.c_float), ("max_scale", C.c_float), ("max_screen_radius", C.c_float)]


class r4g_params_out(C.Structure):
    _fields_ = [("mean", C.c_void_p), ("rotor", C.c_void_p), ("logscale", C.c_void_p),
                ("logit", C.c_void_p), ("sh", C.c_void_p)]


class r4g_frame_info(C.Structure):
    _fields_ = [("n_visible", C.c_int64), ("key_count", C.c_int64), ("key_needed", C.c_int64),
                ("composited_pairs", C.c_int64), ("status", C.c_int32), ("reserved", C.c_int32),
                ("reached_pairs", C.c_int64), ("visible_gaussians", C.c_int64)]


class r4g_view(C.Structure):
    _fields_ = [("cam", r4g_camera), ("t", C.c_float)]


class r4g_tune_result(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("ms", C.c_float * 3),
                ("keys_needed", C.c_int64 * 3)]


TUNE_SHAPES = ((8, 8), (16, 16), (16, 32))


# (name, restype, argtypes) of every exported entry point
SIGNATURES = [
    ("r4g_version", C.c_int32, []),
    ("r4g_create", C.c_int, [C.POINTER(C.c_void_p), C.POINTER(r4g_config)]),
    ("r4g_destroy", None, [C.c_void_p]),
    ("r4g_last_error", C.c_char_p, [C.c_void_p]),
    ("r4g_frame_bytes", C.c_int, [C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.c_int64,
                                  C.POINTER(C.c_size_t)]),
    ("r4g_frame_status", C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.POINTER(C.c_int64), C.c_void_p]),
    ("r4g_frame_status_async", C.c_int, [C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p]),
    ("r4g_frame_status_decode", C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    ("r4g_frame_stats", C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.POINTER(r4g_frame_info), C.c_void_p]),
    ("r4g_frame_export", C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t, C.c_int64, C.c_int32, C.c_int32,
                                   C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("r4g_render", C.c_int, [C.c_void_p, C.POINTER(r4g_gaussians), C.POINTER(r4g_camera), C.c_float,
                             C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_int64,
                             C.c_void_p]),
    ("r4g_render_backward", C.c_int, [C.c_void_p, C.POINTER(r4g_gaussians), C.POINTER(r4g_camera),
                                      C.c_float, C.c_void_p, C.POINTER(r4g_grads), C.c_void_p,
                                      C.c_size_t, C.c_int64, C.c_void_p]),
    ("r4g_batch_frame_bytes", C.c_int, [C.c_void_p, C.c_int64, C.POINTER(r4g_view), C.c_int32, C.c_int64,
                                        C.c_int32, C.c_int32, C.POINTER(C.c_size_t)]),
    ("r4g_render_batch", C.c_int, [C.c_void_p, C.POINTER(r4g_gaussians), C.POINTER(r4g_view), C.c_int32,
                                   C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t, C.c_int64,
                                   C.c_void_p]),
    ("r4g_render_batch_backward", C.c_int, [C.c_void_p, C.POINTER(r4g_gaussians), C.POINTER(r4g_view),
                                            C.c_int32, C.c_void_p, C.POINTER(r4g_grads), C.c_void_p,
                                            C.c_size_t, C.c_int64, C.c_void_p]),
    ("r4g_autotune_batch", C.c_int, [C.c_void_p, C.POINTER(r4g_gaussians), C.POINTER(r4g_view), C.c_int32,
                                     C.c_void_p, C.c_void_p, C.POINTER(r4g_grads), C.c_void_p, C.c_size_t,
                                     C.c_int64, C.c_int32, C.c_void_p, C.POINTER(r4g_tune_result)]),
    ("r4g_set_tile", C.c_int, [C.c_void_p, C.c_int32, C.c_int32]),
    ("r4g_get_config", C.c_int, [C.c_void_p, C.POINTER(r4g_config)]),
    ("r4g_knn_scratch_bytes", C.c_int, [C.c_int64, C.POINTER(C.c_size_t)]),
    ("r4g_knn4d", C.c_int, [C.c_void_p, C.c_int64, C.c_float, C.c_float, C.c_int32, C.c_void_p, C.c_void_p,
                            C.c_void_p, C.c_size_t, C.c_void_p]),
    ("r4g_knn_status", C.c_int, [C.c_void_p, C.c_int64, C.c_void_p]),
    ("r4g_regularizers_scratch_bytes", C.c_int, [C.c_int64, C.POINTER(C.c_size_t)]),
    ("r4g_regularizers", C.c_int, [C.POINTER(r4g_gaussians), C.c_void_p, C.c_int32, C.c_float, C.c_float,
                                   C.c_void_p, C.POINTER(r4g_grads), C.c_void_p, C.c_size_t, C.c_void_p]),
    ("r4g_image_loss_scratch_bytes", C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_size_t)]),
    ("r4g_image_loss", C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_float, C.c_void_p,
                                 C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]),
    ("r4g_densify_scratch_bytes", C.c_int, [C.c_int64, C.POINTER(C.c_size_t)]),
    ("r4g_densify_plan", C.c_int, [C.POINTER(r4g_gaussians), C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.POINTER(r4g_densify_config), C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p]),
    ("r4g_densify_apply", C.c_int, [C.POINTER(r4g_gaussians), C.c_void_p, C.POINTER(r4g_densify_config),
                                    C.c_void_p, C.c_size_t, C.POINTER(r4g_params_out), C.c_int64, C.c_void_p,
                                    C.c_void_p]),
    ("r4g_opacity_reset", C.c_int, [C.c_void_p, C.c_int64, C.c_float, C.c_void_p]),
    ("r4g_set_timing", C.c_int, [C.c_void_p, C.c_int32]),
    ("r4g_stage_times", C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.c_int32]),
    ("r4g_sort_scratch_bytes", C.c_int, [C.c_int64, C.POINTER(C.c_size_t)]),
    ("r4g_sort_pairs", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                 C.c_int32, C.c_int32, C.c_void_p, C.c_size_t, C.c_void_p]),
    ("r4g_sort_pairs_noalloc", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                         C.c_int32, C.c_int32, C.c_void_p]),
    ("r4g_sort32_scratch_bytes", C.c_int, [C.c_int64, C.c_int32, C.POINTER(C.c_size_t)]),
    ("r4g_sort32", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int32,
                             C.c_void_p, C.c_size_t, C.c_void_p]),
    ("r4g_sort32_status", C.c_int, [C.c_void_p, C.c_void_p]),
    ("r4g_sort32_wait_test", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int32,
                                       C.c_void_p, C.c_size_t, C.c_void_p, C.c_uint32, C.c_uint32]),
]


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load libr4g.so and declare every entry point; raise if it is absent."""
    if not os.path.exists(path):
        raise ImportError(
            f"{path} is missing: build it with paper_2402_03307_gb300.build.build() "
            "(nvcc, sm_103a). There is no CPU fallback.")
    lib = C.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


class R4GError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib: C.CDLL | None = None


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        _lib = load()
    return _lib


def check(status: int, ctx=None) -> None:
    if status != R4G_OK:
        msg = lib().r4g_last_error(ctx)
        raise R4GError(status, msg.decode() if msg else "")


# thin wrappers with the ABI's names ------------------------------------------

def r4g_version() -> int:
    return lib().r4g_version()


def r4g_create(cfg: r4g_config | None = None) -> C.c_void_p:
    h = C.c_void_p()
    check(lib().r4g_create(C.byref(h), C.byref(cfg) if cfg is not None else None))
    return h


def r4g_destroy(ctx) -> None:
    lib().r4g_destroy(ctx)


def r4g_frame_bytes(ctx, n: int, width: int, height: int, key_capacity: int) -> int:
    out = C.c_size_t()
    check(lib().r4g_frame_bytes(ctx, n, width, height, key_capacity, C.byref(out)), ctx)
    return out.value


def r4g_frame_status(ctx, frame: int, frame_bytes: int, stream: int) -> tuple[int, int]:
    need = C.c_int64()
    st = lib().r4g_frame_status(ctx, frame, frame_bytes, C.byref(need), stream)
    if st not in (R4G_OK, R4G_EOVERFLOW):
        check(st, ctx)
    return st, need.value


def r4g_frame_status_async(frame: int, frame_bytes: int, host_out: int, stream: int) -> None:
    check(lib().r4g_frame_status_async(frame, frame_bytes, host_out, stream))


def r4g_frame_status_decode(words: int) -> tuple[int, int]:
    need = C.c_int64()
    st = lib().r4g_frame_status_decode(words, C.byref(need))
    if st not in (R4G_OK, R4G_EOVERFLOW, R4G_ETIMEOUT, R4G_EDEVICE):
        check(st)
    return st, need.value


def r4g_frame_stats(ctx, frame: int, frame_bytes: int, stream: int) -> dict:
    info = r4g_frame_info()
    check(lib().r4g_frame_stats(ctx, frame, frame_bytes, C.byref(info), stream), ctx)
    return {k: getattr(info, k) for k, _ in r4g_frame_info._fields_ if k != "reserved"}


def r4g_frame_export(ctx, frame, frame_bytes, n, width, height, key_count, keys, values, ranges,
                     records, stream) -> None:
    check(lib().r4g_frame_export(ctx, frame, frame_bytes, n, width, height, key_count, keys, values,
                                 ranges, records, stream), ctx)


def r4g_render(ctx, g: r4g_gaussians, cam: r4g_camera, t: float, out_rgb, out_T, out_last, frame,
               frame_bytes, key_capacity, stream) -> None:
    check(lib().r4g_render(ctx, C.byref(g), C.byref(cam), t, out_rgb, out_T, out_last, frame,
                           frame_bytes, key_capacity, stream), ctx)


def r4g_render_backward(ctx, g: r4g_gaussians, cam: r4g_camera, t: float, grad_rgb, grads: r4g_grads,
                        frame, frame_bytes, key_capacity, stream) -> None:
    check(lib().r4g_render_backward(ctx, C.byref(g), C.byref(cam), t, grad_rgb, C.byref(grads), frame,
                                    frame_bytes, key_capacity, stream), ctx)


def view_array(views) -> C.Array:
    """Host r4g_view[] from a sequence of r4g_view."""
    arr = (r4g_view * len(views))()
    for k, v in enumerate(views):
        arr[k] = v
    return arr


def r4g_batch_frame_bytes(ctx, n: int, views, key_capacity: int, tile=(0, 0)) -> int:
    out = C.c_size_t()
    arr = view_array(views)
    check(lib().r4g_batch_frame_bytes(ctx, n, arr, len(views), key_capacity, tile[0], tile[1], C.byref(out)), ctx)
    return out.value


def r4g_render_batch(ctx, g: r4g_gaussians, views, views_dev, out_rgb, out_T, frame, frame_bytes,
                     key_capacity, stream) -> None:
    arr = view_array(views)
    check(lib().r4g_render_batch(ctx, C.byref(g), arr, len(views), views_dev, out_rgb, out_T, frame, frame_bytes,
                                 key_capacity, stream), ctx)


def r4g_render_batch_backward(ctx, g: r4g_gaussians, views, grad_rgb, grads: r4g_grads, frame, frame_bytes,
                              key_capacity, stream) -> None:
    arr = view_array(views)
    check(lib().r4g_render_batch_backward(ctx, C.byref(g), arr, len(views), grad_rgb, C.byref(grads), frame,
                                          frame_bytes, key_capacity, stream), ctx)


def r4g_autotune_batch(ctx, g: r4g_gaussians, views, out_rgb, grad_rgb, grads, frame, frame_bytes,
                       key_capacity, reps, stream) -> dict:
    arr = view_array(views)
    res = r4g_tune_result()
    check(lib().r4g_autotune_batch(ctx, C.byref(g), arr, len(views), out_rgb, grad_rgb,
                                   C.byref(grads) if grads is not None else None, frame, frame_bytes,
                                   key_capacity, reps, stream, C.byref(res)), ctx)
    return {"tile": (res.tile_w, res.tile_h),
            "ms": {f"{w}x{h}": (res.ms[k] if res.ms[k] >= 0 else None) for k, (w, h) in enumerate(TUNE_SHAPES)},
            "keys_needed": {f"{w}x{h}": res.keys_needed[k] for k, (w, h) in enumerate(TUNE_SHAPES)}}


def r4g_knn_scratch_bytes(n: int) -> int:
    out = C.c_size_t()
    check(lib().r4g_knn_scratch_bytes(n, C.byref(out)))
    return out.value


def r4g_knn4d(means, n, scale_xyz, scale_t, k, out_idx, out_dist2, scratch, scratch_bytes, stream) -> None:
    check(lib().r4g_knn4d(means, n, scale_xyz, scale_t, k, out_idx, out_dist2, scratch, scratch_bytes, stream))


def r4g_knn_status(scratch, n, stream) -> int:
    st = lib().r4g_knn_status(scratch, n, stream)
    if st not in (R4G_OK, R4G_ETIMEOUT):
        check(st)
    return st


def r4g_regularizers_scratch_bytes(n: int) -> int:
    out = C.c_size_t()
    check(lib().r4g_regularizers_scratch_bytes(n, C.byref(out)))
    return out.value


def r4g_regularizers(g: r4g_gaussians, knn_idx, k, lambda_entropy, lambda_consistency, out_loss,
                     grads: r4g_grads | None, scratch, scratch_bytes, stream) -> None:
    check(lib().r4g_regularizers(C.byref(g), knn_idx, k, lambda_entropy, lambda_consistency, out_loss,
                                 C.byref(grads) if grads is not None else None, scratch, scratch_bytes, stream))


def r4g_image_loss_scratch_bytes(c: int, h: int, w: int) -> int:
    out = C.c_size_t()
    check(lib().r4g_image_loss_scratch_bytes(c, h, w, C.byref(out)))
    return out.value


def r4g_image_loss(image, target, c, h, w, lam, out_loss, grad, scratch, scratch_bytes, stream) -> None:
    check(lib().r4g_image_loss(image, target, c, h, w, lam, out_loss, grad, scratch, scratch_bytes, stream))


def r4g_densify_scratch_bytes(n: int) -> int:
    out = C.c_size_t()
    check(lib().r4g_densify_scratch_bytes(n, C.byref(out)))
    return out.value


def r4g_densify_plan(g: r4g_gaussians, vs_grad, vs_count, max_radius, cfg: r4g_densify_config, scratch,
                     scratch_bytes, out_count, stream) -> None:
    check(lib().r4g_densify_plan(C.byref(g), vs_grad, vs_count, max_radius, C.byref(cfg), scratch, scratch_bytes,
                                 out_count, stream))


def r4g_densify_apply(g: r4g_gaussians, z, cfg: r4g_densify_config, scratch, scratch_bytes,
                      out: r4g_params_out, capacity, out_src, stream) -> None:
    check(lib().r4g_densify_apply(C.byref(g), z, C.byref(cfg), scratch, scratch_bytes, C.byref(out), capacity,
                                  out_src, stream))


def r4g_opacity_reset(logit, n, max_opacity, stream) -> None:
    check(lib().r4g_opacity_reset(logit, n, max_opacity, stream))


def r4g_set_tile(ctx, tile_w: int, tile_h: int) -> None:
    check(lib().r4g_set_tile(ctx, tile_w, tile_h), ctx)


def r4g_get_config(ctx) -> r4g_config:
    cfg = r4g_config()
    check(lib().r4g_get_config(ctx, C.byref(cfg)), ctx)
    return cfg


STAGES = ("preprocess", "binning", "sort", "ranges", "blend", "blend_bwd", "preprocess_bwd")


def r4g_set_timing(ctx, enable: bool) -> None:
    check(lib().r4g_set_timing(ctx, 1 if enable else 0), ctx)


def r4g_stage_times(ctx, reset: bool = True) -> tuple[dict, dict]:
    ms = (C.c_double * len(STAGES))()
    ln = (C.c_int64 * len(STAGES))()
    check(lib().r4g_stage_times(ctx, ms, ln, 1 if reset else 0), ctx)
    return ({k: ms[i] for i, k in enumerate(STAGES)}, {k: ln[i] for i, k in enumerate(STAGES)})


def r4g_sort_scratch_bytes(n: int) -> int:
    out = C.c_size_t()
    check(lib().r4g_sort_scratch_bytes(n, C.byref(out)))
    return out.value


def r4g_sort32_scratch_bytes(n: int, bits: int) -> int:
    out = C.c_size_t()
    check(lib().r4g_sort32_scratch_bytes(n, bits, C.byref(out)))
    return out.value


def r4g_sort32(keys_in, values_in, keys_out, values_out, n, bits, scratch, scratch_bytes, stream) -> None:
    check(lib().r4g_sort32(keys_in, values_in, keys_out, values_out, n, bits, scratch, scratch_bytes, stream))


def r4g_sort_pairs(keys_in, values_in, keys_out, values_out, n, begin_bit, end_bit, scratch,
                   scratch_bytes, stream) -> None:
    check(lib().r4g_sort_pairs(keys_in, values_in, keys_out, values_out, n, begin_bit, end_bit,
                               scratch, scratch_bytes, stream))
