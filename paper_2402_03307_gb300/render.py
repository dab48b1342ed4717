"""PyTorch-facing API over the r4g C ABI: device memory and streams come from
PyTorch, every step of the render and of its backward runs in libr4g's CUDA
kernels.

    r = Renderer()                       # 16x16 tiles, black background, SH degree 3
    img = r.render(params, cam, t).image # [3, H, W] float32 on the GPU
    img = render(params, cam, t)         # autograd-aware (Render4DFunction)
    res = r.render_batch(params, [(cam0, t0), (cam1, t1)])   # many views, one launch sequence
    g = BatchGraph(r, params, views)     # the same, captured in a CUDA graph
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import abi

PARAM_NAMES = ("mean", "rotor", "logscale", "logit", "sh")


def camera_struct(cam) -> abi.r4g_camera:
    """r4g_camera from any object (or dict) with world_to_cam [3,4], fx, fy,
    cx, cy, width, height."""
    get = (lambda k: cam[k]) if isinstance(cam, dict) else (lambda k: getattr(cam, k))
    c = abi.r4g_camera()
    w2c = [float(x) for x in torch.as_tensor(get("world_to_cam"), dtype=torch.float32).flatten().tolist()]
    if len(w2c) != 12:
        raise ValueError("world_to_cam must have 12 entries (3x4)")
    for k in range(12):
        c.world_to_cam[k] = w2c[k]
    c.fx, c.fy, c.cx, c.cy = float(get("fx")), float(get("fy")), float(get("cx")), float(get("cy"))
    c.width, c.height = int(get("width")), int(get("height"))
    return c


def view_struct(cam, t: float) -> abi.r4g_view:
    v = abi.r4g_view()
    v.cam = camera_struct(cam)
    v.t = float(t)
    return v


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return abi.R4G_F32
    if t.dtype == torch.bfloat16:
        return abi.R4G_BF16
    raise TypeError(f"unsupported dtype {t.dtype}")


def gaussians_struct(p: dict) -> abi.r4g_gaussians:
    n = int(p["mean"].shape[0])
    shapes = {"mean": (n, 4), "rotor": (n, 8), "logscale": (n, 4), "logit": (n,), "sh": (n, 16, 3)}
    for k, shp in shapes.items():
        t = p[k]
        if not t.is_cuda:
            raise ValueError(f"{k} must be a CUDA tensor")
        if tuple(t.shape) != shp:
            raise ValueError(f"{k} has shape {tuple(t.shape)}, expected {shp}")
        if not t.is_contiguous():
            raise ValueError(f"{k} must be contiguous")
    for k in ("mean", "rotor", "logit"):
        if p[k].dtype != torch.float32:
            raise TypeError(f"{k} must be float32")
    g = abi.r4g_gaussians()
    g.mean, g.rotor, g.logscale = p["mean"].data_ptr(), p["rotor"].data_ptr(), p["logscale"].data_ptr()
    g.logit, g.sh, g.n = p["logit"].data_ptr(), p["sh"].data_ptr(), n
    g.scale_dtype, g.sh_dtype = _dtype_code(p["logscale"]), _dtype_code(p["sh"])
    return g


@dataclass
class RenderResult:
    image: torch.Tensor        # [3, H, W]
    frame: torch.Tensor        # uint8 frame buffer (saved state for the backward)
    key_capacity: int
    width: int
    height: int
    n: int


@dataclass
class BatchResult:
    images: list               # per view [3, H_v, W_v] views into `packed`
    packed: torch.Tensor       # all views' images, view after view
    frame: torch.Tensor
    key_capacity: int
    views: list                # r4g_view structs of the call
    n: int


class PendingStatus:
    """A render's status words on their way to pinned host memory
    (r4g_frame_status_async) and the event after which they are there."""

    def __init__(self, res, stream, key):
        self.key = key  # the renderer's capacity-hint key of the render
        self.words = torch.zeros(3, dtype=torch.int32, pin_memory=True)
        abi.r4g_frame_status_async(res.frame.data_ptr(), res.frame.numel(), self.words.data_ptr(), stream.cuda_stream)
        self.event = torch.cuda.Event()
        self.event.record(stream)

    def result(self) -> tuple[int, int]:
        """(status, keys_needed); waits for the event only."""
        self.event.synchronize()
        return abi.r4g_frame_status_decode(self.words.data_ptr())


def _packed_views(packed: torch.Tensor, structs) -> list:
    out, off = [], 0
    for v in structs:
        h, w = v.cam.height, v.cam.width
        out.append(packed[off:off + 3 * h * w].view(3, h, w))
        off += 3 * h * w
    return out


STAT_NAMES = ("vs_grad", "vs_count", "max_radius")


def density_stats(n: int, device) -> dict:
    """Zeroed density-control statistics for n Gaussians (float32 [n] each):
    the summed view-space gradient norms, the number of views that
    composited each Gaussian, and its largest screen radius."""
    return {k: torch.zeros(n, dtype=torch.float32, device=device) for k in STAT_NAMES}


def _set_stats(out: abi.r4g_grads, stats: dict | None, params: dict) -> None:
    if stats is None:
        return
    n = int(params["mean"].shape[0])
    for k in STAT_NAMES:
        t_ = stats.get(k)
        if t_ is None:
            continue
        if t_.dtype != torch.float32 or not t_.is_contiguous() or t_.numel() != n or not t_.is_cuda:
            raise ValueError(f"stats[{k}] must be a contiguous float32 CUDA tensor [N]")
        setattr(out, k, t_.data_ptr())


class Renderer:
    """Owns an r4g context (tile shape, background, SH degree, flags)."""

    def __init__(self, tile=(16, 16), bg=(0.0, 0.0, 0.0), sh_degree: int = 3, flags: int = 0,
                 keys_per_gaussian: float = 32.0):
        cfg = abi.r4g_config()
        cfg.tile_w, cfg.tile_h = int(tile[0]), int(tile[1])
        for k in range(3):
            cfg.bg[k] = float(bg[k])
        cfg.sh_degree = int(sh_degree)
        cfg.flags = int(flags)
        self.cfg = cfg
        self.tile = (cfg.tile_w, cfg.tile_h)
        self.bg = tuple(float(x) for x in bg)
        self.ctx = abi.r4g_create(cfg)
        self.keys_per_gaussian = float(keys_per_gaussian)
        self._cap_hint: dict = {}
        # density-control statistics the backward updates when set (see density_stats)
        self.density: dict | None = None

    def __del__(self):
        ctx = getattr(self, "ctx", None)
        if ctx is not None and abi._lib is not None:
            abi.r4g_destroy(ctx)
            self.ctx = None

    # ---- memory ---------------------------------------------------------------
    def frame_bytes(self, n: int, width: int, height: int, key_capacity: int) -> int:
        return abi.r4g_frame_bytes(self.ctx, n, width, height, key_capacity)

    def new_frame(self, n: int, width: int, height: int, key_capacity: int, device=None) -> torch.Tensor:
        nbytes = self.frame_bytes(n, width, height, key_capacity)
        return torch.empty(nbytes, dtype=torch.uint8, device=device or torch.cuda.current_device())

    def default_capacity(self, n: int, width: int, height: int) -> int:
        hint = self._cap_hint.get((n, width, height))
        if hint:
            return hint
        return int(max(1 << 16, self.keys_per_gaussian * max(n, 1)))

    # ---- render ---------------------------------------------------------------
    def render(self, params: dict, cam, t: float, *, frame: torch.Tensor | None = None,
               key_capacity: int | None = None, out: torch.Tensor | None = None,
               check: bool = True, stream=None) -> RenderResult:
        """Render one view. With ``check`` the call waits for the stream to read
        the frame status and re-renders with a larger key buffer on overflow;
        without it the caller must call :meth:`status` before trusting the image."""
        g = gaussians_struct(params)
        c = camera_struct(cam)
        dev = params["mean"].device
        cap = int(key_capacity or self.default_capacity(g.n, c.width, c.height))
        s = (stream or torch.cuda.current_stream(dev)).cuda_stream
        while True:
            if frame is None or frame.numel() < self.frame_bytes(g.n, c.width, c.height, cap):
                frame = self.new_frame(g.n, c.width, c.height, cap, dev)
            img = out if out is not None else torch.empty((3, c.height, c.width), dtype=torch.float32, device=dev)
            abi.r4g_render(self.ctx, g, c, float(t), img.data_ptr(), None, None, frame.data_ptr(),
                           frame.numel(), cap, s)
            res = RenderResult(img, frame, cap, c.width, c.height, g.n)
            if not check:
                return res
            st, need = abi.r4g_frame_status(self.ctx, frame.data_ptr(), frame.numel(), s)
            if st == abi.R4G_OK:
                return res
            cap = int(need * 1.25) + 1024
            self._cap_hint[(g.n, c.width, c.height)] = cap
            frame = None

    # ---- deferred status checks (training steps) --------------------------------
    # The first render of a given size waits for its status (and grows the key
    # buffer until it fits, remembering the size); later ones only enqueue the
    # status copy, and settle() -- called by the backward, when the stream is
    # long past the render -- raises if the key buffer overflowed after all
    # (the capacity hint has then grown, so repeating the step succeeds).
    def render_deferred(self, params: dict, cam, t: float, stream=None):
        g = gaussians_struct(params)
        c = camera_struct(cam)
        st = stream or torch.cuda.current_stream(params["mean"].device)
        if (g.n, c.width, c.height) not in self._cap_hint:
            res = self.render(params, cam, t, stream=st)
            self._cap_hint.setdefault((g.n, c.width, c.height), res.key_capacity)
            return res, None
        res = self.render(params, cam, t, check=False, stream=st)
        return res, PendingStatus(res, st, (g.n, c.width, c.height))

    def render_batch_deferred(self, params: dict, views, stream=None):
        vs = self.view_structs(views)
        st = stream or torch.cuda.current_stream(params["mean"].device)
        key = (int(params["mean"].shape[0]), tuple((v.cam.width, v.cam.height) for v in vs), self.tile)
        if key not in self._cap_hint:
            res = self.render_batch(params, vs, stream=st)
            self._cap_hint.setdefault(key, res.key_capacity)
            return res, None
        res = self.render_batch(params, vs, check=False, stream=st)
        return res, PendingStatus(res, st, key)

    def reserve_batch(self, params: dict, view_sets) -> int:
        """Render each list of views of ``view_sets`` once (untimed, waiting
        for each status) and keep 10 % above the largest key count any of them
        needed as the key capacity of batched calls of those sizes, so that
        deferred renders of these views never overflow. Returns the capacity."""
        n = int(params["mean"].shape[0])
        need, key = 0, None
        for views in view_sets:
            vs = self.view_structs(views)
            k = (n, tuple((v.cam.width, v.cam.height) for v in vs), self.tile)
            if key is not None and k != key:
                raise ValueError("every view set must have the same image sizes")
            key = k
            res = self.render_batch(params, vs)
            need = max(need, self.status_of(res)[1])
        cap = int(need * 1.1) + 1024
        if key is not None:
            self._cap_hint[key] = max(cap, self._cap_hint.get(key, 0))
        return cap

    def settle(self, pending: "PendingStatus | None", res) -> None:
        """Raise if a deferred render's frame reports an error."""
        if pending is None:
            return
        status, need = pending.result()
        if status == abi.R4G_OK:
            return
        if status == abi.R4G_EOVERFLOW:
            self._cap_hint[pending.key] = int(need * 1.25) + 1024
            raise abi.R4GError(status, f"the render needed {need} (tile, Gaussian) pairs, more than its key "
                                       f"capacity {res.key_capacity}; the capacity has grown, repeat the step")
        raise abi.R4GError(status, "the render's frame reports an error")

    def stats(self, res: RenderResult, stream=None) -> dict:
        """n_visible, key_count, key_needed, composited_pairs (-1 unless the
        renderer was made with flags including R4G_FLAG_COUNT_PAIRS), status."""
        s = (stream or torch.cuda.current_stream()).cuda_stream
        return abi.r4g_frame_stats(self.ctx, res.frame.data_ptr(), res.frame.numel(), s)

    def status(self, res: RenderResult, stream=None) -> tuple[int, int]:
        s = (stream or torch.cuda.current_stream()).cuda_stream
        return abi.r4g_frame_status(self.ctx, res.frame.data_ptr(), res.frame.numel(), s)

    status_of = status

    def backward(self, params: dict, cam, t: float, res: RenderResult, grad_image: torch.Tensor,
                 grads: dict, stream=None, stats: dict | None = None) -> None:
        """Accumulate dL/dparams into ``grads`` (float32 tensors shaped like the
        parameters) given dL/dimage for a render ``res`` of (params, cam, t).
        ``stats`` (default: ``self.density``), a :func:`density_stats` dict,
        receives the view's density-control statistics."""
        g = gaussians_struct(params)
        c = camera_struct(cam)
        gi = grad_image.contiguous()
        if gi.dtype != torch.float32 or tuple(gi.shape) != (3, c.height, c.width):
            raise ValueError("grad_image must be float32 [3, H, W]")
        out = abi.r4g_grads()
        for k in PARAM_NAMES:
            t_ = grads[k]
            if t_.dtype != torch.float32 or not t_.is_contiguous() or t_.numel() != params[k].numel():
                raise ValueError(f"grads[{k}] must be a contiguous float32 tensor like the parameter")
            setattr(out, k, t_.data_ptr())
        _set_stats(out, stats if stats is not None else self.density, params)
        s = (stream or torch.cuda.current_stream(gi.device)).cuda_stream
        abi.r4g_render_backward(self.ctx, g, c, float(t), gi.data_ptr(), out, res.frame.data_ptr(),
                                res.frame.numel(), res.key_capacity, s)

    # ---- batched views ---------------------------------------------------------
    @staticmethod
    def view_structs(views) -> list:
        """r4g_view structs from (camera, t) pairs (or r4g_view structs)."""
        return [v if isinstance(v, abi.r4g_view) else view_struct(v[0], v[1]) for v in views]

    def batch_frame_bytes(self, n: int, views, key_capacity: int, tile=None) -> int:
        return abi.r4g_batch_frame_bytes(self.ctx, n, self.view_structs(views), key_capacity, tile or (0, 0))

    def render_batch(self, params: dict, views, *, frame: torch.Tensor | None = None,
                     key_capacity: int | None = None, out: torch.Tensor | None = None,
                     views_dev: torch.Tensor | None = None, check: bool = True, stream=None) -> BatchResult:
        """Render every (camera, t) view of ``views`` in one batched call. The
        images come back packed view after view (``packed``) and as per-view
        [3, H, W] views (``images``). ``views_dev``: optional device copy of the
        view structs (see :func:`views_tensor`) read by the kernels."""
        g = gaussians_struct(params)
        vs = self.view_structs(views)
        dev = params["mean"].device
        npix = sum(v.cam.width * v.cam.height for v in vs)
        key = (g.n, tuple((v.cam.width, v.cam.height) for v in vs), self.tile)
        cap = int(key_capacity or self._cap_hint.get(key) or max(1 << 16, self.keys_per_gaussian * max(g.n, 1) * len(vs)))
        s = (stream or torch.cuda.current_stream(dev)).cuda_stream
        while True:
            need_bytes = self.batch_frame_bytes(g.n, vs, cap)
            if frame is None or frame.numel() < need_bytes:
                frame = torch.empty(need_bytes, dtype=torch.uint8, device=dev)
            packed = out if out is not None else torch.empty(3 * npix, dtype=torch.float32, device=dev)
            abi.r4g_render_batch(self.ctx, g, vs, views_dev.data_ptr() if views_dev is not None else None,
                                 packed.data_ptr(), None, frame.data_ptr(), frame.numel(), cap, s)
            res = BatchResult(_packed_views(packed, vs), packed, frame, cap, vs, g.n)
            if not check:
                return res
            st, need = abi.r4g_frame_status(self.ctx, frame.data_ptr(), frame.numel(), s)
            if st == abi.R4G_OK:
                return res
            cap = int(need * 1.25) + 1024
            self._cap_hint[key] = cap
            frame = None

    def backward_batch(self, params: dict, res: BatchResult, grad_packed: torch.Tensor, grads: dict,
                       stream=None, stats: dict | None = None) -> None:
        """Accumulate dL/dparams (summed over the views) into ``grads`` given
        dL/d(packed images) of a batched render ``res``; ``stats`` as in
        :meth:`backward` (updated once per view)."""
        g = gaussians_struct(params)
        gp = grad_packed.contiguous()
        if gp.dtype != torch.float32 or gp.numel() != res.packed.numel():
            raise ValueError("grad_packed must be float32 with as many elements as the packed images")
        out = abi.r4g_grads()
        for k in PARAM_NAMES:
            t_ = grads[k]
            if t_.dtype != torch.float32 or not t_.is_contiguous() or t_.numel() != params[k].numel():
                raise ValueError(f"grads[{k}] must be a contiguous float32 tensor like the parameter")
            setattr(out, k, t_.data_ptr())
        _set_stats(out, stats if stats is not None else self.density, params)
        s = (stream or torch.cuda.current_stream(gp.device)).cuda_stream
        abi.r4g_render_batch_backward(self.ctx, g, res.views, gp.data_ptr(), out, res.frame.data_ptr(),
                                      res.frame.numel(), res.key_capacity, s)

    def autotune(self, params: dict, views, *, backward: bool = True, reps: int = 3,
                 key_capacity: int | None = None) -> dict:
        """Time the batched render (and backward) for 8x8, 16x16 and 16x32 tiles
        and keep the fastest on this renderer (r4g_autotune_batch)."""
        g = gaussians_struct(params)
        vs = self.view_structs(views)
        dev = params["mean"].device
        npix = sum(v.cam.width * v.cam.height for v in vs)
        cap = int(key_capacity or max(1 << 16, self.keys_per_gaussian * max(g.n, 1) * len(vs)))
        nbytes = max(self.batch_frame_bytes(g.n, vs, cap, tile) for tile in abi.TUNE_SHAPES)
        frame = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        packed = torch.empty(3 * npix, dtype=torch.float32, device=dev)
        gimg = grads = gstruct = None
        if backward:
            gimg = torch.full((3 * npix,), 1.0 / (3 * npix), dtype=torch.float32, device=dev)
            grads = {k: torch.zeros(v.shape, dtype=torch.float32, device=dev) for k, v in params.items()}
            gstruct = abi.r4g_grads()
            for k in PARAM_NAMES:
                setattr(gstruct, k, grads[k].data_ptr())
        s = torch.cuda.current_stream(dev).cuda_stream
        out = abi.r4g_autotune_batch(self.ctx, g, vs, packed.data_ptr(), gimg.data_ptr() if backward else None,
                                     gstruct, frame.data_ptr(), frame.numel(), cap, reps, s)
        self.tile = tuple(out["tile"])
        return out

    def set_tile(self, tile) -> None:
        abi.r4g_set_tile(self.ctx, int(tile[0]), int(tile[1]))
        self.tile = (int(tile[0]), int(tile[1]))

    def export(self, res: RenderResult, stream=None) -> dict:
        """Sorted keys / values, tile ranges and screen records of a frame (tests, tools)."""
        dev = res.frame.device
        s = (stream or torch.cuda.current_stream(dev)).cuda_stream
        cnt = torch.zeros(1, dtype=torch.int32, device=dev)
        abi.r4g_frame_export(self.ctx, res.frame.data_ptr(), res.frame.numel(), res.n, res.width,
                             res.height, cnt.data_ptr(), None, None, None, None, s)
        k = int(cnt.item())
        keys = torch.empty(max(k, 1), dtype=torch.int64, device=dev)
        vals = torch.empty(max(k, 1), dtype=torch.int32, device=dev)
        tx = (res.width + self.tile[0] - 1) // self.tile[0]
        ty = (res.height + self.tile[1] - 1) // self.tile[1]
        ranges = torch.empty((tx * ty, 2), dtype=torch.int32, device=dev)
        rec = torch.empty((max(res.n, 1), 12), dtype=torch.float32, device=dev)
        abi.r4g_frame_export(self.ctx, res.frame.data_ptr(), res.frame.numel(), res.n, res.width,
                             res.height, None, keys.data_ptr(), vals.data_ptr(), ranges.data_ptr(),
                             rec.data_ptr(), s)
        return {"key_count": k, "keys": keys[:k], "values": vals[:k], "ranges": ranges, "records": rec[:res.n]}


class Render4DFunction(torch.autograd.Function):
    """image = render(mean, rotor, logscale, logit, sh; camera, t) with a
    hand-written CUDA backward (r4g_render_backward)."""

    @staticmethod
    def forward(ctx, mean, rotor, logscale, logit, sh, renderer: Renderer, cam, t: float):
        params = {"mean": mean.detach(), "rotor": rotor.detach(), "logscale": logscale.detach(),
                  "logit": logit.detach(), "sh": sh.detach()}
        res, ctx.pending = renderer.render_deferred(params, cam, t)
        ctx.renderer, ctx.cam, ctx.t, ctx.res = renderer, cam, t, res
        ctx.save_for_backward(mean, rotor, logscale, logit, sh)
        return res.image

    @staticmethod
    def backward(ctx, grad_image):
        mean, rotor, logscale, logit, sh = ctx.saved_tensors
        ctx.renderer.settle(ctx.pending, ctx.res)
        params = {"mean": mean, "rotor": rotor, "logscale": logscale, "logit": logit, "sh": sh}
        grads = {k: torch.zeros(v.shape, dtype=torch.float32, device=v.device) for k, v in params.items()}
        ctx.renderer.backward(params, ctx.cam, ctx.t, ctx.res, grad_image.float(), grads)
        out = [grads[k].to(params[k].dtype) for k in PARAM_NAMES]
        return (*out, None, None, None)


class Render4DBatchFunction(torch.autograd.Function):
    """packed images of V views = render_batch(mean, ..., sh; views) with the
    batched CUDA backward (r4g_render_batch_backward)."""

    @staticmethod
    def forward(ctx, mean, rotor, logscale, logit, sh, renderer: Renderer, views):
        params = {"mean": mean.detach(), "rotor": rotor.detach(), "logscale": logscale.detach(),
                  "logit": logit.detach(), "sh": sh.detach()}
        res, ctx.pending = renderer.render_batch_deferred(params, views)
        ctx.renderer, ctx.res = renderer, res
        ctx.save_for_backward(mean, rotor, logscale, logit, sh)
        return res.packed

    @staticmethod
    def backward(ctx, grad_packed):
        mean, rotor, logscale, logit, sh = ctx.saved_tensors
        ctx.renderer.settle(ctx.pending, ctx.res)
        params = {"mean": mean, "rotor": rotor, "logscale": logscale, "logit": logit, "sh": sh}
        grads = {k: torch.zeros(v.shape, dtype=torch.float32, device=v.device) for k, v in params.items()}
        ctx.renderer.backward_batch(params, ctx.res, grad_packed.float(), grads)
        out = [grads[k].to(params[k].dtype) for k in PARAM_NAMES]
        return (*out, None, None)


def views_tensor(structs, device) -> torch.Tensor:
    """Device copy (uint8 bytes) of r4g_view structs, for ``views_dev``."""
    arr = abi.view_array(structs)
    host = torch.frombuffer(bytearray(bytes(arr)), dtype=torch.uint8)
    return host.to(device)


class BatchGraph:
    """One batched render, and optionally its backward, captured in a CUDA
    graph. The cameras and times live in a device table the kernels read, so
    :meth:`replay` can take new views of the same image sizes. ``grad_fn``
    (optional) maps the packed image to dL/d(packed image) with torch ops; it
    is captured too. Gradients accumulate into ``self.grads`` (zeroed inside
    the graph before the backward)."""

    def __init__(self, renderer: Renderer, params: dict, views, key_capacity: int | None = None,
                 grad_fn=None):
        self.r = renderer
        self.params = params
        self.structs = renderer.view_structs(views)
        dev = params["mean"].device
        first = renderer.render_batch(params, self.structs, key_capacity=key_capacity)  # sizes the key buffer
        self.cap = first.key_capacity if key_capacity else int(renderer.status_of(first)[1] * 1.2) + 4096
        self.views_dev = views_tensor(self.structs, dev)
        self.frame = torch.empty(renderer.batch_frame_bytes(first.n, self.structs, self.cap), dtype=torch.uint8,
                                 device=dev)
        self.packed = torch.empty_like(first.packed)
        self.grad_fn = grad_fn
        self.grads = {k: torch.zeros(v.shape, dtype=torch.float32, device=dev) for k, v in params.items()} \
            if grad_fn is not None else None
        side = torch.cuda.Stream(dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):
            for _ in range(2):  # warm up outside the capture
                self._body(side)
        torch.cuda.current_stream(dev).wait_stream(side)
        torch.cuda.synchronize(dev)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._body(torch.cuda.current_stream(dev))
        self.images = _packed_views(self.packed, self.structs)

    def _body(self, stream) -> None:
        res = self.r.render_batch(self.params, self.structs, frame=self.frame, key_capacity=self.cap,
                                  out=self.packed, views_dev=self.views_dev, check=False, stream=stream)
        if self.grad_fn is not None:
            for v in self.grads.values():
                v.zero_()
            gp = self.grad_fn(self.packed)
            self.r.backward_batch(self.params, res, gp, self.grads, stream=stream)

    def views_table(self, views) -> torch.Tensor:
        """Device copy of new (camera, t) views of the captured sizes, for
        :meth:`replay` (build these ahead of a timed loop)."""
        structs = self.r.view_structs(views)
        if [(v.cam.width, v.cam.height) for v in structs] != [(v.cam.width, v.cam.height) for v in self.structs]:
            raise ValueError("replayed views must keep the captured image sizes")
        return views_tensor(structs, self.views_dev.device)

    def replay(self, views=None, table: torch.Tensor | None = None) -> None:
        """Run the graph, with new (camera, t) views of the same sizes if given
        (``views``, copied from host memory, or a device ``table`` from
        :meth:`views_table`, copied on the stream)."""
        if views is not None:
            table = self.views_table(views)
        if table is not None:
            self.views_dev.copy_(table)
        self.graph.replay()

    def status(self) -> tuple[int, int]:
        """(status, keys needed) of the last replay (waits for the stream)."""
        s = torch.cuda.current_stream(self.frame.device).cuda_stream
        return abi.r4g_frame_status(self.r.ctx, self.frame.data_ptr(), self.frame.numel(), s)


_default: Renderer | None = None


def default_renderer() -> Renderer:
    global _default
    if _default is None:
        _default = Renderer()
    return _default


_flow: Renderer | None = None


def render_flow(params: dict, cam, t: float, renderer: Renderer | None = None) -> torch.Tensor:
    """Optical-flow render (R4G_FLAG_FLOW): [2, H, W] image-plane velocity of
    the sliced centres, d(mean2d)/dt, composited with the colour weights."""
    global _flow
    if renderer is None:
        if _flow is None:
            _flow = Renderer(flags=abi.R4G_FLAG_FLOW)
        renderer = _flow
    return renderer.render(params, cam, t).image[:2]


def render_batch(params: dict, views, renderer: Renderer | None = None) -> torch.Tensor:
    """Differentiable batched render -> packed images of all views."""
    r = renderer or default_renderer()
    return Render4DBatchFunction.apply(params["mean"], params["rotor"], params["logscale"], params["logit"],
                                       params["sh"], r, list(views))


def render(params: dict, cam, t: float, renderer: Renderer | None = None) -> torch.Tensor:
    """Differentiable render of ``params`` (dict of CUDA tensors) -> [3, H, W]."""
    r = renderer or default_renderer()
    return Render4DFunction.apply(params["mean"], params["rotor"], params["logscale"], params["logit"],
                                  params["sh"], r, cam, t)


def knn4d(means: torch.Tensor, scale_xyz: float, scale_t: float, k: int = 8, with_dist: bool = False):
    """K nearest neighbours of the 4D means ([N, 4] float32 CUDA) after
    dividing x, y, z by scale_xyz and t by scale_t (r4g_knn4d). Returns int32
    [N, k] (and the squared scaled distances [N, k] with ``with_dist``)."""
    m = means.contiguous()
    if m.dtype != torch.float32 or m.dim() != 2 or m.shape[1] != 4 or not m.is_cuda:
        raise ValueError("means must be a float32 CUDA tensor [N, 4]")
    n = int(m.shape[0])
    idx = torch.empty((n, k), dtype=torch.int32, device=m.device)
    d2 = torch.empty((n, k), dtype=torch.float32, device=m.device) if with_dist else None
    nb = abi.r4g_knn_scratch_bytes(n)
    scratch = torch.empty(nb, dtype=torch.uint8, device=m.device)
    s = torch.cuda.current_stream(m.device).cuda_stream
    abi.r4g_knn4d(m.data_ptr(), n, float(scale_xyz), float(scale_t), int(k), idx.data_ptr(),
                  d2.data_ptr() if d2 is not None else None, scratch.data_ptr(), nb, s)
    if abi.r4g_knn_status(scratch.data_ptr(), n, s) != abi.R4G_OK:
        raise abi.R4GError(abi.R4G_ETIMEOUT, "knn sort wait gave up")
    return (idx, d2) if with_dist else idx


def regularizers(params: dict, knn_idx: torch.Tensor, lambda_entropy: float = 1.0,
                 lambda_consistency: float = 1.0, grads: dict | None = None) -> torch.Tensor:
    """(L_entropy, L_consistent4D) as a float32 CUDA tensor [2]; with ``grads``
    (float32 tensors shaped like the parameters) adds lambda-weighted
    gradients into grads['logit'], grads['rotor'] and grads['logscale']."""
    g = gaussians_struct(params)
    k = int(knn_idx.shape[1])
    idx = knn_idx.contiguous()
    if idx.dtype != torch.int32 or idx.shape[0] != g.n:
        raise ValueError("knn_idx must be int32 [N, k]")
    dev = params["mean"].device
    loss = torch.empty(2, dtype=torch.float32, device=dev)
    gs = None
    if grads is not None:
        gs = abi.r4g_grads()
        for name in PARAM_NAMES:
            setattr(gs, name, grads[name].data_ptr())
    nb = abi.r4g_regularizers_scratch_bytes(g.n)
    scratch = torch.empty(nb, dtype=torch.uint8, device=dev)
    s = torch.cuda.current_stream(dev).cuda_stream
    abi.r4g_regularizers(g, idx.data_ptr(), k, float(lambda_entropy), float(lambda_consistency), loss.data_ptr(),
                         gs, scratch.data_ptr(), nb, s)
    return loss


def image_loss(image: torch.Tensor, target: torch.Tensor, lambda_ssim: float = 0.2, with_grad: bool = True):
    """(L, L1, SSIM) as a float32 CUDA tensor [3] and, with ``with_grad``,
    dL/d image (r4g_image_loss: (1 - lambda) L1 + lambda (1 - SSIM))."""
    x, y = image.contiguous(), target.contiguous()
    if x.shape != y.shape or x.dim() != 3 or x.dtype != torch.float32 or y.dtype != torch.float32:
        raise ValueError("image and target must be float32 [C, H, W] of one shape")
    c, h, w = (int(v) for v in x.shape)
    out = torch.empty(3, dtype=torch.float32, device=x.device)
    grad = torch.empty_like(x) if with_grad else None
    nb = abi.r4g_image_loss_scratch_bytes(c, h, w)
    scratch = torch.empty(nb, dtype=torch.uint8, device=x.device)
    s = torch.cuda.current_stream(x.device).cuda_stream
    abi.r4g_image_loss(x.data_ptr(), y.data_ptr(), c, h, w, float(lambda_ssim), out.data_ptr(),
                       grad.data_ptr() if grad is not None else None, scratch.data_ptr(), nb, s)
    return (out, grad) if with_grad else out


def sort_pairs(keys: torch.Tensor, values: torch.Tensor, begin_bit: int = 0, end_bit: int = 64):
    """Stable radix sort of (int64 key as uint64 bits, int32 value) pairs on bits
    [begin_bit, end_bit) with the library's kernels. Returns new tensors."""
    n = int(keys.numel())
    ko = torch.empty_like(keys)
    vo = torch.empty_like(values)
    if n == 0:
        return ko, vo
    nb = abi.r4g_sort_scratch_bytes(n)
    scratch = torch.empty(nb, dtype=torch.uint8, device=keys.device)
    s = torch.cuda.current_stream(keys.device).cuda_stream
    abi.r4g_sort_pairs(keys.data_ptr(), values.data_ptr(), ko.data_ptr(), vo.data_ptr(), n, begin_bit,
                       end_bit, scratch.data_ptr(), nb, s)
    return ko, vo


def sort32(keys: torch.Tensor, values: torch.Tensor | None = None, bits: int = 32):
    """Stable radix sort of (int32 key as uint32 bits, int32 value) pairs on
    key bits [0, bits) with the render's own sort kernels (r4g_sort32);
    ``values`` None sorts the positions 0..n-1. Returns new tensors; raises
    R4GError if a look-back wait gave up (r4g_sort32_status)."""
    n = int(keys.numel())
    ko = torch.empty_like(keys)
    vo = torch.empty(n, dtype=torch.int32, device=keys.device)
    nb = abi.r4g_sort32_scratch_bytes(n, bits)
    scratch = torch.empty(nb, dtype=torch.uint8, device=keys.device)
    s = torch.cuda.current_stream(keys.device).cuda_stream
    abi.r4g_sort32(keys.data_ptr(), values.data_ptr() if values is not None else None, ko.data_ptr(), vo.data_ptr(),
                   n, bits, scratch.data_ptr(), nb, s)
    abi.check(abi.lib().r4g_sort32_status(scratch.data_ptr(), s))
    return ko, vo


def densify_config(grad_threshold: float = 2e-4, dense_scale: float = 0.06, split_divisor: float = 1.6,
                   min_opacity: float = 0.005, max_scale: float = 0.0,
                   max_screen_radius: float = 0.0) -> abi.r4g_densify_config:
    """r4g_densify_config; the defaults are the paper's Plenoptic threshold and
    the 3D Gaussian Splatting rules (dense_scale = 0.01 x a scene extent of 6)."""
    c = abi.r4g_densify_config()
    c.grad_threshold, c.dense_scale, c.split_divisor = float(grad_threshold), float(dense_scale), float(split_divisor)
    c.min_opacity, c.max_scale, c.max_screen_radius = float(min_opacity), float(max_scale), float(max_screen_radius)
    return c


def densify(params: dict, stats: dict, z: torch.Tensor, cfg: abi.r4g_densify_config | None = None):
    """One densify-and-prune step (r4g_densify_plan + r4g_densify_apply).
    ``z``: float32 [N, 2, 4] standard normal draws for the split children.
    Returns (new params dict, int32 [M] source map: i for a row continuing
    Gaussian i, -(i + 1) for a new row). Reads the row count back to the host
    to size the outputs."""
    cfg = cfg or densify_config()
    g = gaussians_struct(params)
    dev = params["mean"].device
    zz = z.contiguous()
    if zz.dtype != torch.float32 or tuple(zz.shape) != (g.n, 2, 4):
        raise ValueError("z must be float32 [N, 2, 4]")
    for k in ("vs_grad", "vs_count"):
        if k not in stats:
            raise ValueError(f"stats needs {k}")
    rad = stats.get("max_radius")
    nb = abi.r4g_densify_scratch_bytes(g.n)
    scratch = torch.empty(max(nb, 1), dtype=torch.uint8, device=dev)
    count = torch.zeros(1, dtype=torch.int64, device=dev)
    s = torch.cuda.current_stream(dev).cuda_stream
    abi.r4g_densify_plan(g, stats["vs_grad"].data_ptr(), stats["vs_count"].data_ptr(),
                         rad.data_ptr() if rad is not None else None, cfg, scratch.data_ptr(), nb,
                         count.data_ptr(), s)
    m = int(count.item())
    new = {"mean": torch.empty((m, 4), dtype=torch.float32, device=dev),
           "rotor": torch.empty((m, 8), dtype=torch.float32, device=dev),
           "logscale": torch.empty((m, 4), dtype=torch.float32, device=dev),
           "logit": torch.empty((m,), dtype=torch.float32, device=dev),
           "sh": torch.empty((m, 16, 3), dtype=torch.float32, device=dev)}
    src = torch.empty(m, dtype=torch.int32, device=dev)
    out = abi.r4g_params_out()
    for k in PARAM_NAMES:
        setattr(out, k, new[k].data_ptr())
    abi.r4g_densify_apply(g, zz.data_ptr(), cfg, scratch.data_ptr(), nb, out, m, src.data_ptr(), s)
    return new, src


def opacity_reset(params: dict, max_opacity: float = 0.01) -> None:
    """In place: opacity = min(opacity, max_opacity) (r4g_opacity_reset)."""
    lg = params["logit"]
    if lg.dtype != torch.float32 or not lg.is_contiguous() or not lg.is_cuda:
        raise ValueError("logit must be a contiguous float32 CUDA tensor")
    abi.r4g_opacity_reset(lg.data_ptr(), int(lg.numel()), float(max_opacity),
                          torch.cuda.current_stream(lg.device).cuda_stream)
