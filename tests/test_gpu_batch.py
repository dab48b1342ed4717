"""Batched multi-view render and backward (r4g_render_batch / _backward):
each view of a batch must be bit-identical to the single-view render of that
view (the same per-item arithmetic, the same depth order within a view, the
same blend); the batched gradient equals the sum of the single-view
gradients up to float summation order, and matches the FP64 oracle's
gradient summed over the views (tolerance as in test_gpu_backward). A CUDA
graph of the batch replayed with new device-side views gives the same bits
as a direct call; the tile autotuner picks a shape without changing the
image."""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import ambiguous, to_device

pytestmark = pytest.mark.gpu
NAMES = ("mean", "rotor", "logscale", "logit", "sh")


@pytest.fixture(scope="module")
def r4g():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2402_03307_gb300 as m
    return m


def _uneven_views(seed, sizes, radius=4.0):
    rng = np.random.default_rng(seed)
    out = []
    for w, h in sizes:
        a = rng.uniform(0.0, 2.0 * math.pi)
        eye = (radius * math.sin(a), 0.3 * rng.uniform(-1, 1), -radius * math.cos(a))
        out.append((synth.look_at(eye, (0.0, 0.0, 0.0), w, h), float(np.float32(rng.uniform(0.0, 1.0)))))
    return out


SIZES = [(128, 128), (96, 64), (37, 29), (200, 120), (64, 64), (1, 1)]


def _zeros_like(p):
    return {k: torch.zeros(v.shape, dtype=torch.float32, device=v.device) for k, v in p.items()}


def test_batch_images_equal_single_views(r4g):
    g, _, _ = synth.small_scene(seed=41)
    p = to_device(g)
    views = _uneven_views(1, SIZES)
    rend = r4g.Renderer()
    res = rend.render_batch(p, views)
    for (cam, t), img in zip(views, res.images):
        single = rend.render(p, cam, t).image
        assert torch.equal(single, img), (cam.width, cam.height)


def test_batch_full_size_mixed_resolutions(r4g):
    """100k Gaussians, 16 views of 800x800, 640x480 and 1352x1014."""
    g = synth.gaussians(100_000, 5, mean_lo=-3.0, mean_hi=3.0)
    p = to_device(g)
    views = synth.batched_views(6)
    rend = r4g.Renderer()
    res = rend.render_batch(p, views)
    st, need = rend.status(res)
    assert st == 0 and need > 0
    for k in (0, 5, 10, 15):
        cam, t = views[k]
        assert torch.equal(rend.render(p, cam, t).image, res.images[k]), k


def test_batch_three_tile_sort_passes(r4g):
    """Four 1352x1014 views at 8x8 tiles: 85,852 tiles, tile ids of 17 bits,
    so the tile sort takes three radix passes (the emission's, then two
    onesweep passes) instead of the emission's and the grouped second pass;
    every view's image equals its single-view 16x16 render bit for bit."""
    g = synth.gaussians(100_000, 5, mean_lo=-3.0, mean_hi=3.0)
    p = to_device(g)
    views = [synth.orbit_camera(k, 300, 8.0, 1352, 1014) for k in (5, 80, 150, 230)]
    rend = r4g.Renderer(tile=(8, 8))
    res = rend.render_batch(p, views)
    st, need = rend.status(res)
    assert st == 0 and need > 0
    for k, (cam, t) in enumerate(views):
        assert torch.equal(r4g.Renderer().render(p, cam, t).image, res.images[k]), k


def test_batch_tile_shapes_and_autotune(r4g):
    g, _, _ = synth.small_scene(seed=42)
    p = to_device(g)
    views = _uneven_views(2, SIZES[:4])
    ref = r4g.Renderer().render_batch(p, views).packed
    for tile in ((8, 8), (16, 32)):
        assert torch.equal(r4g.Renderer(tile=tile).render_batch(p, views).packed, ref), tile
    rend = r4g.Renderer()
    out = rend.autotune(p, views, backward=True, reps=2)
    assert tuple(out["tile"]) in ((8, 8), (16, 16), (16, 32))
    assert any(v is not None and v > 0 for v in out["ms"].values())
    assert rend.tile == tuple(out["tile"])
    assert torch.equal(rend.render_batch(p, views).packed, ref)


@pytest.mark.parametrize("fp64", [False, True])
def test_batch_backward_equals_sum_of_views(r4g, fp64):
    """Both multi-view backward paths: the two-pass FP32 one (items, then
    Gaussians) and the one-pass FP64 debug one."""
    g, _, _ = synth.small_scene(seed=43)
    p = to_device(g)
    views = _uneven_views(3, SIZES[:5])
    rend = r4g.Renderer(bg=(0.2, 0.4, 0.6), flags=r4g.abi.R4G_FLAG_FP64_SLICE if fp64 else 0)
    res = rend.render_batch(p, views)
    w = torch.as_tensor(np.random.default_rng(0).normal(0, 1, res.packed.numel()).astype(np.float32)).cuda()
    gb = _zeros_like(p)
    rend.backward_batch(p, res, w, gb)
    gs = _zeros_like(p)
    off = 0
    for cam, t in views:
        n = 3 * cam.width * cam.height
        r1 = rend.render(p, cam, t)
        rend.backward(p, cam, t, r1, w[off:off + n].view(3, cam.height, cam.width), gs)
        off += n
    torch.cuda.synchronize()
    for k in NAMES:
        a, b = gb[k].double(), gs[k].double()
        rel = (a - b).norm() / b.norm()
        assert rel < 1e-5, (k, float(rel))


def test_batch_backward_oracle(r4g):
    g, _, _ = synth.small_scene(seed=44, n=300)
    views = _uneven_views(4, [(48, 40), (40, 32)])
    p = to_device(g)
    gd = oracle.to_f64(g)
    ws, ref = [], None
    for k, (cam, t) in enumerate(views):
        r = oracle.render(gd, cam, t)
        w = np.random.default_rng(10 + k).normal(0, 1, (3, cam.height, cam.width))
        w[:, ambiguous(r, image=False)] = 0.0
        w = w.astype(np.float32)
        ws.append(w.reshape(-1))
        gr = oracle.render_grad(gd, cam, t, w)
        ref = {n: gr[n].clone() for n in NAMES} if ref is None else {n: ref[n] + gr[n] for n in NAMES}
    rend = r4g.Renderer()
    res = rend.render_batch(p, views)
    got = _zeros_like(p)
    rend.backward_batch(p, res, torch.as_tensor(np.concatenate(ws)).cuda(), got)
    torch.cuda.synchronize()
    for k in NAMES:
        a = got[k].double().cpu().numpy().reshape(-1)
        b = ref[k].numpy().reshape(-1)
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        assert rel <= 1e-2, (k, rel)
        bad = np.abs(a - b) > 1e-2 * (np.abs(b) + 1e-3 * np.abs(b).max())
        assert bad.mean() <= 1e-3, (k, bad.mean())


def test_batch_autograd_function(r4g):
    g, _, _ = synth.small_scene(seed=45)
    p = to_device(g)
    views = _uneven_views(5, SIZES[:3])
    rend = r4g.Renderer()
    leaves = {k: v.clone().requires_grad_(True) for k, v in p.items()}
    packed = r4g.render_batch(leaves, views, renderer=rend)
    w = torch.linspace(-1, 1, packed.numel(), device="cuda")
    (packed * w).sum().backward()
    res = rend.render_batch(p, views)
    ref = _zeros_like(p)
    rend.backward_batch(p, res, w, ref)
    for k in NAMES:
        assert torch.equal(leaves[k].grad, ref[k]), k


def test_batch_graph_replay_new_views(r4g):
    g, _, _ = synth.small_scene(seed=46)
    p = to_device(g)
    views = _uneven_views(6, SIZES[:4])
    rend = r4g.Renderer()
    target = torch.full((sum(3 * c.width * c.height for c, _ in views),), 0.25, device="cuda")
    graph = r4g.BatchGraph(rend, p, views, key_capacity=1 << 16,
                           grad_fn=lambda img: torch.sign(img - target) * 1e-3)
    for seed in (7, 8):
        new = _uneven_views(seed, SIZES[:4])
        graph.replay(new)
        torch.cuda.synchronize()
        assert graph.status()[0] == 0
        direct = rend.render_batch(p, new, key_capacity=graph.cap)
        assert torch.equal(graph.packed, direct.packed), seed
        ref = _zeros_like(p)
        rend.backward_batch(p, direct, torch.sign(direct.packed - target) * 1e-3, ref)
        for k in NAMES:
            assert torch.equal(graph.grads[k], ref[k]), (seed, k)


def test_batch_overflow_retry(r4g):
    g, _, _ = synth.small_scene(seed=47)
    p = to_device(g)
    views = _uneven_views(9, SIZES[:3])
    rend = r4g.Renderer()
    small = rend.render_batch(p, views, key_capacity=64, check=False)
    st, need = rend.status(small)
    assert st == r4g.abi.R4G_EOVERFLOW and need > 64
    res = rend.render_batch(p, views, key_capacity=64)  # retries with a larger key buffer
    assert res.key_capacity >= need
    assert torch.equal(res.packed, rend.render_batch(p, views).packed)


def test_autograd_deferred_status(r4g):
    """The autograd functions check a render's key capacity without stalling:
    the first render of a size waits (and sizes the key buffer), later ones
    are checked by the backward, which raises on an overflow and grows the
    capacity so that the repeated step succeeds."""
    g, cam, t = synth.small_scene(seed=49)
    p = to_device(g)
    views = _uneven_views(12, SIZES[:3])
    rend = r4g.Renderer()
    leaves = {k: v.clone().requires_grad_(True) for k, v in p.items()}
    for _ in range(2):  # checked on the first call, deferred on the second
        r4g.render_batch(leaves, views, renderer=rend).sum().backward()
    key = next(k for k in rend._cap_hint if isinstance(k[1], tuple))
    rend._cap_hint[key] = 64  # too small for this scene
    for v in leaves.values():
        v.grad = None
    with pytest.raises(r4g.abi.R4GError) as e:
        r4g.render_batch(leaves, views, renderer=rend).sum().backward()
    assert e.value.status == r4g.abi.R4G_EOVERFLOW and rend._cap_hint[key] > 64
    for v in leaves.values():
        v.grad = None
    packed = r4g.render_batch(leaves, views, renderer=rend)
    assert torch.equal(packed.detach(), rend.render_batch(p, views).packed)
    packed.sum().backward()
    ref = _zeros_like(p)
    rend.backward_batch(p, rend.render_batch(p, views), torch.ones_like(packed), ref)
    for k in NAMES:
        assert torch.equal(leaves[k].grad, ref[k]), k
    # the single-view function the same way
    one = r4g.Renderer()
    img = r4g.render(leaves, cam, t, renderer=one)
    img.sum().backward()
    one._cap_hint[(1000, cam.width, cam.height)] = 64
    with pytest.raises(r4g.abi.R4GError):
        r4g.render(leaves, cam, t, renderer=one).sum().backward()
    r4g.render(leaves, cam, t, renderer=one).sum().backward()


def test_batch_limits_and_device_view_mismatch(r4g):
    g, _, _ = synth.small_scene(seed=48)
    p = to_device(g)
    rend = r4g.Renderer()
    views = _uneven_views(10, [(16, 16)] * 65)
    with pytest.raises(r4g.abi.R4GError):
        rend.render_batch(p, views)
    views = _uneven_views(11, [(32, 32), (16, 16)])
    wrong = rend.view_structs(_uneven_views(11, [(32, 32), (16, 8)]))
    vd = r4g.views_tensor(wrong, "cuda")
    with pytest.raises(r4g.abi.R4GError) as e:
        rend.render_batch(p, views, views_dev=vd)
    assert e.value.status == r4g.abi.R4G_EDEVICE
