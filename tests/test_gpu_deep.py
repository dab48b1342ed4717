"""Full-size checks of the 300k-Gaussian 1352x1014 frame where the lists are
deep (about a hundred composited Gaussians per pixel):

* the backward against the oracle's gradient with the upstream gradient
  non-zero on two 64x64 blocks only: the back-to-front recovery of the
  transmittance T_i = T_{i+1} / (1 - alpha_i) runs through the whole depth of
  each pixel's list, the regime of the training configuration. The oracle
  composites each block over the Gaussians whose 3-sigma box meets it (every
  other Gaussian fails the cutoff at every pixel of the block), in its global
  depth order;
* the render's own radix sorts, bit for bit: the exported (tile | depth) keys
  and Gaussian indices must equal their own stable order (np.lexsort by key,
  then by index), each key's depth bits must be its Gaussian's depth, every
  Gaussian's pairs must form one interval of columns in each of consecutive
  tile rows and each tile's range must hold exactly its pairs."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import ambiguous, block_pixels, box_keep, compare_grads, to_device

pytestmark = pytest.mark.gpu
W, H = 1352, 1014
BLOCK = 64


@pytest.fixture(scope="module")
def r4g():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2402_03307_gb300 as m
    return m


@pytest.fixture(scope="module")
def scene():
    return synth.fwd300k_scene()


def _blocks(seed):
    rng = np.random.default_rng(seed)
    return [(int(rng.integers(300, W - 300 - BLOCK)), int(rng.integers(200, H - 200 - BLOCK))) for _ in range(2)]


@pytest.mark.parametrize("rho,frame,seed", [(8.0, 37, 61), (4.0, 120, 62)])
def test_backward_deep_lists(r4g, scene, rho, frame, seed):
    g = scene
    cam, t = synth.orbit_camera(frame, 300, rho, W, H)
    sc = oracle.to_f64(g)
    rec = oracle.preprocess(sc, cam, t)
    blocks = _blocks(seed)
    pix = np.concatenate([block_pixels(x0, y0, BLOCK, BLOCK) for x0, y0 in blocks])
    keep = np.zeros(len(g["logit"]), bool)
    for x0, y0 in blocks:
        keep |= box_keep(rec, x0, y0, BLOCK, BLOCK)
    idx = torch.as_tensor(np.nonzero(keep)[0])
    n = rec["visible"].numel()
    sub = {k: (v[idx] if torch.is_tensor(v) and v.dim() > 0 and v.shape[0] == n else v) for k, v in rec.items()}
    ref = oracle.render_pixels(None, cam, t, pix, rec=sub)
    depth = ref["n_composited"].double()
    print(f"radius {rho} frame {frame}: {int(keep.sum())} Gaussians meet the blocks; composited per pixel "
          f"mean {float(depth.mean()):.1f}, max {int(depth.max())}")
    assert float(depth.mean()) >= 50  # the deep-list regime
    amb = ambiguous(ref, image=False)
    assert amb.mean() < 0.01, amb.mean()
    w = np.random.default_rng(seed).normal(0, 1, (len(pix), 3))
    w[amb] = 0.0
    w = w.astype(np.float32)
    gr = oracle.render_grad_pixels(sc, cam, t, pix, w.astype(np.float64), keep=keep)
    grad_img = np.zeros((3, H, W), np.float32)
    grad_img[:, pix[:, 1], pix[:, 0]] = w.T
    rend = r4g.Renderer()
    p = to_device(g)
    res = rend.render(p, cam, t)
    grads = {k: torch.zeros(v.shape, dtype=torch.float32, device="cuda") for k, v in p.items()}
    rend.backward(p, cam, t, res, torch.as_tensor(grad_img).cuda(), grads)
    torch.cuda.synchronize()
    got = {k: v.double().cpu().numpy() for k, v in grads.items()}
    rel = compare_grads(got, gr, f"deep r{rho}")
    print(f"radius {rho} frame {frame} backward: relative L2 error per group "
          + ", ".join(f"{k} {v:.2e}" for k, v in rel.items()))


@pytest.mark.parametrize("rho,frame", [(8.0, 37), (4.0, 120)])
def test_render_sort_bit_exact_full_size(r4g, scene, rho, frame):
    from test_gpu_forward import _rectangles_check
    cam, t = synth.orbit_camera(frame, 300, rho, W, H)
    rend = r4g.Renderer()
    res = rend.render(to_device(scene), cam, t)
    ex = rend.export(res)
    keys = ex["keys"].cpu().numpy().view(np.uint64)
    vals = ex["values"].cpu().numpy().view(np.uint32)
    rec = ex["records"].cpu().numpy()
    assert ex["key_count"] > 1_500_000
    order = np.lexsort((vals, keys))  # by key, ties by Gaussian index
    assert np.array_equal(keys[order], keys)
    assert np.array_equal(vals[order], vals)
    assert np.array_equal((keys & np.uint64(0xFFFFFFFF)).astype(np.uint32), rec[vals, 6].view(np.uint32))
    _rectangles_check(ex, (W + 15) // 16)
    print(f"radius {rho} frame {frame}: {ex['key_count']} pairs in stable key order")
