"""Pins of the oracle's image loss (Sec. 3.3 total loss: L1 and SSIM, as in
3D Gaussian Splatting): the conv2d SSIM map against explicit window sums;
SSIM(x, x) = 1; constant images away from the border reduce to
(2ab + C1)/(a^2 + b^2 + C1); the L1 part and the gradient against central
differences."""
import numpy as np
import torch

from oracle import imageloss as il


def _imgs(seed, c=3, h=17, w=23):
    rng = np.random.default_rng(seed)
    return (torch.as_tensor(rng.uniform(0, 1, (c, h, w))), torch.as_tensor(rng.uniform(0, 1, (c, h, w))))


def test_ssim_map_matches_window_sums():
    x, y = _imgs(0, c=2, h=13, w=16)
    assert torch.allclose(il.ssim_map(x, y), il.ssim_brute(x, y), rtol=1e-12, atol=1e-12)


def test_ssim_of_an_image_with_itself_is_one():
    x, _ = _imgs(1)
    assert torch.allclose(il.ssim_map(x, x), torch.ones_like(x), atol=1e-12)


def test_constant_images_interior():
    a, b = 0.3, 0.7
    x = torch.full((1, 30, 30), a, dtype=torch.float64)
    y = torch.full((1, 30, 30), b, dtype=torch.float64)
    m = il.ssim_map(x, y)[0, 5:-5, 5:-5]  # every window inside the image
    want = (2 * a * b + il.C1) / (a * a + b * b + il.C1)
    assert torch.allclose(m, torch.full_like(m, want), rtol=1e-12)


def test_loss_parts_and_gradient():
    x, y = _imgs(2, c=3, h=12, w=14)
    out = il.image_loss(x, y, 0.2)
    assert abs(float(out["l1"]) - float((x - y).abs().mean())) < 1e-15
    want = 0.8 * float(out["l1"]) + 0.2 * (1 - float(out["ssim"]))
    assert abs(float(out["loss"]) - want) < 1e-15
    rng = np.random.default_rng(3)
    for flat in rng.choice(x.numel(), 8, replace=False):
        h = 1e-6
        xp, xm = x.clone(), x.clone()
        xp.view(-1)[flat] += h
        xm.view(-1)[flat] -= h
        fd = (float(il.image_loss(xp, y)["loss"]) - float(il.image_loss(xm, y)["loss"])) / (2 * h)
        assert abs(fd - float(out["grad"].view(-1)[flat])) < 1e-7
