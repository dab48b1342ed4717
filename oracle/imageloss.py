"""The image loss of the optimisation (Sec. 3.3 total loss, following 3D
Gaussian Splatting): L = (1 - lambda) L1 + lambda (1 - SSIM), plain FP64.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``.

SSIM is the structural similarity of Wang et al. (2004) with the window of
3D Gaussian Splatting: an 11 x 11 Gaussian of standard deviation 1.5
(normalised to sum 1), zero padding at the border, C1 = 0.01^2,
C2 = 0.03^2, per channel, averaged over every pixel and channel:
  mu_x = G * x,  sigma_x^2 = G * x^2 - mu_x^2,  sigma_xy = G * (x y) - mu_x mu_y,
  SSIM = (2 mu_x mu_y + C1)(2 sigma_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(sigma_x^2 + sigma_y^2 + C2)).
L1 = mean |x - y|. The gradient with respect to x is torch.autograd's.
"""
from __future__ import annotations

import math

import torch
import torch.nn.functional as F

WINDOW = 11
SIGMA = 1.5
C1 = 0.01 ** 2
C2 = 0.03 ** 2


def window_1d() -> torch.Tensor:
    k = torch.arange(WINDOW, dtype=torch.float64) - WINDOW // 2
    g = torch.exp(-(k * k) / (2.0 * SIGMA * SIGMA))
    return g / g.sum()


def _filter(img: torch.Tensor) -> torch.Tensor:
    """G * img for img [C, H, W] (the 2D window is the outer product)."""
    g = window_1d()
    w2 = (g[:, None] * g[None, :])[None, None].repeat(img.shape[0], 1, 1, 1)
    return F.conv2d(img[None], w2, padding=WINDOW // 2, groups=img.shape[0])[0]


def ssim_map(x: torch.Tensor, y: torch.Tensor) -> torch.Tensor:
    mx, my = _filter(x), _filter(y)
    sxx = _filter(x * x) - mx * mx
    syy = _filter(y * y) - my * my
    sxy = _filter(x * y) - mx * my
    return ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))


def image_loss(x, y, lam: float = 0.2) -> dict:
    """{"loss", "l1", "ssim", "grad"} for images [C, H, W] (grad = dL/dx)."""
    xt = torch.as_tensor(x, dtype=torch.float64).clone().requires_grad_(True)
    yt = torch.as_tensor(y, dtype=torch.float64)
    l1 = (xt - yt).abs().mean()
    ss = ssim_map(xt, yt).mean()
    loss = (1.0 - lam) * l1 + lam * (1.0 - ss)
    loss.backward()
    return {"loss": loss.detach(), "l1": l1.detach(), "ssim": ss.detach(), "grad": xt.grad.detach()}


def ssim_brute(x: torch.Tensor, y: torch.Tensor) -> torch.Tensor:
    """The same SSIM map by explicit sums over each pixel's window (small images)."""
    g = window_1d()
    C, H, W = x.shape
    r = WINDOW // 2
    out = torch.zeros((C, H, W), dtype=torch.float64)
    for c in range(C):
        for i in range(H):
            for j in range(W):
                s = {"x": 0.0, "y": 0.0, "xx": 0.0, "yy": 0.0, "xy": 0.0}
                for a in range(-r, r + 1):
                    for b in range(-r, r + 1):
                        ii, jj = i + a, j + b
                        if 0 <= ii < H and 0 <= jj < W:
                            w = float(g[a + r] * g[b + r])
                            xv, yv = float(x[c, ii, jj]), float(y[c, ii, jj])
                            s["x"] += w * xv
                            s["y"] += w * yv
                            s["xx"] += w * xv * xv
                            s["yy"] += w * yv * yv
                            s["xy"] += w * xv * yv
                mx, my = s["x"], s["y"]
                vx, vy, cxy = s["xx"] - mx * mx, s["yy"] - my * my, s["xy"] - mx * my
                out[c, i, j] = ((2 * mx * my + C1) * (2 * cxy + C2)) / ((mx * mx + my * my + C1) * (vx + vy + C2))
    return out


def gaussian_normaliser() -> float:
    """Sum of the unnormalised 1D window (for the closed-form pin)."""
    return sum(math.exp(-(k * k) / (2.0 * SIGMA * SIGMA)) for k in range(-(WINDOW // 2), WINDOW // 2 + 1))
