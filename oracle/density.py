"""Adaptive density control: the view-space gradient statistics and one
densify-and-prune step.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper (Sec. 4.2, implementation details) densifies by the view-space
positional gradient with thresholds 2e-4 (Plenoptic) and 5e-5 (D-NeRF),
duplicates and prunes the 4D Gaussians on the GPU, and otherwise follows the
densification, pruning and opacity-reset settings of 3D Gaussian Splatting.
Read for 4D Gaussians:

statistics, per view in which Gaussian i is composited into >= 1 pixel
    vs_grad[i]    += |(dL/du * W/2, dL/dv * H/2)|   (the gradient with respect
                     to the projected centre in normalised device coordinates;
                     only the compositing's direct dependence on (u, v))
    vs_count[i]   += 1
    max_radius[i]  = max(max_radius[i], 3 sqrt(lambda_max(Sigma')))

step
    densify  vs_count > 0 and vs_grad / vs_count >= grad_threshold
    clone    densified and largest spatial scale <= dense_scale: keep, plus a copy
    split    densified otherwise: two children with means drawn from the
             Gaussian's own 4D distribution, mean + R diag(s) z, and all four
             scales divided by split_divisor
    prune    output rows with opacity < min_opacity; rows with a spatial scale
             above max_scale (when > 0); rows continuing a Gaussian whose
             max_radius exceeds max_screen_radius (when > 0)
    order    Gaussian after Gaussian; kept: i; clone: i then its copy; split:
             child 0 then child 1

The decisions compare FP32 inputs with thresholds in double precision (the
exact reading of each rule on the stored values); the arithmetic of the new
rows is FP64 and rounded to FP32 once.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from .render import composited_counts, render_grad
from .rotor import rotor_normalize, rotor_to_matrix

DEFAULTS = {"grad_threshold": 2e-4, "dense_scale": 0.06, "split_divisor": 1.6, "min_opacity": 0.005,
            "max_scale": 0.0, "max_screen_radius": 0.0}


def view_stats(scene: dict, cam, t: float, grad_image, stats: dict | None = None) -> dict:
    """Add one view's statistics into ``stats`` (float64 [N] arrays; created
    zeroed when None) for L = sum(grad_image * image)."""
    from .render import _cam, preprocess
    camd = _cam(cam)
    n = int(scene["mean"].shape[0])
    if stats is None:
        stats = {k: np.zeros(n) for k in ("vs_grad", "vs_count", "max_radius")}
    g = render_grad(scene, camd, t, grad_image)
    with torch.no_grad():
        rec = preprocess(scene, camd, t)
        counts = composited_counts(scene, camd, t, rec=rec).numpy()
        d = g["rec_mean2d"].numpy()
        ndc = np.hypot(d[:, 0] * (camd["width"] / 2.0), d[:, 1] * (camd["height"] / 2.0))
        cov = rec["cov2d"].numpy()
        a, b, c = cov[:, 0, 0], cov[:, 0, 1], cov[:, 1, 1]
        lam = 0.5 * (a + c) + np.sqrt(0.25 * (a - c) ** 2 + b * b)
        radius = 3.0 * np.sqrt(np.maximum(lam, 0.0))
    hit = counts > 0
    stats["vs_grad"] = stats["vs_grad"] + np.where(hit, ndc, 0.0)
    stats["vs_count"] = stats["vs_count"] + hit
    stats["max_radius"] = np.maximum(stats["max_radius"], np.where(hit, radius, 0.0))
    stats["counts"] = counts
    return stats


def _rules(cfg: dict) -> dict:
    c = dict(DEFAULTS)
    c.update(cfg or {})
    m = float(np.float32(c["min_opacity"]))
    return {
        "grad_thr": float(np.float32(c["grad_threshold"])),
        "log_dense": math.log(float(np.float32(c["dense_scale"]))),
        "logit_min": math.log(m / (1.0 - m)) if m > 0 else -math.inf,
        "log_max_scale": math.log(float(np.float32(c["max_scale"]))) if c["max_scale"] > 0 else math.inf,
        "max_radius": float(np.float32(c["max_screen_radius"])) if c["max_screen_radius"] > 0 else math.inf,
        "ls_shift": np.float32(math.log(float(np.float32(c["split_divisor"])))),
    }


def densify(g: dict, vs_grad, vs_count, max_radius, z, cfg: dict | None = None):
    """One densify-and-prune step on float32 numpy parameters. ``z``: float32
    [N, 2, 4] standard normal draws for split children; ``max_radius`` may be
    None. Returns (new float32 parameters, int32 source map: i for a row
    continuing Gaussian i, -(i + 1) for a new row)."""
    r = _rules(cfg)
    mean = np.asarray(g["mean"], np.float32)
    ls = np.asarray(g["logscale"], np.float32)
    logit = np.asarray(g["logit"], np.float32)
    gs = np.asarray(vs_grad, np.float32).astype(np.float64)
    cnt = np.asarray(vs_count, np.float32).astype(np.float64)
    rad = (np.asarray(max_radius, np.float32).astype(np.float64) if max_radius is not None
           else np.zeros(len(mean)))
    dens = (cnt > 0) & (gs >= r["grad_thr"] * cnt)
    lmax = ls[:, :3].max(axis=1).astype(np.float64)
    clone = dens & (lmax <= r["log_dense"])
    split = dens & ~clone
    opaque = logit.astype(np.float64) >= r["logit_min"]
    small = lmax <= r["log_max_scale"]
    ls_child = (ls - r["ls_shift"]).astype(np.float32)  # FP32 subtraction, as stored
    child_ok = opaque & (ls_child[:, :3].max(axis=1).astype(np.float64) <= r["log_max_scale"])
    keep0 = ~split & opaque & small & ~(rad > r["max_radius"])
    keep1 = clone & opaque & small

    # children of the split Gaussians: mean + R diag(s) z, in FP64
    R = rotor_to_matrix(rotor_normalize(torch.as_tensor(np.asarray(g["rotor"]), dtype=torch.float64))).numpy()
    s = np.exp(ls.astype(np.float64))
    zz = np.asarray(z, np.float32).astype(np.float64)
    child = mean.astype(np.float64)[:, None, :] + np.einsum("nab,ncb->nca", R, s[:, None, :] * zz)

    # output slots (i, 0) and (i, 1) in the order i = 0..n-1, slot 0 first
    slot_ok = np.stack([keep0 | (split & child_ok), keep1 | (split & child_ok)], axis=1).reshape(-1)
    pos = np.nonzero(slot_ok)[0]
    src, slot = pos // 2, pos % 2
    is_child = split[src]
    out = {"mean": np.where(is_child[:, None], child[src, slot].astype(np.float32), mean[src]),
           "rotor": np.asarray(g["rotor"], np.float32)[src],
           "logscale": np.where(is_child[:, None], ls_child[src], ls[src]),
           "logit": logit[src],
           "sh": np.asarray(g["sh"], np.float32)[src]}
    src_map = np.where((slot == 0) & ~is_child, src, -(src + 1)).astype(np.int32)
    return out, src_map


def opacity_reset(logit, max_opacity: float = 0.01):
    """opacity = min(opacity, max_opacity) on the logits (FP32)."""
    m = float(np.float32(max_opacity))
    cap = np.float32(math.log(m / (1.0 - m)))
    return np.minimum(np.asarray(logit, np.float32), cap)
