"""Shared helpers of the GPU parity tests (no method arithmetic here)."""
from __future__ import annotations

import math

import numpy as np
import torch

# A pixel is "ambiguous" when one of the oracle's threshold decisions is within
# this relative margin of flipping (FP32 vs FP64 rounding can then change it),
# or when two contributing Gaussians' depths are within AMBIG_DEPTH. For image
# comparisons only decisions whose flip could move the colour by 1e-4 or more
# count (the oracle's margin_img / margin_depth_img); final transmittance,
# last-contributor and gradient comparisons use every decision.
# FP32 power carries ~1e-6 relative error (conic inversion and projection of
# the sliced mean amplify the 6e-8 unit roundoff ~10x); depth z = r . mu + t
# takes ~4 roundings, ~2.4e-7 relative.
AMBIG_REL = 1e-5
AMBIG_DEPTH = 3e-7
MAX_ABS = 2e-3
MIN_PSNR = 60.0


def to_device(g: dict, dev="cuda", dtypes: dict | None = None) -> dict:
    out = {}
    for k, v in g.items():
        t = torch.as_tensor(np.ascontiguousarray(v)).to(dev)
        if dtypes and k in dtypes:
            t = t.to(dtypes[k])
        out[k] = t.contiguous()
    return out


def psnr(a: np.ndarray, b: np.ndarray) -> float:
    mse = float(np.mean((a - b) ** 2))
    return math.inf if mse == 0 else 10.0 * math.log10(1.0 / mse)


def gpu_last_ids(last: np.ndarray, values: np.ndarray, ranges: np.ndarray, tile: tuple[int, int]) -> np.ndarray:
    """Map the per-pixel 'last position + 1' to Gaussian ids (-1 for none)."""
    H, W = last.shape
    tw, th = tile
    tiles_x = (W + tw - 1) // tw
    jj, ii = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    tid = (jj // th) * tiles_x + (ii // tw)
    pos = ranges[tid, 0].astype(np.int64) + last.astype(np.int64) - 1
    ids = np.where(last > 0, values[np.clip(pos, 0, max(len(values) - 1, 0))] if len(values) else -1, -1)
    return ids.astype(np.int64)


def ambiguous(ref: dict, image: bool = True) -> np.ndarray:
    if image:
        return (ref["margin_img"].numpy() < AMBIG_REL) | (ref["margin_depth_img"].numpy() < AMBIG_DEPTH)
    return (ref["margin"].numpy() < AMBIG_REL) | (ref["margin_depth"].numpy() < AMBIG_DEPTH)


def resolve_ambiguous(got: np.ndarray, rec: dict, pixels: np.ndarray, bg=(0.0, 0.0, 0.0)) -> np.ndarray:
    """For pixels whose result the rounding leaves open: the smallest max-abs
    distance of the GPU colour (got [P,3]) to any of the oracle's valid
    colours of that pixel (``oracle.pixel_alternatives``)."""
    import oracle
    out = np.zeros(len(pixels))
    for k, px in enumerate(pixels):
        alts = oracle.pixel_alternatives(rec, (int(px[0]), int(px[1])), AMBIG_REL, AMBIG_DEPTH, bg)
        out[k] = min(float(np.abs(got[k] - a.numpy()).max()) for a in alts)
    return out


def sampled_report(got: np.ndarray, ref: dict, rec: dict, pixels: np.ndarray, bg=(0.0, 0.0, 0.0)) -> dict:
    """GPU colours got [P,3] of the listed pixels against ``oracle.render_pixels``
    (``ref``, computed over ``rec``): max-abs error over the unambiguous pixels;
    each ambiguous pixel must lie within MAX_ABS of one of its valid colours
    (``unresolved`` counts those that do not); PSNR over all pixels."""
    amb = ambiguous(ref, image=True)
    r = ref["rgb"].numpy()
    err = np.abs(got.astype(np.float64) - r)
    alt = resolve_ambiguous(got[amb].astype(np.float64), rec, pixels[amb], bg) if amb.any() else np.zeros(0)
    return {
        "max_abs": float(err[~amb].max()) if (~amb).any() else 0.0,
        "max_abs_all": float(err.max()) if len(err) else 0.0,
        "max_abs_ambiguous": float(alt.max()) if len(alt) else 0.0,
        "unresolved": int((alt > MAX_ABS).sum()),
        "ambiguous": float(amb.mean()) if len(amb) else 0.0,
        "n_ambiguous": int(amb.sum()),
        "psnr": psnr(got.astype(np.float64), r),
    }


def image_report(img_gpu: np.ndarray, ref: dict, bg=(0.0, 0.0, 0.0)) -> dict:
    """Max-abs error over unambiguous pixels, PSNR over all, ambiguous
    fraction; every ambiguous pixel is checked against its valid colours."""
    ref_img = ref["image"].numpy()
    amb = ambiguous(ref, image=True)
    err = np.abs(img_gpu.astype(np.float64) - ref_img)
    ok = ~amb
    jj, ii = np.nonzero(amb)
    pix = np.stack([ii, jj], axis=1)
    got = img_gpu[:, jj, ii].T.astype(np.float64)
    alt = resolve_ambiguous(got, ref["rec"], pix, bg) if len(pix) else np.zeros(0)
    return {
        "max_abs": float(err[:, ok].max()) if ok.any() else 0.0,
        "max_abs_all": float(err.max()),
        "max_abs_ambiguous": float(alt.max()) if len(alt) else 0.0,
        "unresolved": int((alt > MAX_ABS).sum()),
        "psnr": psnr(img_gpu.astype(np.float64), ref_img),
        "ambiguous": float(amb.mean()),
        "amb_mask": amb,
    }


def box_keep(rec: dict, x0: int, y0: int, w: int, h: int) -> np.ndarray:
    """Gaussians (bool [N]) whose 3-sigma box, from the oracle's own 2D
    covariance, meets the pixel block [x0, x0+w) x [y0, y0+h). Every other
    Gaussian fails the power >= -4.5 cutoff at every pixel of the block, so
    restricting the oracle to these changes none of its pixels."""
    m = rec["mean2d"].detach()
    cov = rec["cov2d"].detach()
    hx = 3.0 * torch.sqrt(torch.clamp(cov[:, 0, 0], min=0)) + 1.0
    hy = 3.0 * torch.sqrt(torch.clamp(cov[:, 1, 1], min=0)) + 1.0
    keep = (rec["visible"] & (m[:, 0] + hx >= x0) & (m[:, 0] - hx <= x0 + w)
            & (m[:, 1] + hy >= y0) & (m[:, 1] - hy <= y0 + h))
    return keep.numpy()


def block_pixels(x0: int, y0: int, w: int, h: int) -> np.ndarray:
    """The pixels of a block as int [w*h, 2] (column, row), row-major."""
    yy, xx = np.meshgrid(np.arange(y0, y0 + h), np.arange(x0, x0 + w), indexing="ij")
    return np.stack([xx.reshape(-1), yy.reshape(-1)], axis=1)


NAMES = ("mean", "rotor", "logscale", "logit", "sh")


def grad_weights(g, cam, t, seed, bg=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Seeded upstream gradient f32 [3,H,W], zero on the pixels where any
    decision of the oracle is within rounding of flipping (there two
    different gradients are both right)."""
    import oracle
    ref = oracle.render(oracle.to_f64(g), cam, t, bg=bg)
    amb = ambiguous(ref, image=False)
    w = np.random.default_rng(seed).normal(0, 1, (3, cam.height, cam.width))
    w[:, amb] = 0.0
    return w.astype(np.float32)


def gpu_grads(r4g, g, cam, t, w, **kw) -> dict:
    """Parameter gradients of L = sum(w * image) from r4g_render_backward."""
    rend = r4g.Renderer(**kw)
    p = to_device(g)
    res = rend.render(p, cam, t)
    grads = {k: torch.zeros(v.shape, dtype=torch.float32, device="cuda") for k, v in p.items()}
    rend.backward(p, cam, t, res, torch.as_tensor(w).cuda(), grads)
    torch.cuda.synchronize()
    return {k: v.double().cpu().numpy() for k, v in grads.items()}


def compare_grads(got: dict, ref: dict, tag, names=NAMES) -> dict:
    """Per parameter group ||g - g_ref|| <= 1e-2 ||g_ref||, and per element
    |g - g_ref| <= 1e-2 (|g_ref| + 1e-3 max|g_ref|) for 99.9% of elements.
    Returns the relative L2 error of each group."""
    out = {}
    for k in names:
        a = np.asarray(got[k]).reshape(-1)
        b = ref[k].numpy().reshape(-1) if torch.is_tensor(ref[k]) else np.asarray(ref[k]).reshape(-1)
        nb = np.linalg.norm(b)
        assert nb > 0, (tag, k)
        rel = np.linalg.norm(a - b) / nb
        assert rel <= 1e-2, (tag, k, rel)
        bad = np.abs(a - b) > 1e-2 * (np.abs(b) + 1e-3 * np.abs(b).max())
        assert bad.mean() <= 1e-3, (tag, k, bad.mean(), int(bad.sum()))
        out[k] = float(rel)
    return out
