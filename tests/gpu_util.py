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


def image_report(img_gpu: np.ndarray, ref: dict) -> dict:
    """Max-abs error over unambiguous pixels, PSNR over all, ambiguous fraction."""
    ref_img = ref["image"].numpy()
    amb = ambiguous(ref, image=True)
    err = np.abs(img_gpu.astype(np.float64) - ref_img)
    ok = ~amb
    return {
        "max_abs": float(err[:, ok].max()) if ok.any() else 0.0,
        "max_abs_all": float(err.max()),
        "psnr": psnr(img_gpu.astype(np.float64), ref_img),
        "ambiguous": float(amb.mean()),
        "amb_mask": amb,
    }
