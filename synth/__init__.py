"""Seeded synthetic inputs for the 4D-rotor Gaussian renderer.

This module is shared by the CPU oracle tests, the GPU parity tests and the
benchmark, and it holds none of the rendering method's arithmetic: it only
draws random Gaussian parameters from the stated distributions and builds
pinhole cameras (look-at frames) that the renderer receives as inputs.
Every array is returned as float32 so that the GPU path and the FP64 oracle
consume bit-identical values (the oracle upcasts them).

Parameter layout (one row per Gaussian):
  mean      f32[N,4]    (x, y, z, t)
  rotor     f32[N,8]    (s, b01, b02, b12, b03, b13, b23, p), raw draws;
                        the renderer normalises them (rotor normalisation of
                        the paper's appendix A.1 runs inside the render path)
  logscale  f32[N,4]    log of (s_x, s_y, s_z, s_t)
  logit     f32[N]      opacity logit, opacity = sigmoid(logit)
  sh        f32[N,16,3] degree-3 SH coefficients, [coefficient][rgb]

Workloads (the paper's datasets are absent; these stand in for them at the
paper's resolutions, 1352x1014 for Plenoptic Video):
  small    1,000 Gaussians, means in [-1,1]^3, 128x128, camera at distance 4
  fwd300k  300,000 Gaussians, means in [-3,3]^3, 1352x1014, 300 frames on a
           circle of radius 8 around the origin, t_k = k/299
  train    300,000 Gaussians, 4 views per step at seeded (t, angle), L1 loss
           against a seeded smooth target image
  batched  100,000 Gaussians, 16 views of mixed resolution
  large    2,000,000 Gaussians, 1920x1080, 8 views
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "gaussians", "look_at", "orbit_camera", "Camera", "smooth_target",
    "small_scene", "fwd300k_scene", "train_views", "batched_views", "large_views",
    "random_pixels", "random_keys", "density_inputs",
]


@dataclass
class Camera:
    """Pinhole camera. ``world_to_cam`` is a row-major 3x4 [R | t] with OpenCV
    axes (x right, y down, z forward); pixel (i, j) samples the point
    (i + 0.5, j + 0.5) on the image plane."""
    world_to_cam: np.ndarray  # f32 [3,4]
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int

    @property
    def center(self) -> np.ndarray:
        r = self.world_to_cam[:, :3].astype(np.float64)
        t = self.world_to_cam[:, 3].astype(np.float64)
        return -r.T @ t


def _f32(x: float) -> float:
    return float(np.float32(x))


def gaussians(n: int, seed: int, mean_lo: float = -1.0, mean_hi: float = 1.0,
              t_lo: float = 0.0, t_hi: float = 1.0,
              ls_xyz: tuple[float, float] = (-3.0, 0.5),
              ls_t: tuple[float, float] = (-2.0, 0.5),
              sh_dc: tuple[float, float] = (0.5, 0.2),
              sh_rest_std: float = 0.05,
              logit_dist: tuple[float, float] = (0.0, 1.0)) -> dict[str, np.ndarray]:
    """Draw N Gaussians; draw order mean, logscale, rotor, logit, SH. The
    opacity logit is N(logit_dist); N(4, 1) gives mostly opaque Gaussians."""
    rng = np.random.default_rng(seed)
    mean = np.empty((n, 4), np.float64)
    mean[:, :3] = rng.uniform(mean_lo, mean_hi, (n, 3))
    mean[:, 3] = rng.uniform(t_lo, t_hi, n)
    logscale = np.empty((n, 4), np.float64)
    logscale[:, :3] = rng.normal(ls_xyz[0], ls_xyz[1], (n, 3))
    logscale[:, 3] = rng.normal(ls_t[0], ls_t[1], n)
    rotor = rng.normal(0.0, 1.0, (n, 8))
    logit = rng.normal(logit_dist[0], logit_dist[1], n)
    sh = np.empty((n, 16, 3), np.float64)
    sh[:, 0, :] = rng.normal(sh_dc[0], sh_dc[1], (n, 3))
    sh[:, 1:, :] = rng.normal(0.0, sh_rest_std, (n, 15, 3))
    return {
        "mean": mean.astype(np.float32),
        "rotor": rotor.astype(np.float32),
        "logscale": logscale.astype(np.float32),
        "logit": logit.astype(np.float32),
        "sh": sh.astype(np.float32),
    }


def look_at(eye, target, width: int, height: int, fov_x_deg: float = 60.0) -> Camera:
    """Camera at ``eye`` looking at ``target``; horizontal field of view
    ``fov_x_deg``; square pixels; principal point at the image centre.
    The camera's y axis is the world's -Y made orthogonal to the view axis."""
    eye = np.asarray(eye, np.float64)
    target = np.asarray(target, np.float64)
    z = target - eye
    z /= np.linalg.norm(z)
    down = np.array([0.0, -1.0, 0.0])
    y = down - np.dot(down, z) * z
    y /= np.linalg.norm(y)
    x = np.cross(y, z)
    r = np.stack([x, y, z])
    t = -r @ eye
    w2c = np.concatenate([r, t[:, None]], axis=1).astype(np.float32)
    f = (width / 2.0) / math.tan(math.radians(fov_x_deg) / 2.0)
    return Camera(w2c, _f32(f), _f32(f), _f32(width / 2.0), _f32(height / 2.0),
                  int(width), int(height))


def orbit_camera(k: int, frames: int, radius: float, width: int, height: int,
                 fov_x_deg: float = 60.0) -> tuple[Camera, float]:
    """Frame k of a circular sweep: eye (r sin a, 0, -r cos a), a = 2 pi k / frames,
    looking at the origin, at time t = k / (frames - 1)."""
    a = 2.0 * math.pi * k / frames
    eye = (radius * math.sin(a), 0.0, -radius * math.cos(a))
    t = k / (frames - 1) if frames > 1 else 0.5
    return look_at(eye, (0.0, 0.0, 0.0), width, height, fov_x_deg), _f32(t)


def small_scene(seed: int = 1, n: int = 1000, width: int = 128, height: int = 128):
    """1,000 Gaussians in [-1,1]^3, one camera at distance 4 looking at the origin, t=0.5."""
    g = gaussians(n, seed)
    cam = look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), width, height)
    return g, cam, _f32(0.5)


def fwd300k_scene(seed: int = 2, n: int = 300_000):
    """300k Gaussians in [-3,3]^3 for the 1352x1014 sweep (cameras via orbit_camera)."""
    return gaussians(n, seed, mean_lo=-3.0, mean_hi=3.0)


def train_views(seed: int, views: int = 4, width: int = 1352, height: int = 1014,
                radius: float = 8.0) -> list[tuple[Camera, float]]:
    """Seeded (camera, t) pairs: t ~ U[0,1], orbit angle ~ U[0, 2 pi)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(views):
        t = rng.uniform(0.0, 1.0)
        a = rng.uniform(0.0, 2.0 * math.pi)
        eye = (radius * math.sin(a), 0.0, -radius * math.cos(a))
        out.append((look_at(eye, (0.0, 0.0, 0.0), width, height), _f32(t)))
    return out


def batched_views(seed: int, views: int = 16, radius: float = 8.0) -> list[tuple[Camera, float]]:
    """16 views of uneven size: a seeded shuffle of 6 x 800x800, 5 x 640x480 and
    5 x 1352x1014, each at a seeded (t, angle)."""
    rng = np.random.default_rng(seed)
    sizes = [(800, 800)] * 6 + [(640, 480)] * 5 + [(1352, 1014)] * 5
    sizes = sizes[:views] if views <= len(sizes) else (sizes * ((views // 16) + 1))[:views]
    order = rng.permutation(len(sizes))
    out = []
    for i in order:
        w, h = sizes[i]
        t = rng.uniform(0.0, 1.0)
        a = rng.uniform(0.0, 2.0 * math.pi)
        eye = (radius * math.sin(a), 0.0, -radius * math.cos(a))
        out.append((look_at(eye, (0.0, 0.0, 0.0), w, h), _f32(t)))
    return out


def large_views(seed: int, views: int = 8) -> list[tuple[Camera, float]]:
    return train_views(seed, views, 1920, 1080)


def smooth_target(seed: int, width: int, height: int) -> np.ndarray:
    """A seeded smooth RGB image f32[3,H,W] in [0,1]: a sum of random sinusoids."""
    rng = np.random.default_rng(seed)
    yy, xx = np.meshgrid(np.arange(height) / height, np.arange(width) / width, indexing="ij")
    img = np.zeros((3, height, width), np.float64)
    for c in range(3):
        for _ in range(4):
            fx, fy = rng.uniform(0.5, 4.0, 2)
            ph = rng.uniform(0, 2 * math.pi)
            img[c] += np.sin(2 * math.pi * (fx * xx + fy * yy) + ph)
        img[c] = 0.5 + 0.125 * img[c]
    return np.clip(img, 0.0, 1.0).astype(np.float32)


def random_pixels(seed: int, width: int, height: int, count: int) -> np.ndarray:
    """``count`` distinct pixel coordinates int32[count, 2] as (column, row)."""
    rng = np.random.default_rng(seed)
    idx = rng.choice(width * height, size=min(count, width * height), replace=False)
    return np.stack([idx % width, idx // width], axis=1).astype(np.int32)


def random_keys(seed: int, n: int, high_bits: int) -> tuple[np.ndarray, np.ndarray]:
    """Seeded (u64 key, u32 value) pairs for sort tests: the key's high word is
    drawn from [0, 2^high_bits) and its low word is a positive float32's bit
    pattern; values are 0..n-1. Many duplicate keys are planted so that
    stability is exercised."""
    rng = np.random.default_rng(seed)
    hi = rng.integers(0, 1 << high_bits, n, dtype=np.uint64)
    depth = rng.uniform(0.2, 20.0, n).astype(np.float32)
    # plant ties: a quarter of the entries copy another entry's depth
    m = n // 4
    if n > 1 and m > 0:
        src = rng.integers(0, n, m)
        dst = rng.integers(0, n, m)
        depth[dst] = depth[src]
    lo = depth.view(np.uint32).astype(np.uint64)
    keys = (hi << np.uint64(32)) | lo
    vals = np.arange(n, dtype=np.uint32)
    return keys, vals


def density_inputs(seed: int, n: int, threshold: float = 2e-4, max_views: int = 8) -> dict[str, np.ndarray]:
    """Seeded statistics and split draws for a densify-and-prune step over n
    Gaussians: vs_count integer in [0, max_views], a mean view-space gradient
    threshold * exp(N(-0.5, 1)) (about a third at or above the threshold),
    vs_grad = mean * count, max_radius ~ U[0, 40] pixels, and z ~ N(0, 1)
    f32[n, 2, 4] for the split children."""
    rng = np.random.default_rng(seed)
    count = rng.integers(0, max_views + 1, n).astype(np.float32)
    mean = threshold * np.exp(rng.normal(-0.5, 1.0, n))
    vs_grad = (mean * count).astype(np.float32)
    max_radius = rng.uniform(0.0, 40.0, n).astype(np.float32)
    z = rng.normal(0.0, 1.0, (n, 2, 4)).astype(np.float32)
    return {"vs_grad": vs_grad, "vs_count": count, "max_radius": max_radius, "z": z}
