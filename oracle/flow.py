"""Speed field and optical-flow render (Sec. 3.2.2: slicing a 4D Gaussian at
t adds the motion term (t - mu_t) V / W to its centre, so V / W is the
Gaussian's speed, the same at every t; the paper visualises it as optical
flow).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``.

The image-plane velocity of a Gaussian is the time derivative of its
projected sliced centre. With p_c = R mu(t) + t_c = (x, y, z) and
u = fx x / z + cx, v = fy y / z + cy:
    dp_c/dt = R V / W,
    du/dt = fx (x' z - x z') / z^2,   dv/dt = fy (y' z - y z') / z^2.
The flow image composites these 2-vectors with the weights of the colour
render (alpha_i T_i of the same Gaussians in the same order), over a zero
background.
"""
from __future__ import annotations

import torch

from .render import _cam, preprocess, render


def speed(rec: dict) -> torch.Tensor:
    """V / W [N,3] from a record's Sigma4 (V = Sigma_{xyz,t}, W = Sigma_tt)."""
    s4 = rec["sigma4"]
    return s4[..., :3, 3] / s4[..., 3:4, 3]


def image_velocity(rec: dict, cam: dict) -> torch.Tensor:
    """d(mean2d)/dt [N,2] in pixels per unit time."""
    pdot = speed(rec) @ cam["R"].T
    x, y, z = rec["pc"][:, 0], rec["pc"][:, 1], rec["pc"][:, 2]
    du = cam["fx"] * (pdot[:, 0] * z - x * pdot[:, 2]) / (z * z)
    dv = cam["fy"] * (pdot[:, 1] * z - y * pdot[:, 2]) / (z * z)
    return torch.stack([du, dv], -1)


def render_flow(scene: dict, cam, t: float, cull_temporal: bool = True) -> dict:
    """``flow`` [2,H,W] plus the colour render's decision margins (the flow
    shares every decision with the colour render)."""
    c = _cam(cam)
    rec = preprocess(scene, c, t, cull_temporal)
    vel = image_velocity(rec, c)
    rec_f = dict(rec)
    rec_f["rgb"] = torch.cat([vel, torch.zeros_like(vel[:, :1])], -1)
    out = render(scene, cam, t, bg=(0.0, 0.0, 0.0), cull_temporal=cull_temporal, rec=rec_f)
    out["flow"] = out["image"][:2]
    out["velocity"] = vel
    return out
