"""Pins of the oracle's speed field and flow render (Sec. 3.2.2: the sliced
centre moves by (t - mu_t) V / W, so V / W is the speed): the analytic
image-plane velocity against a central difference in t of the oracle's own
projected sliced centre; zero flow for Gaussians without space-time
coupling; a single Gaussian's flow equals its velocity times its alpha
footprint, which a colour render with rgb = 1 gives independently."""
import math

import numpy as np
import torch

import oracle
import synth
from oracle import flow as oflow


def _scene(seed=3, n=40):
    g = synth.gaussians(n, seed, ls_xyz=(-1.8, 0.3), ls_t=(-0.8, 0.3))
    return oracle.to_f64(g)


def test_velocity_is_the_time_derivative_of_the_projected_centre():
    sc = _scene()
    cam = synth.look_at((0.3, -0.2, -4.0), (0.0, 0.0, 0.0), 96, 80)
    t, h = 0.4, 1e-6
    c = oracle.camera_tensors(cam)
    rec = oracle.preprocess(sc, cam, t)
    vel = oflow.image_velocity(rec, c)
    mp = oracle.preprocess(sc, cam, t + h)["mean2d"]
    mm = oracle.preprocess(sc, cam, t - h)["mean2d"]
    fd = (mp - mm) / (2 * h)
    scale = vel.abs().max()
    assert scale > 1.0
    assert torch.allclose(vel, fd, rtol=1e-6, atol=1e-6 * float(scale))


def test_no_space_time_coupling_means_no_flow():
    sc = _scene(seed=4)
    sc["rotor"][:, 4:] = 0.0  # b03 = b13 = b23 = p = 0: R keeps t on its own axis
    cam = synth.look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 64, 64)
    out = oflow.render_flow(sc, cam, 0.5)
    assert float(oflow.speed(out["rec"]).abs().max()) < 1e-12
    assert float(out["flow"].abs().max()) < 1e-12


def test_single_gaussian_flow_is_velocity_times_alpha():
    sc = _scene(seed=5, n=1)
    sc["mean"][0, :3] = 0.0
    sc["mean"][0, 3] = 0.5
    cam = synth.look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 48, 48)
    out = oflow.render_flow(sc, cam, 0.5)
    v = out["velocity"][0]
    white = {k: v_.clone() for k, v_ in sc.items()}
    white["sh"].zero_()
    white["sh"][0, 0, :] = 0.5 / (0.5 / math.sqrt(math.pi))  # rgb = Y00 c + 0.5 = 1
    alpha = oracle.render(white, cam, 0.5)["image"][0]
    assert float(alpha.max()) > 0.1
    for k in range(2):
        assert torch.allclose(out["flow"][k], v[k] * alpha, rtol=1e-12, atol=1e-12 * float(v.abs().max()))
