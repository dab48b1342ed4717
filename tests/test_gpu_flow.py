"""Optical-flow render (R4G_FLAG_FLOW) against the oracle's flow render:
the image-plane velocity d(mean2d)/dt of every sliced centre composited with
the colour render's weights. Tolerance: 2e-3 of the largest flow magnitude
on the pixels the colour comparison calls unambiguous (the flow shares every
threshold decision with the colour render)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import ambiguous, to_device
from oracle import flow as oflow

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def r4g():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2402_03307_gb300 as m
    return m


@pytest.mark.parametrize("size", [(128, 128), (77, 53)])
def test_flow_matches_oracle(r4g, size):
    g, cam, t = synth.small_scene(seed=31, width=size[0], height=size[1])
    ref = oflow.render_flow(oracle.to_f64(g), cam, t)
    rf = ref["flow"].numpy()
    got = r4g.render_flow(to_device(g), cam, t).double().cpu().numpy()
    amb = ambiguous(ref, image=False)
    scale = float(np.abs(rf).max())
    assert scale > 1e-3
    err = np.abs(got - rf)[:, ~amb]
    assert err.max() <= 2e-3 * scale, (err.max(), scale)
    assert amb.mean() < 0.01


def test_flow_of_static_scene_is_zero_and_flow_has_no_backward(r4g):
    g, cam, t = synth.small_scene(seed=32)
    g = dict(g)
    rot = g["rotor"].copy()
    rot[:, 4:] = 0.0
    g["rotor"] = rot
    rend = r4g.Renderer(flags=r4g.abi.R4G_FLAG_FLOW, bg=(1.0, 1.0, 1.0))
    p = to_device(g)
    res = rend.render(p, cam, t)
    assert float(res.image.abs().max()) < 1e-6  # no speed, and no background
    grads = {k: torch.zeros(v.shape, dtype=torch.float32, device="cuda") for k, v in p.items()}
    with pytest.raises(r4g.abi.R4GError):
        rend.backward(p, cam, t, res, torch.zeros_like(res.image), grads)
