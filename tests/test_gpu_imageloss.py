"""The fused L1 + SSIM image loss (r4g_image_loss) against the FP64 oracle:
loss parts within 1e-5 relative, the gradient within 1e-4 relative L2 and
1e-3 of its largest element elementwise; ragged sizes (tiles and halo at the
border), one channel, and a full 1352x1014 frame."""
import numpy as np
import pytest
import torch

from oracle import imageloss as il

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def r4g():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2402_03307_gb300 as m
    return m


@pytest.mark.parametrize("shape", [(3, 64, 64), (3, 37, 53), (1, 5, 7), (3, 101, 33)])
@pytest.mark.parametrize("lam", [0.2, 0.0, 1.0])
def test_image_loss_matches_oracle(r4g, shape, lam):
    rng = np.random.default_rng(sum(shape))
    x = rng.uniform(0, 1, shape).astype(np.float32)
    y = np.clip(x + rng.normal(0, 0.1, shape), 0, 1).astype(np.float32)
    out, grad = r4g.image_loss(torch.as_tensor(x).cuda(), torch.as_tensor(y).cuda(), lam)
    ref = il.image_loss(torch.as_tensor(x), torch.as_tensor(y), lam)
    o = out.double().cpu().numpy()
    for k, name in enumerate(("loss", "l1", "ssim")):
        want = float(ref[name])
        assert abs(o[k] - want) <= 1e-5 * max(abs(want), 1e-3), (name, o[k], want)
    a = grad.double().cpu().numpy().reshape(-1)
    b = ref["grad"].numpy().reshape(-1)
    if np.abs(b).max() > 0:
        assert np.linalg.norm(a - b) <= 1e-4 * np.linalg.norm(b)
        assert np.abs(a - b).max() <= 1e-3 * np.abs(b).max()


def test_image_loss_full_frame(r4g):
    rng = np.random.default_rng(1)
    shape = (3, 1014, 1352)
    x = rng.uniform(0, 1, shape).astype(np.float32)
    y = np.clip(x + rng.normal(0, 0.05, shape), 0, 1).astype(np.float32)
    out, grad = r4g.image_loss(torch.as_tensor(x).cuda(), torch.as_tensor(y).cuda(), 0.2)
    ref = il.image_loss(torch.as_tensor(x), torch.as_tensor(y), 0.2)
    assert abs(float(out[0]) - float(ref["loss"])) <= 1e-5 * float(ref["loss"])
    a = grad.double().cpu().numpy().reshape(-1)
    b = ref["grad"].numpy().reshape(-1)
    assert np.linalg.norm(a - b) <= 1e-4 * np.linalg.norm(b)
