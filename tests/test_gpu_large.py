"""Large mixed-precision scene: 2M Gaussians, 1920x1080, scales and SH
coefficients stored in BF16, slicing and blending in FP32. The error against
the FP64 oracle is measured on 128x128 crops: the oracle runs on the
BF16-rounded parameters (so the bar is the FP32 arithmetic's: max abs RGB
2e-3 on non-ambiguous pixels, PSNR > 60 dB), and the storage error (the BF16
render against the oracle on the FP32 parameters) is reported.

The oracle composites every crop pixel over the Gaussians whose 3-sigma box
(from the oracle's own preprocess) meets the crop, in its global depth
order: a Gaussian outside that box fails the power >= -4.5 test at every
crop pixel, so the restriction changes no pixel."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import sampled_report

pytestmark = pytest.mark.gpu
CROP = 128


@pytest.fixture(scope="module")
def r4g():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2402_03307_gb300 as m
    return m


def _bf16_round(a: np.ndarray) -> np.ndarray:
    return torch.as_tensor(a).to(torch.bfloat16).float().numpy()


def _crop_rec(rec: dict, x0: int, y0: int) -> dict:
    """The oracle's records restricted to Gaussians whose 3-sigma box meets the crop."""
    m = rec["mean2d"].detach()
    cov = rec["cov2d"].detach()
    hx = 3.0 * torch.sqrt(torch.clamp(cov[:, 0, 0], min=0)) + 1.0
    hy = 3.0 * torch.sqrt(torch.clamp(cov[:, 1, 1], min=0)) + 1.0
    keep = (rec["visible"] & (m[:, 0] + hx >= x0) & (m[:, 0] - hx <= x0 + CROP)
            & (m[:, 1] + hy >= y0) & (m[:, 1] - hy <= y0 + CROP))
    idx = torch.nonzero(keep).flatten()
    n = rec["visible"].numel()
    return {k: (v[idx] if torch.is_tensor(v) and v.dim() > 0 and v.shape[0] == n else v) for k, v in rec.items()}


def _crop_pixels(x0: int, y0: int) -> np.ndarray:
    yy, xx = np.meshgrid(np.arange(y0, y0 + CROP), np.arange(x0, x0 + CROP), indexing="ij")
    return np.stack([xx.reshape(-1), yy.reshape(-1)], axis=1)


def test_large_bf16_crops_vs_oracle(r4g):
    g = synth.gaussians(2_000_000, 7, mean_lo=-3.0, mean_hi=3.0)
    cam, t = synth.large_views(8, 1)[0]
    gb = dict(g)
    gb["logscale"] = _bf16_round(g["logscale"])
    gb["sh"] = _bf16_round(g["sh"])
    p = {k: torch.as_tensor(v).cuda().contiguous() for k, v in g.items()}
    p["logscale"] = p["logscale"].to(torch.bfloat16).contiguous()
    p["sh"] = p["sh"].to(torch.bfloat16).contiguous()
    img = r4g.Renderer().render(p, cam, t).image.double().cpu().numpy()
    sc = oracle.to_f64(gb)
    rec = oracle.preprocess(sc, cam, t)
    rng = np.random.default_rng(0)
    crops = [(int(rng.integers(0, cam.width - CROP)), int(rng.integers(0, cam.height - CROP))) for _ in range(2)]
    worst, amb_total, store_err = 0.0, 0, []
    for x0, y0 in crops:
        sub = _crop_rec(rec, x0, y0)
        pix = _crop_pixels(x0, y0)
        ref = oracle.render_pixels(sc, cam, t, pix, rec=sub)
        got = img[:, y0:y0 + CROP, x0:x0 + CROP].reshape(3, -1)
        rep = sampled_report(got.T, ref, sub, pix)
        amb_total += rep["n_ambiguous"]
        assert rep["unresolved"] == 0, (x0, y0, rep)
        worst = max(worst, rep["max_abs"])
        assert rep["psnr"] > 60.0, (x0, y0, rep)
        # storage error: the same crop of the oracle on the FP32 parameters
        if not store_err:
            rec32 = oracle.preprocess(oracle.to_f64(g), cam, t)
        ref32 = oracle.render_pixels(None, cam, t, _crop_pixels(x0, y0), rec=_crop_rec(rec32, x0, y0))
        store_err.append(float(np.abs(got - ref32["rgb"].numpy().T).max()))
    assert worst <= 2e-3, worst
    # 2M Gaussians put many pairs of contributors within FP32 rounding of each
    # other's depth (1.9 % of these pixels); each such pixel was checked above
    # against the colours of both orders
    assert amb_total < 0.05 * len(crops) * CROP * CROP
    print(f"bf16 crops: max abs vs oracle(bf16 params) {worst:.2e}; vs oracle(fp32 params) {max(store_err):.2e}; "
          f"{amb_total} of {len(crops) * CROP * CROP} pixels ambiguous, each within 2e-3 of a valid colour")
    assert max(store_err) < 0.1  # storage rounding of scales and SH only
