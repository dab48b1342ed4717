"""Pins of the oracle's adaptive density control (Sec. 4.2 implementation
details: densification by the view-space positional gradient; duplication
and pruning of the 4D Gaussians with the rules of 3D Gaussian Splatting).

The statistics are pinned against quantities computed another way: the
view-space gradient of a lone Gaussian against a central difference of the
image in the principal point (shifting (cx, cy) shifts the projected centre
and nothing else), the composited-pixel count against a per-pixel loop over
the explicit inverse of the 2D covariance, and the screen radius against a
symmetric eigenvalue routine. The densify step is pinned against a plain
per-Gaussian loop over the rules, against the Mahalanobis identity of the
split children ((c - mu)^T Sigma4^-1 (c - mu) = |z|^2), against the sample
moments of many children, and against the closed forms of an identity rotor
and of the scale division."""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import density as od
from oracle.render import composited_counts


def _lone_gaussian(seed=11):
    g = synth.gaussians(1, seed, ls_xyz=(-1.2, 0.1), ls_t=(-0.5, 0.1))
    g["mean"][0] = [0.05, -0.1, 0.0, 0.5]
    g["logit"][0] = 1.0
    return g


def _camd(cam, **kw):
    d = oracle.camera_tensors(cam)
    d.update(kw)
    return d


def test_view_space_gradient_of_a_lone_gaussian_is_the_principal_point_derivative():
    g = _lone_gaussian()
    sc = oracle.to_f64(g)
    cam = synth.look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 48, 40)
    t = 0.5
    w = np.random.default_rng(5).normal(0.0, 1.0, (3, 40, 48))
    base = _camd(cam)
    ref = oracle.render(sc, base, t)
    assert float(ref["margin"].min()) > 1e-4  # no decision near its threshold: L is smooth here
    st = od.view_stats(sc, base, t, w)
    assert st["vs_count"][0] == 1 and st["counts"][0] > 50

    def L(**kw):
        return float((oracle.render(sc, _camd(cam, **kw), t)["image"].numpy() * w).sum())
    h = 1e-6  # in normalised device coordinates
    gx = (L(cx=base["cx"] + h * 24.0) - L(cx=base["cx"] - h * 24.0)) / (2 * h)
    gy = (L(cy=base["cy"] + h * 20.0) - L(cy=base["cy"] - h * 20.0)) / (2 * h)
    assert st["vs_grad"][0] == pytest.approx(math.hypot(gx, gy), rel=1e-6)


def test_composited_count_and_radius_of_a_lone_gaussian():
    g = _lone_gaussian(seed=12)
    sc = oracle.to_f64(g)
    cam = synth.look_at((0.2, 0.1, -4.0), (0.0, 0.0, 0.0), 40, 36)
    rec = oracle.preprocess(sc, cam, 0.5)
    cov = rec["cov2d"][0].numpy()
    inv = np.linalg.inv(cov)
    m = rec["mean2d"][0].numpy()
    o = float(rec["opacity_t"][0])
    n = 0
    for j in range(36):
        for i in range(40):
            d = np.array([i + 0.5, j + 0.5]) - m
            p = -0.5 * d @ inv @ d
            if -4.5 <= p <= 0.0 and min(0.99, o * math.exp(p)) >= 1.0 / 255.0:
                n += 1
    counts = composited_counts(sc, cam, 0.5)
    assert n > 20 and int(counts[0]) == n
    st = od.view_stats(sc, cam, 0.5, np.ones((3, 36, 40)))
    lam = np.linalg.eigvalsh(cov)[-1]
    assert st["max_radius"][0] == pytest.approx(3.0 * math.sqrt(lam), rel=1e-12)


def test_statistics_skip_views_that_composite_nothing():
    g = _lone_gaussian(seed=13)
    sc = oracle.to_f64(g)
    cam = synth.look_at((0.0, 0.0, 4.0), (0.0, 0.0, 8.0), 32, 32)  # looking away
    st = od.view_stats(sc, cam, 0.5, np.ones((3, 32, 32)))
    assert st["vs_count"][0] == 0 and st["vs_grad"][0] == 0 and st["max_radius"][0] == 0


def _loop_densify(g, vs_grad, vs_count, max_radius, z, cfg):
    """The rules written one Gaussian at a time with Python floats."""
    c = dict(od.DEFAULTS)
    c.update(cfg)
    f32 = lambda x: float(np.float32(x))  # noqa: E731
    rows, srcs = [], []
    for i in range(len(g["mean"])):
        cnt, gs = float(vs_count[i]), float(vs_grad[i])
        dens = cnt > 0 and gs >= f32(c["grad_threshold"]) * cnt  # exact in double
        scales = [math.exp(float(v)) for v in g["logscale"][i][:3]]
        big = max(scales)
        opacity = 1.0 / (1.0 + math.exp(-float(g["logit"][i])))
        alive = opacity >= f32(c["min_opacity"]) if c["min_opacity"] > 0 else True
        ok_scale = (lambda s: s <= f32(c["max_scale"])) if c["max_scale"] > 0 else (lambda s: True)
        screen_ok = not (c["max_screen_radius"] > 0 and float(max_radius[i]) > f32(c["max_screen_radius"]))
        if dens and big > f32(c["dense_scale"]):
            shift = np.float32(math.log(f32(c["split_divisor"])))
            ls = (g["logscale"][i] - shift).astype(np.float32)
            if alive and ok_scale(max(math.exp(float(v)) for v in ls[:3])):
                R = oracle.rotor_to_matrix(oracle.rotor_normalize(
                    torch.as_tensor(g["rotor"][i:i + 1], dtype=torch.float64)))[0].numpy()
                s = np.exp(g["logscale"][i].astype(np.float64))
                for k in range(2):
                    mu = g["mean"][i].astype(np.float64) + R @ (s * z[i, k].astype(np.float64))
                    rows.append((mu.astype(np.float32), ls, i))
                    srcs.append(-(i + 1))
        else:
            if alive and ok_scale(big) and screen_ok:
                rows.append((g["mean"][i], g["logscale"][i], i))
                srcs.append(i)
            if dens and alive and ok_scale(big):
                rows.append((g["mean"][i], g["logscale"][i], i))
                srcs.append(-(i + 1))
    return rows, np.asarray(srcs, np.int32)


@pytest.mark.parametrize("cfg", [
    {},
    {"min_opacity": 0.2, "max_scale": 0.09, "max_screen_radius": 30.0},
    {"grad_threshold": 1e-4, "dense_scale": 0.045, "split_divisor": 2.0, "min_opacity": 0.4},
])
def test_densify_matches_a_per_gaussian_loop(cfg):
    n = 400
    g = synth.gaussians(n, 21)
    d = synth.density_inputs(22, n)
    out, src = od.densify(g, d["vs_grad"], d["vs_count"], d["max_radius"], d["z"], cfg)
    rows, src_ref = _loop_densify(g, d["vs_grad"], d["vs_count"], d["max_radius"], d["z"], cfg)
    assert np.array_equal(src, src_ref)
    assert len(rows) == len(out["mean"])
    kinds = set()
    for j, (mu, ls, i) in enumerate(rows):
        assert np.array_equal(out["logscale"][j], ls)
        assert np.array_equal(out["rotor"][j], g["rotor"][i])
        assert np.array_equal(out["sh"][j], g["sh"][i])
        assert out["logit"][j] == g["logit"][i]
        assert np.allclose(out["mean"][j], mu, rtol=0, atol=2e-7 * (1 + np.abs(mu).max()))
        kinds.add("child" if not np.array_equal(out["logscale"][j], g["logscale"][i]) else
                  ("copy" if src[j] < 0 else "keep"))
    assert kinds == {"child", "copy", "keep"}  # every kind of row is exercised
    assert len(rows) < 2 * n


def test_split_children_are_drawn_from_the_parent_distribution():
    n = 64
    g = synth.gaussians(n, 31)
    d = synth.density_inputs(32, n)
    d["vs_count"][:] = 1.0
    d["vs_grad"][:] = 1.0  # everything densifies
    cfg = {"dense_scale": 1e-6, "min_opacity": 0.0}  # everything splits, nothing is pruned
    out, src = od.densify(g, d["vs_grad"], d["vs_count"], None, d["z"], cfg)
    assert len(src) == 2 * n and np.array_equal(src, -(np.repeat(np.arange(n), 2) + 1))
    sc = oracle.to_f64(g)
    R = oracle.rotor_to_matrix(oracle.rotor_normalize(sc["rotor"]))
    S4 = oracle.covariance4(R, torch.exp(sc["logscale"])).numpy()
    for i in range(n):
        for k in range(2):
            dlt = out["mean"][2 * i + k].astype(np.float64) - g["mean"][i].astype(np.float64)
            maha = dlt @ np.linalg.solve(S4[i], dlt)
            zz = float(np.sum(d["z"][i, k].astype(np.float64) ** 2))
            assert maha == pytest.approx(zz, rel=2e-3, abs=2e-4)
    # the children's own covariance is the parent's divided by split_divisor^2
    ch = oracle.to_f64({k: v[0::2] for k, v in out.items()})
    S4c = oracle.covariance4(oracle.rotor_to_matrix(oracle.rotor_normalize(ch["rotor"])),
                             torch.exp(ch["logscale"])).numpy()
    # (up to the FP32 rounding of the stored log-scales: |d ln s| <= 2.4e-7 at |ln s| < 4)
    scale = np.abs(S4).max(axis=(1, 2))[:, None, None]
    assert np.all(np.abs(S4c - S4 / 1.6 ** 2) <= 2e-6 * scale)


def test_identity_rotor_children_are_mean_plus_scaled_draws():
    n = 8
    g = synth.gaussians(n, 41)
    g["rotor"][:] = 0.0
    g["rotor"][:, 0] = 1.0
    d = synth.density_inputs(42, n)
    d["vs_count"][:] = 2.0
    d["vs_grad"][:] = 1.0
    out, _ = od.densify(g, d["vs_grad"], d["vs_count"], None, d["z"], {"dense_scale": 1e-6, "min_opacity": 0.0})
    s = np.exp(g["logscale"].astype(np.float64))
    want = g["mean"].astype(np.float64)[:, None, :] + s[:, None, :] * d["z"].astype(np.float64)
    assert np.array_equal(out["mean"], want.reshape(-1, 4).astype(np.float32))


def test_sample_moments_of_many_children():
    m = 20000
    g1 = synth.gaussians(1, 51, ls_xyz=(-1.0, 0.3), ls_t=(-1.0, 0.3))
    g = {k: np.repeat(v, m, axis=0) for k, v in g1.items()}
    z = np.random.default_rng(52).normal(0.0, 1.0, (m, 2, 4)).astype(np.float32)
    out, _ = od.densify(g, np.ones(m, np.float32), np.ones(m, np.float32), None, z,
                        {"dense_scale": 1e-6, "min_opacity": 0.0})
    x = out["mean"].astype(np.float64)
    sc = oracle.to_f64(g1)
    S4 = oracle.covariance4(oracle.rotor_to_matrix(oracle.rotor_normalize(sc["rotor"])),
                            torch.exp(sc["logscale"]))[0].numpy()
    mu = g1["mean"][0].astype(np.float64)
    sd = np.sqrt(np.diag(S4))
    assert np.all(np.abs(x.mean(axis=0) - mu) < 5 * sd / math.sqrt(len(x)))
    C = np.cov(x.T)
    assert np.allclose(C, S4, atol=0.05 * float(np.max(np.diag(S4))))


def test_prune_and_opacity_reset():
    n = 500
    g = synth.gaussians(n, 61)
    d = synth.density_inputs(62, n)
    out, src = od.densify(g, d["vs_grad"], d["vs_count"], d["max_radius"], d["z"], {"min_opacity": 0.3})
    op = 1.0 / (1.0 + np.exp(-out["logit"].astype(np.float64)))
    assert op.min() >= np.float32(0.3) and len(src) > 0
    gone = 1.0 / (1.0 + np.exp(-g["logit"].astype(np.float64))) < np.float32(0.3)
    assert not np.isin(np.where(src >= 0, src, -src - 1), np.nonzero(gone)[0]).any()
    lg = od.opacity_reset(g["logit"], 0.01)
    assert float(1.0 / (1.0 + math.exp(-float(lg.max())))) == pytest.approx(0.01, rel=1e-6)
    low = g["logit"] <= lg.max()
    assert np.array_equal(lg[low], g["logit"][low]) and np.all(lg <= lg.max())
