"""Pins for the oracle's projection and compositing (Sec. 3.1 Eq. 3, Sec. 3.2.2):
analytic single-Gaussian footprints (Jacobian of the projection by automatic
differentiation, slice by textbook conditioning, rotation from closed forms),
two-layer closed form, the transmittance stop, the spatial/temporal
separability of Sec. 3.2.1, cull neutrality and finite-difference gradients.
Both clamps are pinned: alpha <= 0.99 (closed form 0.99 rgb + 0.01 bg and a
zero gradient on the clamped core) and the Jacobian of the projection taken at
the point clamped to 1.3 tan(fov/2) (footprint with the Jacobian of the
clamped point by automatic differentiation; central differences with both
clamps active)."""
import math
import os

import numpy as np
import pytest
import torch

import oracle
import synth
from oracle.render import PARAM_NAMES, _inclusion, depth_order

special = pytest.importorskip("scipy.special")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_rotors():
    rows = [ln for ln in open(os.path.join(GOLDEN, "rotor_cases.txt")) if ln.strip() and not ln.startswith("#")]
    out = []
    for ln in rows:
        v = np.array([float(x) for x in ln.split()])
        out.append((v[:8], v[8:].reshape(4, 4)))
    return out


def _real_sh_l1(d):
    th = math.acos(d[2])
    ph = math.atan2(d[1], d[0])
    out = [special.sph_harm_y(0, 0, th, ph).real]
    Y11 = special.sph_harm_y(1, 1, th, ph)
    out += [math.sqrt(2) * Y11.imag, special.sph_harm_y(1, 0, th, ph).real, math.sqrt(2) * Y11.real]
    return np.array(out)


def _frustum_limits(cam):
    """1.3 tan(fov/2) on each axis of the image plane (tan(fov_x/2) = W / 2fx)."""
    return 1.3 * cam.width / (2.0 * cam.fx), 1.3 * cam.height / (2.0 * cam.fy)


def expected_single(mean4, Rm, s, logit, sh, cam, t, bg=np.zeros(3), jclamp=False, out_alpha=None):
    """Independent footprint of one Gaussian: image [3,H,W], T [H,W].

    The 2D covariance uses the Jacobian of the pinhole projection obtained by
    automatic differentiation. With ``jclamp`` that Jacobian is taken at the
    camera-space point whose x/z and y/z are clamped to the frustum limits
    (the mean itself still projects unclamped). ``out_alpha``, when a list,
    receives the unclamped o_t e^power map (zero outside the 3-sigma cutoff)."""
    S4 = Rm @ np.diag(s ** 2) @ Rm.T
    dt = t - mean4[3]
    mu3 = mean4[:3] + S4[:3, 3] / S4[3, 3] * dt
    S3 = S4[:3, :3] - np.outer(S4[:3, 3], S4[:3, 3]) / S4[3, 3]
    temporal = math.exp(-0.5 * dt * dt / S4[3, 3])
    w2c = cam.world_to_cam.astype(np.float64)

    def pi(x):
        pc = torch.as_tensor(w2c[:, :3]) @ x + torch.as_tensor(w2c[:, 3])
        return torch.stack([cam.fx * pc[0] / pc[2] + cam.cx, cam.fy * pc[1] / pc[2] + cam.cy])

    x0 = torch.as_tensor(mu3)
    if jclamp:
        pc = w2c[:, :3] @ mu3 + w2c[:, 3]
        lx, ly = _frustum_limits(cam)
        pcc = np.array([np.clip(pc[0] / pc[2], -lx, lx) * pc[2], np.clip(pc[1] / pc[2], -ly, ly) * pc[2], pc[2]])

        def pi_c(p):
            return torch.stack([cam.fx * p[0] / p[2] + cam.cx, cam.fy * p[1] / p[2] + cam.cy])

        J = torch.autograd.functional.jacobian(pi_c, torch.as_tensor(pcc)).numpy() @ w2c[:, :3]
    else:
        J = torch.autograd.functional.jacobian(pi, x0).numpy()
    m2 = pi(x0).numpy()
    cov = J @ S3 @ J.T + 0.3 * np.eye(2)
    inv = np.linalg.inv(cov)
    d = mu3 - cam.center
    d = d / np.linalg.norm(d)
    Y = _real_sh_l1(d)
    rgb = np.maximum(0.0, (Y[:, None] * sh[:4]).sum(0) + 0.5)
    o = 1.0 / (1.0 + math.exp(-logit)) * temporal
    H, W = cam.height, cam.width
    img = np.zeros((3, H, W))
    T = np.ones((H, W))
    araw = np.zeros((H, W))
    for j in range(H):
        for i in range(W):
            dd = np.array([i + 0.5, j + 0.5]) - m2
            power = -0.5 * dd @ inv @ dd
            if power > 0 or power < -4.5:
                continue
            araw[j, i] = o * math.exp(power)
            a = min(0.99, o * math.exp(power))
            if a < 1 / 255:
                continue
            img[:, j, i] = rgb * a
            T[j, i] = 1 - a
    img += T[None] * bg[:, None, None]
    if out_alpha is not None:
        out_alpha.append(araw)
    return img, T, m2


def _one(mean4, rotor, ls, logit, sh):
    return {
        "mean": torch.as_tensor(np.asarray(mean4, np.float64)[None]),
        "rotor": torch.as_tensor(np.asarray(rotor, np.float64)[None]),
        "logscale": torch.as_tensor(np.asarray(ls, np.float64)[None]),
        "logit": torch.as_tensor(np.array([logit], np.float64)),
        "sh": torch.as_tensor(np.asarray(sh, np.float64)[None]),
    }


@pytest.mark.parametrize("case", range(8))
def test_single_gaussian_footprint(case):
    rotor, Rm = _golden_rotors()[case]
    cam = synth.look_at((0.3, -0.2, -4.0), (0.0, 0.0, 0.0), 64, 48)
    rng = np.random.default_rng(case)
    mean4 = np.array([0.1, -0.05, 0.2, 0.4])
    ls = np.log(np.array([0.35, 0.15, 0.25, 0.5]))
    sh = np.zeros((16, 3))
    sh[:4] = rng.normal(0, 0.4, (4, 3))
    sh[4:] = 0.0
    logit = 1.2
    t = 0.55
    bg = np.array([0.2, 0.4, 0.8])
    img_ref, T_ref, _ = expected_single(mean4, Rm, np.exp(ls), logit, sh, cam, t, bg)
    out = oracle.render(_one(mean4, rotor, ls, logit, sh), cam, t, bg=tuple(bg))
    np.testing.assert_allclose(out["image"].numpy(), img_ref, atol=1e-12)
    np.testing.assert_allclose(out["T"].numpy(), T_ref, atol=1e-12)
    covered = T_ref < 1
    assert covered.sum() > 50  # the footprint spans many pixels
    assert (out["last"].numpy()[covered] == 0).all() and (out["last"].numpy()[~covered] == -1).all()


def test_two_layers_closed_form():
    """C = c1 a1 + c2 a2 (1 - a1) with Gaussian 1 nearer (Eq. 3)."""
    cam = synth.look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 40, 40)
    ident = np.zeros(8)
    ident[0] = 1
    g = []
    for mean4, col in (((0.05, 0.0, 0.5, 0.5), 0.3), ((-0.05, 0.02, -0.5, 0.5), -0.2)):
        sh = np.zeros((16, 3))
        sh[0] = col
        g.append((np.array(mean4), sh))
    ls = np.log(np.array([0.3, 0.25, 0.2, 1.0]))
    scene = {k: torch.cat([_one(m, ident, ls, 0.8, sh)[k] for m, sh in g]) for k in PARAM_NAMES}
    out = oracle.render(scene, cam, 0.5)
    # Gaussian 1 has the larger z so it is behind; the nearer one is index 1
    i1, T1, _ = expected_single(g[1][0], np.eye(4), np.exp(ls), 0.8, g[1][1], cam, 0.5)
    i0, T0, _ = expected_single(g[0][0], np.eye(4), np.exp(ls), 0.8, g[0][1], cam, 0.5)
    a_near, a_far = 1 - T1, 1 - T0
    ref = i1 + i0 * (1 - a_near)[None]
    np.testing.assert_allclose(out["image"].numpy(), ref, atol=1e-12)
    np.testing.assert_allclose(out["T"].numpy(), (1 - a_near) * (1 - a_far), atol=1e-12)


def test_transmittance_stop_on_opaque_stack():
    """Five Gaussians on the optical axis, alpha = 0.95 at the centre pixel:
    T goes 0.05, 0.0025, 1.25e-4, then 6.25e-6 < 1e-4, so the 4th is not
    composited and the 3rd nearest is the last one."""
    cam = synth.look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 33, 33)  # centre pixel 16 at 16.5
    ident = np.zeros(8)
    ident[0] = 1
    logit = math.log(0.95 / 0.05)
    zs = [0.9, -0.3, 0.6, 0.0, -0.6]
    cols = [0.1, 0.2, 0.3, 0.4, 0.5]
    parts = []
    for z, c in zip(zs, cols):
        sh = np.zeros((16, 3))
        sh[0] = c
        parts.append(_one((0.0, 0.0, z, 0.5), ident, np.log([0.2, 0.2, 0.2, 1.0]), logit, sh))
    scene = {k: torch.cat([p[k] for p in parts]) for k in parts[0]}
    out = oracle.render(scene, cam, 0.5)
    near = np.argsort(zs)  # nearest first
    C0 = 0.5 / math.sqrt(math.pi)
    rgb = [0.5 + C0 * cols[k] for k in near]
    T = 1.0
    ref = 0.0
    for k in range(3):
        ref += rgb[k] * 0.95 * T
        T *= 0.05
    assert out["last"][16, 16].item() == near[2]
    assert abs(out["T"][16, 16].item() - 1.25e-4) < 1e-15
    assert abs(out["image"][0, 16, 16].item() - ref) < 1e-13


def test_temporal_cull_never_changes_the_image():
    """lambda (t - mu_t)^2 > 16 gives alpha <= exp(-8) < 1/255 (Sec. 3.2.2)."""
    g, cam, t = synth.small_scene(seed=7, n=600, width=64, height=64)
    sc = oracle.to_f64(g)
    a = oracle.render(sc, cam, t, cull_temporal=True)
    b = oracle.render(sc, cam, t, cull_temporal=False)
    assert int(a["rec"]["visible"].sum()) < int(b["rec"]["visible"].sum())
    # same decisions; only the summation's rounding may differ
    assert torch.equal(a["last"], b["last"])
    assert (a["image"] - b["image"]).abs().max() < 1e-14 and (a["T"] - b["T"]).abs().max() < 1e-14


def test_static_rotor_reduces_to_3d_splatting():
    """tau = 0 (Sec. 3.2.1): the 4D render equals a 3D Gaussian splat with
    Sigma3 = Q diag(s^2) Q^T (Q the quaternion matrix of (s, -b12, b02, -b01))
    and opacity o exp(-1/2 (t - mu_t)^2 / s_t^2)."""
    g, cam, t = synth.small_scene(seed=8, n=400, width=64, height=64)
    g["rotor"][:, 4:] = 0.0
    sc = oracle.to_f64(g)
    out4 = oracle.render(sc, cam, t)
    q = sc["rotor"][:, :4].numpy()
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    from test_oracle_rotor import quat_matrix
    Q = np.stack([quat_matrix(a, -d, c, -b) for a, b, c, d in q])
    s = np.exp(sc["logscale"].numpy())
    S3 = Q @ (s[:, :3, None] ** 2 * np.transpose(Q, (0, 2, 1)))
    mu3 = torch.as_tensor(sc["mean"][:, :3].numpy())
    camt = oracle.camera_tensors(cam)
    pr = oracle.project(mu3, torch.as_tensor(S3), camt)
    dt = t - sc["mean"][:, 3].numpy()
    op = 1 / (1 + np.exp(-sc["logit"].numpy())) * np.exp(-0.5 * dt * dt / s[:, 3] ** 2)
    d = mu3 - torch.as_tensor(cam.center)
    d = d / torch.linalg.norm(d, dim=-1, keepdim=True)
    rec = {"visible": (pr["z"] > 0.2) & (pr["det"] > 0) & torch.as_tensor(dt * dt / s[:, 3] ** 2 <= 16),
           "mean2d": pr["mean2d"], "conic": pr["conic"], "z": pr["z"],
           "opacity_t": torch.as_tensor(op), "rgb": oracle.sh_color(sc["sh"], d)}
    out3 = oracle.render(None, cam, t, rec=rec)
    np.testing.assert_allclose(out4["image"].numpy(), out3["image"].numpy(), atol=1e-12)
    assert torch.equal(out4["last"], out3["last"])


def test_input_order_does_not_matter():
    g, cam, t = synth.small_scene(seed=9, n=500, width=48, height=48)
    sc = oracle.to_f64(g)
    perm = torch.as_tensor(np.random.default_rng(0).permutation(500))
    sp = {k: v[perm] for k, v in sc.items()}
    a = oracle.render(sc, cam, t)
    b = oracle.render(sp, cam, t)
    np.testing.assert_allclose(a["image"].numpy(), b["image"].numpy(), atol=1e-14)
    la, lb = a["last"], b["last"]
    mapped = torch.where(lb >= 0, perm[lb.clamp(min=0)], lb)
    assert torch.equal(la, mapped)


def test_background_adds_final_transmittance():
    g, cam, t = synth.small_scene(seed=10, n=300, width=32, height=32)
    sc = oracle.to_f64(g)
    a = oracle.render(sc, cam, t)
    b = oracle.render(sc, cam, t, bg=(1.0, 0.5, 0.25))
    bg = torch.tensor([1.0, 0.5, 0.25], dtype=torch.float64)
    assert torch.allclose(b["image"], a["image"] + a["T"][None] * bg[:, None, None], atol=1e-15)


def fd_scene():
    """64 Gaussians sized to cover a 32x32 view (the finite-difference workload)."""
    g = synth.gaussians(64, 11, ls_xyz=(-1.6, 0.3), ls_t=(-0.7, 0.3))
    cam = synth.look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 32, 32)
    return g, cam, 0.5


def _decisions(sc, cam, t):
    rec = oracle.preprocess(sc, cam, t)
    order = depth_order(rec)
    jj, ii = torch.meshgrid(torch.arange(cam.height), torch.arange(cam.width), indexing="ij")
    px = ii.flatten().double() + 0.5
    py = jj.flatten().double() + 0.5
    m2, con = rec["mean2d"][order], rec["conic"][order]
    dx = px[:, None] - m2[None, :, 0]
    dy = py[:, None] - m2[None, :, 1]
    power = -0.5 * (con[None, :, 0] * dx * dx + con[None, :, 2] * dy * dy) - con[None, :, 1] * dx * dy
    alpha = torch.clamp(rec["opacity_t"][order][None] * torch.exp(power), max=0.99)
    valid = (power <= 0) & (power >= -4.5) & (alpha >= 1 / 255)
    T = torch.cumprod(1 - torch.where(valid, alpha, torch.zeros_like(alpha)), 1)
    inc = valid & (T >= 1e-4)
    clamp = (alpha >= 0.99) & valid
    return (tuple(order.tolist()), valid.numpy().tobytes(), inc.numpy().tobytes(), clamp.numpy().tobytes())


def test_gradient_matches_central_differences():
    g, cam, t = fd_scene()
    sc = oracle.to_f64(g)
    rng = np.random.default_rng(12)
    wimg = rng.normal(0, 1, (3, 32, 32))
    grads = oracle.render_grad(sc, cam, t, wimg)
    W = torch.as_tensor(wimg)

    def L(s):
        return float((oracle.render(s, cam, t)["image"] * W).sum())

    base = _decisions(sc, cam, t)
    checked = 0
    for name in PARAM_NAMES:
        flat = sc[name].reshape(-1)
        idx = rng.choice(flat.numel(), size=min(60, flat.numel()), replace=False)
        for k in idx:
            x = flat[k].item()
            h = 1e-6 * max(1.0, abs(x))
            vals = []
            ok = True
            for sgn in (1, -1):
                s2 = {kk: vv.clone() for kk, vv in sc.items()}
                s2[name].reshape(-1)[k] = x + sgn * h
                if _decisions(s2, cam, t) != base:
                    ok = False
                    break
                vals.append(L(s2))
            if not ok:
                continue
            fd = (vals[0] - vals[1]) / (2 * h)
            an = grads[name].reshape(-1)[k].item()
            scale = grads[name].abs().max().item()
            assert abs(fd - an) <= 1e-5 * (abs(an) + 1e-3 * scale) + 1e-9, (name, int(k), fd, an)
            checked += 1
    assert checked >= 200
    # every parameter group receives gradient
    for name in ("mean", "rotor", "logscale", "logit", "sh"):
        assert grads[name].abs().max() > 0


# ---------------------------------------------------------------------------
# The two clamps: alpha <= 0.99 (Sec. 3.1 Eq. 3, with the compositing rules of
# the 3D Gaussian Splatting rasteriser that the paper follows) and the
# Jacobian of the projection taken at a point clamped to 1.3 tan(fov/2) (the
# EWA convention of the same rasteriser, to which Sec. 3.1 defers).

C0 = 0.5 / math.sqrt(math.pi)  # real Y_00


def _opaque_scene():
    """One large Gaussian of opacity 1 - 1e-3 (logit ln 999), centred on the
    optical axis at its temporal centre, DC-only colour."""
    rotor, Rm = _golden_rotors()[3]
    mean4 = np.array([0.05, -0.03, 0.1, 0.5])
    ls = np.log(np.array([1.9, 1.4, 1.6, 0.6]))
    sh = np.zeros((16, 3))
    sh[0] = [0.3, -0.2, 0.6]
    logit = math.log(999.0)
    return rotor, Rm, mean4, ls, sh, logit


def test_alpha_clamp_closed_form():
    """Where o_t e^power exceeds 0.99 the pixel is 0.99 rgb + 0.01 bg, for any
    opacity: the clamp applies to the product, after the exponential, and its
    value is 0.99. Elsewhere the footprint is o_t e^power."""
    rotor, Rm, mean4, ls, sh, logit = _opaque_scene()
    cam = synth.look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 48, 48)
    bg = np.array([0.2, 0.4, 0.8])
    t = 0.5
    araw = []
    img_ref, T_ref, _ = expected_single(mean4, Rm, np.exp(ls), logit, sh, cam, t, bg, out_alpha=araw)
    araw = araw[0]
    out = oracle.render(_one(mean4, rotor, ls, logit, sh), cam, t, bg=tuple(bg))
    img = out["image"].numpy()
    rgb = 0.5 + C0 * sh[0]
    closed = (0.99 * rgb + 0.01 * bg)[:, None, None]
    clamped = araw > 0.99
    assert clamped.sum() >= 8  # several pixels sit inside the clamped core
    assert (araw[clamped] < 0.999).all()  # ... with o_t e^power strictly between 0.99 and o_t
    np.testing.assert_allclose(img[:, clamped], np.broadcast_to(closed, img.shape)[:, clamped], atol=1e-14)
    np.testing.assert_allclose(out["T"].numpy()[clamped], 0.01, atol=1e-15)
    # unclamped pixels of the footprint: alpha = o_t e^power exactly
    ring = (araw >= 1 / 255) & ~clamped
    assert ring.sum() > 100
    a = araw[ring]
    np.testing.assert_allclose(img[:, ring], rgb[:, None] * a[None] + bg[:, None] * (1 - a)[None], atol=1e-13)
    np.testing.assert_allclose(img, img_ref, atol=1e-13)


def test_alpha_clamp_has_zero_gradient():
    """On pixels where alpha is clamped, the image depends on neither the
    opacity nor the footprint's shape or position: the gradient of those pixels
    w.r.t. the logit, log-scales, rotor and mean is zero (the colour is
    DC-only, so it does not depend on the view direction either), and
    d/d sh_00 = 0.99 C0 per clamped pixel."""
    rotor, Rm, mean4, ls, sh, logit = _opaque_scene()
    cam = synth.look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 48, 48)
    t = 0.5
    araw = []
    expected_single(mean4, Rm, np.exp(ls), logit, sh, cam, t, out_alpha=araw)
    clamped = araw[0] > 0.99
    w = np.zeros((3, 48, 48))
    w[:, clamped] = 1.0
    gr = oracle.render_grad(_one(mean4, rotor, ls, logit, sh), cam, t, w)
    for k in ("logit", "logscale", "rotor", "mean"):
        assert gr[k].abs().max().item() < 1e-12, (k, gr[k])
    np.testing.assert_allclose(gr["sh"][0, 0].numpy(), 0.99 * C0 * clamped.sum(), rtol=1e-12)
    # the same image weights on the unclamped ring do move the logit
    w2 = np.zeros((3, 48, 48))
    w2[:, (araw[0] >= 1 / 255) & ~clamped] = 1.0
    assert abs(oracle.render_grad(_one(mean4, rotor, ls, logit, sh), cam, t, w2)["logit"].item()) > 1e-3


@pytest.mark.parametrize("off", [(0.9, 0.0), (-0.95, 0.1), (0.1, 0.7), (-0.85, -0.68)])
def test_jacobian_clamp_outside_the_frustum(off):
    """A Gaussian whose camera-space x/z or y/z lies beyond 1.3 tan(fov/2) but
    whose footprint still reaches the image: its 2D covariance uses the
    Jacobian at the clamped point, while its centre projects unclamped."""
    cam = synth.look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 64, 48)
    lx, ly = _frustum_limits(cam)
    assert abs(off[0]) > lx or abs(off[1]) > ly
    # camera axes of this look-at: x_c = -x, y_c = -y, z_c = z + 4
    zc = 4.0
    mean4 = np.array([-off[0] * zc, -off[1] * zc, 0.0, 0.5])
    rotor, Rm = _golden_rotors()[5]
    ls = np.log(np.array([1.0, 0.7, 0.8, 0.5]))
    sh = np.zeros((16, 3))
    sh[:4] = np.random.default_rng(3).normal(0, 0.4, (4, 3))
    logit = 2.0
    bg = np.array([0.1, 0.2, 0.3])
    ref_c, T_c, m2 = expected_single(mean4, Rm, np.exp(ls), logit, sh, cam, 0.5, bg, jclamp=True)
    ref_u, _, _ = expected_single(mean4, Rm, np.exp(ls), logit, sh, cam, 0.5, bg, jclamp=False)
    assert not (0 <= m2[0] <= cam.width and 0 <= m2[1] <= cam.height)  # centre off the image
    covered = T_c < 1
    assert covered.sum() > 30  # the footprint reaches into the image
    assert np.abs(ref_c - ref_u).max() > 1e-3  # the clamp changes the image (compared at 1e-12 below)
    out = oracle.render(_one(mean4, rotor, ls, logit, sh), cam, 0.5, bg=tuple(bg))
    np.testing.assert_allclose(out["image"].numpy(), ref_c, atol=1e-12)
    np.testing.assert_allclose(out["T"].numpy(), T_c, atol=1e-12)


def _clamp_flags(sc, cam, t):
    """Which Gaussians have their Jacobian clamped (x/z or y/z beyond the limits)."""
    rec = oracle.preprocess(sc, cam, t)
    pc = rec["pc"].detach()
    lx, ly = _frustum_limits(cam)
    return ((pc[:, 0] / pc[:, 2]).abs() > lx) | ((pc[:, 1] / pc[:, 2]).abs() > ly)


def _clamp_scene():
    """Eight Gaussians on a 32x32 view: two opaque ones whose centres clamp
    alpha, two beyond the frustum limits whose footprints reach the image
    (clamped Jacobian), four ordinary ones."""
    g = synth.gaussians(8, 31, ls_xyz=(-1.4, 0.2), ls_t=(-0.5, 0.2))
    g["mean"][:, 3] = 0.5 + 0.05 * g["mean"][:, 3]
    g["logit"][:2] = [7.0, 6.0]
    g["logscale"][:2, :3] = np.log(2.0)
    g["mean"][:2, :3] = [[0.1, 0.05, 0.3], [-0.2, -0.1, -0.2]]
    # camera at (0,0,-4) looking at the origin: x_c = -x, z_c = z + 4
    g["mean"][2, :3] = [-0.95 * 4.2, 0.1, 0.2]
    g["mean"][3, :3] = [0.3, 0.85 * 3.8, -0.2]
    g["logscale"][2:4, :3] = np.log(1.0)
    g["logit"][2:4] = 2.0
    cam = synth.look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 32, 32)
    return g, cam, 0.5


def test_gradient_with_active_clamps_matches_central_differences():
    """Central differences (FP64, h = 1e-6 max(1, |x|)) of every parameter of
    a scene where both clamps are active, against the analytic gradient: the
    clamps are differentiated as the piecewise functions they are (zero
    derivative through an active clamp)."""
    g, cam, t = _clamp_scene()
    sc = oracle.to_f64(g)
    jflag = _clamp_flags(sc, cam, t)
    assert bool(jflag[2]) and bool(jflag[3]) and not bool(jflag[:2].any())
    base_img = oracle.render(sc, cam, t)
    n_clamped_alpha = 0
    rec = base_img["rec"]
    order = depth_order(rec)
    for k in range(2):  # both opaque Gaussians clamp alpha somewhere
        _, _, alpha_raw, *_ = _inclusion(
            rec["mean2d"][[k]].detach(), rec["conic"][[k]].detach(), rec["opacity_t"][[k]].detach(),
            torch.arange(32).repeat(32).double() + 0.5, torch.arange(32).repeat_interleave(32).double() + 0.5)
        n_clamped_alpha += int((alpha_raw > 0.99).sum())
    assert n_clamped_alpha >= 4 and order.numel() == 8
    rng = np.random.default_rng(13)
    wimg = rng.normal(0, 1, (3, 32, 32))
    grads = oracle.render_grad(sc, cam, t, wimg)
    W = torch.as_tensor(wimg)

    def L(s):
        return float((oracle.render(s, cam, t)["image"] * W).sum())

    base = _decisions(sc, cam, t) + (jflag.numpy().tobytes(),)
    checked = 0
    for name in PARAM_NAMES:
        flat = sc[name].reshape(-1)
        for k in range(flat.numel()):
            x = flat[k].item()
            h = 1e-6 * max(1.0, abs(x))
            vals = []
            for sgn in (1, -1):
                s2 = {kk: vv.clone() for kk, vv in sc.items()}
                s2[name].reshape(-1)[k] = x + sgn * h
                if _decisions(s2, cam, t) + (_clamp_flags(s2, cam, t).numpy().tobytes(),) != base:
                    break
                vals.append(L(s2))
            if len(vals) < 2:
                continue
            fd = (vals[0] - vals[1]) / (2 * h)
            an = grads[name].reshape(-1)[k].item()
            scale = grads[name].abs().max().item()
            assert abs(fd - an) <= 1e-5 * (abs(an) + 1e-3 * scale) + 1e-9, (name, int(k), fd, an)
            checked += 1
    assert checked >= 480
    # the off-frustum Gaussians receive gradient through their visible footprint
    assert grads["mean"][2:4].abs().max() > 0 and grads["logscale"][2:4].abs().max() > 0


def test_pixel_gradient_restricted_to_a_block():
    """The gradient over a listed block of pixels, compositing only the
    Gaussians whose 3-sigma box meets the block, equals the full-image
    gradient with the upstream gradient zero outside the block."""
    from gpu_util import block_pixels, box_keep
    g, cam, t = synth.small_scene(seed=33, n=400, width=48, height=40)
    sc = oracle.to_f64(g)
    x0, y0, w, h = 13, 9, 20, 16
    rng = np.random.default_rng(4)
    gimg = np.zeros((3, 40, 48))
    gimg[:, y0:y0 + h, x0:x0 + w] = rng.normal(0, 1, (3, h, w))
    full = oracle.render_grad(sc, cam, t, gimg)
    rec = oracle.preprocess(sc, cam, t)
    keep = box_keep(rec, x0, y0, w, h)
    assert 0 < keep.sum() < rec["visible"].sum()  # the restriction drops Gaussians
    pix = block_pixels(x0, y0, w, h)
    part = oracle.render_grad_pixels(sc, cam, t, pix, gimg[:, pix[:, 1], pix[:, 0]].T, keep=keep)
    for k in PARAM_NAMES:
        np.testing.assert_allclose(part[k].numpy(), full[k].numpy(), atol=1e-12, rtol=1e-9)
    out = oracle.render_pixels(sc, cam, t, pix)
    ref = oracle.render(sc, cam, t)
    assert torch.equal(out["last"], ref["last"][y0:y0 + h, x0:x0 + w].reshape(-1))
    # composited count: consistent with the final transmittance (no Gaussian -> T = 1)
    assert ((out["n_composited"] == 0) == (out["T"] == 1.0)).all()


def test_alternatives_closed_forms():
    """Alternatives of one pixel (Eq. 3 under each open decision):
    two Gaussians whose depths differ by 1e-9 relative give the two
    compositing orders c1 a1 + c2 a2 (1 - a1) and c2 a2 + c1 a1 (1 - a2);
    two clamped layers give T' = (1 - 0.99)^2, at the 1e-4 stop threshold, so
    both 0.99 c1 + 0.0099 c2 (composited) and 0.99 c1 (stopped) are open;
    a pixel with no open decision has one colour."""
    cam = synth.look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 33, 33)
    ident = np.zeros(8)
    ident[0] = 1

    def scene(specs):
        parts = []
        for dz, c, logit in specs:
            sh = np.zeros((16, 3))
            sh[0] = c
            parts.append(_one((0.0, 0.0, dz, 0.5), ident, np.log([0.3, 0.3, 0.3, 1.0]), logit, sh))
        return oracle.preprocess({k: torch.cat([p[k] for p in parts]) for k in parts[0]}, cam, 0.5)

    c = [0.5 + C0 * 0.4, 0.5 + C0 * -0.3]
    rec = scene(((0.0, 0.4, 0.5), (4e-9, -0.3, 1.5)))
    alts = oracle.pixel_alternatives(rec, (16, 16), 1e-5, 1e-7)
    assert len(alts) == 2
    a = [1 / (1 + math.exp(-0.5)), 1 / (1 + math.exp(-1.5))]  # centre pixel: power = 0
    first = c[0] * a[0] + c[1] * a[1] * (1 - a[0])  # index 0 nearer (smaller z)
    second = c[1] * a[1] + c[0] * a[0] * (1 - a[1])
    assert abs(alts[0][0].item() - first) < 1e-12 and abs(alts[1][0].item() - second) < 1e-12
    assert len(oracle.pixel_alternatives(rec, (16, 16), 1e-5, 1e-10)) == 1  # gap above the bound
    # two opaque layers 0.5 apart: alpha clamps to 0.99 on both
    rec = scene(((0.0, 0.4, 9.0), (0.5, -0.3, 9.0)))
    alts = oracle.pixel_alternatives(rec, (16, 16), 1e-5, 1e-7)
    got = sorted(float(x[0]) for x in alts)
    want = sorted([0.99 * c[0] + 0.99 * 0.01 * c[1], 0.99 * c[0]])
    assert len(alts) == 2 and max(abs(g - w) for g, w in zip(got, want)) < 1e-12
    ref = oracle.render_pixels(None, cam, 0.5, np.array([[16, 16]]), rec=rec)
    assert abs(float(alts[0][0]) - float(ref["rgb"][0, 0])) < 1e-15  # the computed colour comes first
    # a pixel away from every threshold: one colour, equal to the render's
    rec = scene(((0.0, 0.4, 0.5), (0.5, -0.3, 1.5)))
    alts = oracle.pixel_alternatives(rec, (15, 17), 1e-5, 1e-7)
    ref = oracle.render_pixels(None, cam, 0.5, np.array([[15, 17]]), rec=rec)
    assert len(alts) == 1 and torch.allclose(alts[0], ref["rgb"][0], atol=1e-15, rtol=0)
