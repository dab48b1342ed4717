"""Brute-force per-pixel renderer of sliced 4D Gaussians and its gradient.

The image is the plain definition of Eq. 3 (Sec. 3.1) over the 3D Gaussians
sliced at time t (Sec. 3.2.2): every pixel composites, front to back, every
visible Gaussian in the global order of camera-space depth of its sliced mean
(ties by Gaussian index). There are no tiles, no keys and no sort kernel.

Per-pixel rules (the 3D Gaussian Splatting rasteriser's, which the paper
follows; thresholds as fixed for this renderer):
  d      = pixel centre - mean2d
  power  = -1/2 d^T conic d
  skip   if power > 0 or power < -4.5       (3-sigma ellipse, per pixel)
  alpha  = min(0.99, opacity_t exp(power))
  skip   if alpha < 1/255
  T'     = T (1 - alpha); stop before this Gaussian if T' < 1e-4
  C     += rgb alpha T;  T = T'
  pixel  = C + T bg
Gaussians are culled before the pixel loop when lambda (t - mu_t)^2 > 16
(Sec. 3.2.2), when the sliced mean is at depth <= 0.2, or when the 2D
covariance is not positive definite.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from .projection import camera_tensors, project
from .rotor import rotor_normalize, rotor_to_matrix
from .sh import sh_color
from .slicing import covariance4, slice_at

ALPHA_MIN = 1.0 / 255.0
ALPHA_MAX = 0.99
T_MIN = 1e-4
POWER_CUT = -4.5
TEMPORAL_CUT = 16.0
NEAR = 0.2
DILATION = 0.3
IMPACT_MIN = 1e-4  # smallest colour change a flipped decision must be able to cause to count

PARAM_NAMES = ("mean", "rotor", "logscale", "logit", "sh")


def to_f64(g: dict) -> dict:
    """Upcast a dict of float32 numpy parameter arrays to float64 tensors."""
    return {k: torch.as_tensor(np.asarray(g[k]), dtype=torch.float64).clone() for k in PARAM_NAMES}


def _cam(cam):
    return cam if isinstance(cam, dict) else camera_tensors(cam)


def preprocess(scene: dict, cam, t: float, cull_temporal: bool = True, sh_degree: int = 3) -> dict:
    """Per-Gaussian steps: activations, F_norm, F_map, Sigma4, slice, projection,
    SH colour. Returns float64 tensors (differentiable w.r.t. ``scene``)."""
    cam = _cam(cam)
    scale = torch.exp(scene["logscale"])
    opacity = torch.sigmoid(scene["logit"])
    R = rotor_to_matrix(rotor_normalize(scene["rotor"]))
    sigma4 = covariance4(R, scale)
    mu3, sigma3, temporal, lam_dt2 = slice_at(scene["mean"], sigma4, t)
    proj = project(mu3, sigma3, cam, DILATION)
    centre = -cam["R"].T @ cam["t"]
    dirs = mu3 - centre
    dirs = dirs / torch.linalg.norm(dirs, dim=-1, keepdim=True)
    rgb = sh_color(scene["sh"], dirs, sh_degree)
    visible = (proj["z"] > NEAR) & (proj["det"] > 0)
    if cull_temporal:
        visible = visible & (lam_dt2 <= TEMPORAL_CUT)
    return {
        "visible": visible, "mean2d": proj["mean2d"], "conic": proj["conic"],
        "cov2d": proj["cov2d"], "det": proj["det"], "z": proj["z"], "pc": proj["pc"],
        "opacity_t": opacity * temporal, "rgb": rgb, "mu3": mu3, "sigma3": sigma3,
        "sigma4": sigma4, "lam_dt2": lam_dt2, "R": R,
    }


def depth_order(rec: dict) -> torch.Tensor:
    """Indices of the visible Gaussians in increasing depth, ties by index."""
    vis = torch.nonzero(rec["visible"]).flatten()
    z = rec["z"].detach()[vis]
    _, perm = torch.sort(z, stable=True)
    return vis[perm]


def _inclusion(m2, con, o, px, py):
    """The per-pixel rules for a chunk of pixels (px, py: [P]) over G
    depth-ordered Gaussians: [P, G] exponent, cutoff test, raw and clamped
    alpha, the alpha rule, the effective alpha, the transmittance after and
    before each Gaussian, and which Gaussians are composited."""
    dx = px[:, None] - m2[None, :, 0]
    dy = py[:, None] - m2[None, :, 1]
    power = -0.5 * (con[None, :, 0] * dx * dx + con[None, :, 2] * dy * dy) - con[None, :, 1] * dx * dy
    in_cut = (power <= 0.0) & (power >= POWER_CUT)
    alpha_raw = o[None, :] * torch.exp(power)
    alpha = torch.clamp(alpha_raw, max=ALPHA_MAX)
    valid = in_cut & (alpha >= ALPHA_MIN)
    a_eff = torch.where(valid, alpha, torch.zeros_like(alpha))
    one_minus = 1.0 - a_eff
    T_after = torch.cumprod(one_minus, dim=1)
    ones = torch.ones_like(T_after[:, :1])
    T_before = torch.cat([ones, T_after[:, :-1]], dim=1)
    included = valid & (T_after >= T_MIN)
    return power, in_cut, alpha_raw, alpha, valid, a_eff, one_minus, T_after, T_before, included


def _composite(m2, con, o, col, z, px, py, bg):
    """Composite a chunk of pixels (px, py: [P]) over G depth-ordered Gaussians."""
    G = m2.shape[0]
    pos = torch.arange(G)
    power, in_cut, alpha_raw, alpha, valid, a_eff, one_minus, T_after, T_before, included = \
        _inclusion(m2, con, o, px, py)
    w = torch.where(included, a_eff * T_before, torch.zeros_like(a_eff))
    C = w @ col  # [P,3]
    T_final = torch.prod(torch.where(included, one_minus, torch.ones_like(one_minus)), dim=1)
    img = C + T_final[:, None] * bg[None, :]
    last_pos = torch.where(included, pos[None, :], torch.full_like(pos[None, :], -1)).amax(dim=1) \
        if G > 0 else torch.full((px.shape[0],), -1, dtype=torch.long)
    n_comp = included.sum(dim=1) if G > 0 else torch.zeros(px.shape[0], dtype=torch.long)
    # Decision margins over the Gaussians the pixel reaches (T before >= 1e-4).
    # m_thr / m_dep cover every decision; m_thr_img / m_dep_img only those
    # whose flip could move the pixel colour by IMPACT_MIN or more (a flip of
    # Gaussian i changes the colour by at most alpha_i T_i (|c_i| + |rest|)).
    with torch.no_grad():
        P = px.shape[0]
        inf_row = torch.full((P,), math.inf, dtype=torch.float64)
        if G == 0:
            return img, T_final, last_pos, inf_row, inf_row, inf_row, inf_row, n_comp
        Tb = T_before.detach()
        pw = power.detach()
        ar = alpha_raw.detach()
        al = alpha.detach()
        reached = Tb >= T_MIN
        inf = torch.full_like(pw, math.inf)
        cmax = 2.0 * max(1.0, float(col.detach().max()), float(bg.max()))
        m_cut = torch.where(reached, (pw - POWER_CUT).abs() / abs(POWER_CUT), inf)
        m_alpha = torch.where(reached & in_cut, (ar - ALPHA_MIN).abs() / ALPHA_MIN, inf)
        m_T = torch.where(reached & valid, (T_after.detach() - T_MIN).abs() / T_MIN, inf)
        m_thr = torch.minimum(torch.minimum(m_cut, m_alpha), m_T).amin(dim=1)
        a_cut = torch.clamp(o.detach() * math.exp(POWER_CUT), max=ALPHA_MAX)[None, :]
        imp_cut = a_cut * Tb * cmax
        imp_alpha = ALPHA_MIN * Tb * cmax
        imp_T = al * Tb * cmax  # a flipped stop adds or removes this Gaussian's term
        m_img = torch.minimum(torch.minimum(torch.where(imp_cut >= IMPACT_MIN, m_cut, inf),
                                            torch.where(imp_alpha >= IMPACT_MIN, m_alpha, inf)),
                              torch.where(imp_T >= IMPACT_MIN, m_T, inf)).amin(dim=1)
        # depth order of consecutive contributing Gaussians
        vr = valid & reached
        posm = torch.where(vr, pos[None, :].expand_as(pw), torch.full_like(pos[None, :].expand_as(pw), -1))
        prev = torch.cummax(posm, dim=1).values
        prev = torch.cat([torch.full_like(prev[:, :1], -1), prev[:, :-1]], dim=1)
        has_prev = vr & (prev >= 0)
        pi = prev.clamp(min=0)
        zz = z[None, :].expand_as(pw)
        gap = torch.where(has_prev, (zz - z[pi]) / zz, inf)
        imp_dep = al * al.gather(1, pi) * Tb.gather(1, pi) * cmax
        m_dep = gap.amin(dim=1)
        m_dep_img = torch.where(imp_dep >= IMPACT_MIN, gap, inf).amin(dim=1)
    return img, T_final, last_pos, m_thr, m_dep, m_img, m_dep_img, n_comp


def _pixel_grid(width: int, height: int):
    jj, ii = torch.meshgrid(torch.arange(height), torch.arange(width), indexing="ij")
    return ii.flatten(), jj.flatten()


def _chunked(rec, order, cols, rows, bg, budget=4_000_000):
    G = int(order.numel())
    m2 = rec["mean2d"][order]
    con = rec["conic"][order]
    o = rec["opacity_t"][order]
    col = rec["rgb"][order]
    z = rec["z"].detach()[order]
    P = cols.numel()
    step = max(1, budget // max(G, 1))
    outs = []
    for s in range(0, P, step):
        px = cols[s:s + step].to(torch.float64) + 0.5
        py = rows[s:s + step].to(torch.float64) + 0.5
        outs.append(_composite(m2, con, o, col, z, px, py, bg))
    img = torch.cat([x[0] for x in outs]) if outs else torch.zeros((0, 3), dtype=torch.float64)
    T = torch.cat([x[1] for x in outs]) if outs else torch.zeros(0, dtype=torch.float64)
    lp = torch.cat([x[2] for x in outs]) if outs else torch.zeros(0, dtype=torch.long)
    extra = [torch.cat([x[k] for x in outs]) if outs else torch.zeros(0, dtype=torch.float64) for k in (3, 4, 5, 6)]
    ncomp = torch.cat([x[7] for x in outs]) if outs else torch.zeros(0, dtype=torch.long)
    last = torch.where(lp >= 0, order[lp.clamp(min=0)] if G > 0 else lp, torch.full_like(lp, -1))
    return (img, T, last, *extra, ncomp)


def render(scene: dict, cam, t: float, bg=(0.0, 0.0, 0.0), cull_temporal: bool = True,
           sh_degree: int = 3, rec: dict | None = None) -> dict:
    """Render the full image. Returns ``image`` [3,H,W], ``T`` [H,W] (final
    transmittance), ``last`` [H,W] (index of the last composited Gaussian, -1 if
    none), ``margin`` [H,W] (smallest relative margin of a threshold decision),
    ``margin_depth`` [H,W] (smallest relative depth gap between two Gaussians
    that both contribute), the same two restricted to decisions whose flip
    could change the colour by IMPACT_MIN or more (``margin_img``,
    ``margin_depth_img``), and the per-Gaussian records ``rec``."""
    cam = _cam(cam)
    if rec is None:
        rec = preprocess(scene, cam, t, cull_temporal, sh_degree)
    order = depth_order(rec)
    W, H = cam["width"], cam["height"]
    cols, rows = _pixel_grid(W, H)
    bg_t = torch.as_tensor(bg, dtype=torch.float64)
    img, T, last, mt, md, mi, mdi, _ = _chunked(rec, order, cols, rows, bg_t)
    return {
        "image": img.T.reshape(3, H, W), "T": T.reshape(H, W), "last": last.reshape(H, W),
        "margin": mt.reshape(H, W), "margin_depth": md.reshape(H, W),
        "margin_img": mi.reshape(H, W), "margin_depth_img": mdi.reshape(H, W), "rec": rec, "order": order,
    }


def render_pixels(scene: dict, cam, t: float, pixels, bg=(0.0, 0.0, 0.0), rec: dict | None = None,
                  budget: int = 4_000_000) -> dict:
    """Render only the listed pixels (int [P,2] as (column, row)). Also
    returns ``n_composited``, the number of Gaussians each pixel composited."""
    cam = _cam(cam)
    if rec is None:
        rec = preprocess(scene, cam, t)
    order = depth_order(rec)
    pix = torch.as_tensor(np.asarray(pixels), dtype=torch.long)
    bg_t = torch.as_tensor(bg, dtype=torch.float64)
    img, T, last, mt, md, mi, mdi, nc = _chunked(rec, order, pix[:, 0], pix[:, 1], bg_t, budget)
    return {"rgb": img, "T": T, "last": last, "margin": mt, "margin_depth": md, "margin_img": mi,
            "margin_depth_img": mdi, "n_composited": nc}


def pixel_alternatives(rec: dict, pixel, rel_margin: float, rel_gap: float, bg=(0.0, 0.0, 0.0)) -> list:
    """The colours one pixel takes under every result that the rounding of its
    threshold decisions and depth order leaves open (Eq. 3 with the per-pixel
    rules of this module): the colour in the global depth order with every
    decision as computed, then one colour per open decision with that decision
    taken the other way, and one with all of them taken the other way.

    Open decisions, over the Gaussians the pixel reaches (T before >= 1e-4):
      cutoff   |power + 4.5| / 4.5 < rel_margin         (skip <-> keep)
      alpha    |o_t e^power - 1/255| / (1/255) < rel_margin (skip <-> keep)
      stop     |T' - 1e-4| / 1e-4 < rel_margin           (stop <-> composite)
      depth    consecutive contributors whose depths differ by less than
               rel_gap (relative)                         (order swapped)
    Returns a list of float64 [3] tensors, the computed colour first."""
    order = depth_order(rec)
    bg_t = torch.as_tensor(bg, dtype=torch.float64)
    px = torch.tensor([float(pixel[0]) + 0.5], dtype=torch.float64)
    py = torch.tensor([float(pixel[1]) + 0.5], dtype=torch.float64)
    with torch.no_grad():
        m2 = rec["mean2d"].detach()[order]
        con = rec["conic"].detach()[order]
        o = rec["opacity_t"].detach()[order]
        col = rec["rgb"].detach()[order]
        z = rec["z"].detach()[order]
        G = int(order.numel())
        if G == 0:
            return [bg_t.clone()]
        power, in_cut, alpha_raw, alpha, valid = [x[0] for x in _inclusion(m2, con, o, px, py)[:5]]

        def walk(valid_mask, perm, stop_flips):
            """Front-to-back compositing of one pixel over the positions in
            ``perm`` with the given validity; ``stop_flips`` holds the
            positions whose stop decision is taken the other way. Returns the
            colour and the open decisions met: (kind, position)."""
            C = torch.zeros(3, dtype=torch.float64)
            T = 1.0
            opened = []
            for p in perm:
                if T < T_MIN:
                    break
                if abs(float(power[p]) - POWER_CUT) / abs(POWER_CUT) < rel_margin:
                    opened.append(("cut", p))
                if bool(in_cut[p]) and abs(float(alpha_raw[p]) - ALPHA_MIN) / ALPHA_MIN < rel_margin:
                    opened.append(("alpha", p))
                if not bool(valid_mask[p]):
                    continue
                a = float(alpha[p])
                Tn = T * (1.0 - a)
                stop = Tn < T_MIN
                if abs(Tn - T_MIN) / T_MIN < rel_margin:
                    opened.append(("stop", p))
                if p in stop_flips:
                    stop = not stop
                if stop:
                    break
                C = C + col[p] * (a * T)
                T = Tn
            return C + T * bg_t, opened

        # candidates: positions inside the cutoff or within the margin of it
        near = (power <= 0.0) & (power >= POWER_CUT * (1.0 + 2.0 * rel_margin))
        perm = torch.nonzero(near).flatten().tolist()
        base, opened = walk(valid, perm, set())
        out = [base]
        flips_v, flips_s = [], set()
        for kind, p in opened:
            v = valid.clone()
            if kind == "stop":
                out.append(walk(v, perm, {p})[0])
                flips_s.add(p)
            else:
                v[p] = ~v[p]
                out.append(walk(v, perm, set())[0])
                flips_v.append(p)
        # depth ties between consecutive contributors (composited in the base walk)
        contrib = []  # indices into perm
        T = 1.0
        for i, p in enumerate(perm):
            if not bool(valid[p]):
                continue
            Tn = T * (1.0 - float(alpha[p]))
            if Tn < T_MIN:
                break
            contrib.append(i)
            T = Tn
        close = [(a, b) for a, b in zip(contrib[:-1], contrib[1:])
                 if (z[perm[b]] - z[perm[a]]) / z[perm[b]] < rel_gap]
        for a, b in close:
            p2 = list(perm)
            p2[a], p2[b] = perm[b], perm[a]
            out.append(walk(valid, p2, set())[0])
        if len(opened) + len(close) > 1:
            v = valid.clone()
            for p in flips_v:
                v[p] = ~v[p]
            p2 = list(perm)
            for a, b in close:
                p2[a], p2[b] = perm[b], perm[a]
            out.append(walk(v, p2, flips_s)[0])
    return out


def composited_counts(scene: dict, cam, t: float, rec: dict | None = None, budget: int = 4_000_000) -> torch.Tensor:
    """Number of pixels of the image each Gaussian is composited into (int64
    [N]; 0 for Gaussians no pixel takes), by the same per-pixel rules."""
    cam = _cam(cam)
    if rec is None:
        rec = preprocess(scene, cam, t)
    order = depth_order(rec)
    n = int(rec["z"].shape[0])
    counts = torch.zeros(n, dtype=torch.long)
    G = int(order.numel())
    if G == 0:
        return counts
    with torch.no_grad():
        m2 = rec["mean2d"].detach()[order]
        con = rec["conic"].detach()[order]
        o = rec["opacity_t"].detach()[order]
        cols, rows = _pixel_grid(cam["width"], cam["height"])
        step = max(1, budget // G)
        for s in range(0, cols.numel(), step):
            px = cols[s:s + step].to(torch.float64) + 0.5
            py = rows[s:s + step].to(torch.float64) + 0.5
            included = _inclusion(m2, con, o, px, py)[-1]
            counts[order] += included.sum(dim=0)
    return counts


REC_GRAD_KEYS = ("mean2d", "conic", "opacity_t", "rgb")


def render_grad(scene: dict, cam, t: float, grad_image, bg=(0.0, 0.0, 0.0), sh_degree: int = 3) -> dict:
    """Gradient of L = sum(grad_image * image) w.r.t. every parameter, by
    reverse-mode automatic differentiation of ``render`` in float64. The
    composite is differentiated pixel chunk by pixel chunk into per-Gaussian
    record gradients (d mean2d, d conic, d opacity_t, d rgb), which are then
    pulled back through ``preprocess``. Returns the parameter gradients under
    the parameter names and the record gradients under ``rec_<name>``."""
    cam = _cam(cam)
    W, H = cam["width"], cam["height"]
    cols, rows = _pixel_grid(W, H)
    gi = torch.as_tensor(np.asarray(grad_image), dtype=torch.float64).reshape(3, H * W).T
    return _grad_over(scene, cam, t, cols, rows, gi, bg, sh_degree, None, 2_000_000)


def render_grad_pixels(scene: dict, cam, t: float, pixels, grad_rgb, bg=(0.0, 0.0, 0.0), keep=None,
                       sh_degree: int = 3, budget: int = 2_000_000) -> dict:
    """Gradient of L = sum over the listed pixels (int [P,2] as (column, row))
    of grad_rgb [P,3] * rgb, the same function as ``render_grad`` restricted to
    those pixels. ``keep`` (bool [N]) optionally limits the compositing to a
    subset of the Gaussians, kept in the global depth order; callers pass the
    Gaussians whose 3-sigma box meets the pixels, which changes no listed pixel
    since every other Gaussian fails the power >= -4.5 cutoff there."""
    cam = _cam(cam)
    pix = torch.as_tensor(np.asarray(pixels), dtype=torch.long)
    gi = torch.as_tensor(np.asarray(grad_rgb), dtype=torch.float64).reshape(-1, 3)
    return _grad_over(scene, cam, t, pix[:, 0], pix[:, 1], gi, bg, sh_degree, keep, budget)


def _grad_over(scene, cam, t, cols, rows, gi, bg, sh_degree, keep, budget):
    leaves = {k: v.detach().clone().requires_grad_(True) for k, v in scene.items()}
    rec = preprocess(leaves, cam, t, True, sh_degree)
    recd = {k: (rec[k].detach().clone().requires_grad_(True) if k in REC_GRAD_KEYS else rec[k])
            for k in rec}
    order = depth_order(recd)
    if keep is not None:
        keep_t = torch.as_tensor(np.asarray(keep), dtype=torch.bool)
        order = order[keep_t[order]]
    bg_t = torch.as_tensor(bg, dtype=torch.float64)
    G = max(int(order.numel()), 1)
    step = max(1, budget // G)
    m2 = recd["mean2d"][order]
    con = recd["conic"][order]
    o = recd["opacity_t"][order]
    col = recd["rgb"][order]
    z = recd["z"].detach()[order]
    P = int(cols.numel())
    for s in range(0, P, step):
        px = cols[s:s + step].to(torch.float64) + 0.5
        py = rows[s:s + step].to(torch.float64) + 0.5
        img = _composite(m2, con, o, col, z, px, py, bg_t)[0]
        (img * gi[s:s + step]).sum().backward(retain_graph=True)
    out = {}
    rec_grads = []
    rec_outs = []
    for k in REC_GRAD_KEYS:
        g = recd[k].grad
        if g is None:
            g = torch.zeros_like(recd[k])
        out["rec_" + k] = g.detach()
        rec_grads.append(g)
        rec_outs.append(rec[k])
    torch.autograd.backward(rec_outs, rec_grads)
    for k in leaves:
        g = leaves[k].grad
        out[k] = torch.zeros_like(leaves[k]) if g is None else g.detach()
    return out
