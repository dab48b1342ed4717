"""World -> camera -> screen and the EWA 2D covariance (Sec. 3.1:
Sigma' = J V Sigma V^T J^T with J the Jacobian of the affine approximation of
the perspective projection and V the camera extrinsic rotation).

Conventions (the paper defers them to 3D Gaussian Splatting; stated here):
  * camera: row-major [R | t], p_c = R x + t, OpenCV axes, z forward;
  * screen position u = fx x/z + cx, v = fy y/z + cy (pixel (i, j) is centred
    at (i + 0.5, j + 0.5));
  * J is taken at the camera-space mean with x/z and y/z clamped to
    +-1.3 tan(fov/2) (tan(fov_x/2) = W / (2 fx), tan(fov_y/2) = H / (2 fy));
  * a 0.3 px^2 low-pass term is added to the diagonal of Sigma';
  * Gaussians with z <= near (0.2) or det(Sigma') <= 0 are culled.
"""
from __future__ import annotations

import torch


def camera_tensors(cam) -> dict:
    """Float64 view of a synth.Camera (its f32 values upcast exactly)."""
    w2c = torch.as_tensor(cam.world_to_cam, dtype=torch.float64)
    return {
        "R": w2c[:, :3].clone(), "t": w2c[:, 3].clone(),
        "fx": float(cam.fx), "fy": float(cam.fy),
        "cx": float(cam.cx), "cy": float(cam.cy),
        "width": int(cam.width), "height": int(cam.height),
    }


def project(mu3: torch.Tensor, sigma3: torch.Tensor, cam: dict, dilation: float = 0.3,
            clamp: bool = True):
    """Project sliced 3D Gaussians. Returns a dict with camera-space position
    ``pc`` [N,3], depth ``z`` [N], screen mean ``mean2d`` [N,2], 2D covariance
    ``cov2d`` [N,2,2] (dilated), ``det`` [N] and conic (a, b, c) of its inverse
    such that the exponent is -1/2 (a dx^2 + 2 b dx dy + c dy^2)."""
    R, t = cam["R"], cam["t"]
    fx, fy, cx, cy = cam["fx"], cam["fy"], cam["cx"], cam["cy"]
    pc = mu3 @ R.T + t
    x, y, z = pc[..., 0], pc[..., 1], pc[..., 2]
    if clamp:
        limx = 1.3 * (cam["width"] / (2.0 * fx))
        limy = 1.3 * (cam["height"] / (2.0 * fy))
        tx = torch.clamp(x / z, -limx, limx) * z
        ty = torch.clamp(y / z, -limy, limy) * z
    else:
        tx, ty = x, y
    zero = torch.zeros_like(z)
    J = torch.stack([
        torch.stack([fx / z, zero, -fx * tx / (z * z)], -1),
        torch.stack([zero, fy / z, -fy * ty / (z * z)], -1),
    ], -2)  # [N,2,3]
    T = J @ R  # [N,2,3]
    cov = T @ sigma3 @ T.transpose(-1, -2)
    eye2 = torch.eye(2, dtype=cov.dtype)
    cov = cov + dilation * eye2
    a, b, c = cov[..., 0, 0], cov[..., 0, 1], cov[..., 1, 1]
    det = a * c - b * b
    safe = torch.where(det > 0, det, torch.ones_like(det))
    conic = torch.stack([c / safe, -b / safe, a / safe], -1)
    mean2d = torch.stack([fx * x / z + cx, fy * y / z + cy], -1)
    return {"pc": pc, "z": z, "mean2d": mean2d, "cov2d": cov, "det": det, "conic": conic}
