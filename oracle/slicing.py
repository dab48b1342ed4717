"""4D covariance and its temporal slice (Sec. 3.2.1 Eq. 5; Sec. 3.2.2 Eq. 6-7;
appendix A.3, 'Avoiding Numerical Instability')."""
from __future__ import annotations

import torch


def covariance4(R: torch.Tensor, scale: torch.Tensor) -> torch.Tensor:
    """Sigma4 = R S S^T R^T with S = diag(s_x, s_y, s_z, s_t) (Sec. 3.2.1)."""
    rs = R * scale[..., None, :]  # R S
    return rs @ rs.transpose(-1, -2)


def slice_at(mean4: torch.Tensor, sigma4: torch.Tensor, t: float):
    """Condition a 4D Gaussian on time t (Eq. 7, numerically stable form of A.3).

    With Sigma4 = [[U, V], [V^T, W]] (U 3x3, V 3x1, W scalar):
        lambda   = 1 / W
        Sigma3   = U - V V^T / W        (A^{-1}, without inverting A)
        mu(t)    = mu_xyz + (t - mu_t) V / W
        temporal = exp(-1/2 lambda (t - mu_t)^2)   (decay of the opacity)
    Returns (mu3 [...,3], sigma3 [...,3,3], temporal [...], lam_dt2 [...]) where
    lam_dt2 = lambda (t - mu_t)^2 is the quantity the visibility test compares
    with 16 (Sec. 3.2.2).
    """
    U = sigma4[..., :3, :3]
    V = sigma4[..., :3, 3]
    W = sigma4[..., 3, 3]
    dt = t - mean4[..., 3]
    sigma3 = U - V[..., :, None] * V[..., None, :] / W[..., None, None]
    mu3 = mean4[..., :3] + (dt / W)[..., None] * V
    lam_dt2 = dt * dt / W
    temporal = torch.exp(-0.5 * lam_dt2)
    return mu3, sigma3, temporal, lam_dt2
