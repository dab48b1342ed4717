"""Real spherical harmonics up to degree 3 for the view-dependent colour
(Sec. 3.1: each Gaussian carries SH coefficients for its colour).

Definition used (the paper defers the details to 3D Gaussian Splatting): with
the complex Y_l^m that include the Condon-Shortley phase, the real basis is
    Y_{l,m} = sqrt(2) Im Y_l^{|m|}   (m < 0)
    Y_{l,0} = Y_l^0
    Y_{l,m} = sqrt(2) Re Y_l^m       (m > 0)
at index k = l^2 + l + m, evaluated on the unit direction d = (x, y, z).
The polynomials below are those functions written out in Cartesian form, with
the normalisation constants computed from their closed forms.
"""
from __future__ import annotations

import math

import torch

_PI = math.pi
K00 = 0.5 / math.sqrt(_PI)
K1 = math.sqrt(3.0 / (4.0 * _PI))
K2a = 0.5 * math.sqrt(15.0 / _PI)          # |m| = 1, 2 off-diagonal terms
K2b = 0.25 * math.sqrt(5.0 / _PI)          # m = 0
K2c = 0.25 * math.sqrt(15.0 / _PI)         # m = 2
K3a = 0.25 * math.sqrt(35.0 / (2.0 * _PI))  # |m| = 3
K3b = 0.5 * math.sqrt(105.0 / _PI)         # m = -2
K3c = 0.25 * math.sqrt(21.0 / (2.0 * _PI))  # |m| = 1
K3d = 0.25 * math.sqrt(7.0 / _PI)          # m = 0
K3e = 0.25 * math.sqrt(105.0 / _PI)        # m = 2


def sh_basis(d: torch.Tensor) -> torch.Tensor:
    """The 16 real SH basis values at unit directions d [...,3] -> [...,16]."""
    x, y, z = d[..., 0], d[..., 1], d[..., 2]
    xx, yy, zz = x * x, y * y, z * z
    one = torch.ones_like(x)
    return torch.stack([
        K00 * one,                              # l=0
        -K1 * y, K1 * z, -K1 * x,               # l=1, m=-1,0,1
        K2a * x * y,                            # l=2, m=-2
        -K2a * y * z,                           # m=-1
        K2b * (2 * zz - xx - yy),               # m=0
        -K2a * x * z,                           # m=1
        K2c * (xx - yy),                        # m=2
        -K3a * y * (3 * xx - yy),               # l=3, m=-3
        K3b * x * y * z,                        # m=-2
        -K3c * y * (4 * zz - xx - yy),          # m=-1
        K3d * z * (2 * zz - 3 * xx - 3 * yy),   # m=0
        -K3c * x * (4 * zz - xx - yy),          # m=1
        K3e * z * (xx - yy),                    # m=2
        -K3a * x * (xx - 3 * yy),               # m=3
    ], dim=-1)


def sh_color(coeffs: torch.Tensor, d: torch.Tensor, degree: int = 3) -> torch.Tensor:
    """rgb = max(0, sum_k Y_k(d) c_k + 0.5) using the bands l <= degree.
    coeffs [...,16,3], d [...,3] unit vectors -> [...,3]."""
    basis = sh_basis(d)
    nb = (degree + 1) ** 2
    rgb = (basis[..., :nb, None] * coeffs[..., :nb, :]).sum(-2) + 0.5
    return torch.clamp(rgb, min=0.0)
