"""Pins for the oracle's real SH basis (degree <= 3) against scipy's complex
spherical harmonics and by quadrature on the sphere."""
import math

import numpy as np
import pytest
import torch

import oracle

special = pytest.importorskip("scipy.special")


def _dirs(theta, phi):
    return np.stack([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)], -1)


def test_basis_matches_scipy_real_harmonics():
    """Y_{l,m} = sqrt2 Im Y_l^|m| (m<0), Y_l^0, sqrt2 Re Y_l^m (m>0), k = l^2 + l + m,
    with scipy's Y_l^m (Condon-Shortley phase included)."""
    rng = np.random.default_rng(0)
    theta = np.arccos(rng.uniform(-1, 1, 500))
    phi = rng.uniform(0, 2 * math.pi, 500)
    B = oracle.sh_basis(torch.as_tensor(_dirs(theta, phi))).numpy()
    for l in range(4):
        for m in range(-l, l + 1):
            Y = special.sph_harm_y(l, abs(m), theta, phi)
            if m < 0:
                ref = math.sqrt(2) * Y.imag
            elif m == 0:
                ref = Y.real
            else:
                ref = math.sqrt(2) * Y.real
            np.testing.assert_allclose(B[:, l * l + l + m], ref, atol=1e-12)


def test_basis_is_orthonormal_by_quadrature():
    xg, wg = np.polynomial.legendre.leggauss(16)  # exact for degree <= 31 in cos(theta)
    nphi = 16
    phi = (np.arange(nphi) + 0.5) * 2 * math.pi / nphi
    th = np.arccos(xg)
    TH, PH = np.meshgrid(th, phi, indexing="ij")
    W = np.repeat(wg[:, None], nphi, 1) * (2 * math.pi / nphi)
    B = oracle.sh_basis(torch.as_tensor(_dirs(TH, PH))).numpy().reshape(-1, 16)
    G = (B * W.reshape(-1, 1)).T @ B
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_degree_zero_colour_is_constant():
    c = torch.zeros(10, 16, 3, dtype=torch.float64)
    c[:, 0, :] = torch.linspace(-1, 1, 30, dtype=torch.float64).reshape(10, 3)
    c[:, 1:, :] = 7.0  # ignored at degree 0
    d = torch.nn.functional.normalize(torch.randn(10, 3, dtype=torch.float64), dim=-1)
    rgb = oracle.sh_color(c, d, degree=0)
    ref = torch.clamp(0.5 + c[:, 0, :] / (2 * math.sqrt(math.pi)), min=0)
    assert torch.allclose(rgb, ref, atol=1e-15)


def test_colour_offset_and_clamp():
    c = torch.zeros(1, 16, 3, dtype=torch.float64)
    c[0, 0] = torch.tensor([0.0, -10.0, 1.0], dtype=torch.float64)
    rgb = oracle.sh_color(c, torch.tensor([[0.0, 0.0, 1.0]], dtype=torch.float64))
    assert rgb[0, 0].item() == 0.5 and rgb[0, 1].item() == 0.0
    assert abs(rgb[0, 2].item() - (0.5 + 0.5 / math.sqrt(math.pi))) < 1e-15
