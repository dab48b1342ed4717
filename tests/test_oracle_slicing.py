"""Pins for Sigma4 and the temporal slice (Sec. 3.2.2 Eq. 7, appendix A.3)
against direct Gaussian conditioning by generic matrix inversion."""
import numpy as np
import pytest
import torch

import oracle


def _random_gaussians(n, seed, ls_lo=-4.0, ls_hi=0.5):
    rng = np.random.default_rng(seed)
    rot = torch.as_tensor(rng.normal(0, 1, (n, 8)))
    s = torch.as_tensor(np.exp(rng.uniform(ls_lo, ls_hi, (n, 4))))
    mean = torch.as_tensor(rng.uniform(-1, 1, (n, 4)))
    R = oracle.rotor_to_matrix(oracle.rotor_normalize(rot))
    return mean, oracle.covariance4(R, s), s, R


def test_covariance_is_r_s2_rt():
    mean, S4, s, R = _random_gaussians(100, 0)
    Rn, sn = R.numpy(), s.numpy()
    for i in range(100):
        ref = Rn[i] @ np.diag(sn[i]) @ np.diag(sn[i]).T @ Rn[i].T
        np.testing.assert_allclose(S4[i].numpy(), ref, rtol=1e-12, atol=1e-16)
        w = np.linalg.eigvalsh(S4[i].numpy())
        np.testing.assert_allclose(np.sort(w), np.sort(sn[i] ** 2), rtol=1e-9, atol=1e-15)


@pytest.mark.parametrize("t", [0.0, 0.37, 1.0])
def test_slice_matches_inverse_based_conditioning(t):
    """Appendix A.3 route through Sigma4^{-1} = [[A, eta], [eta^T, Z]]:
    Sigma3 = A^{-1}; A g = eta; mu(t) = mu_xyz - g (t - mu_t); lambda = Z - g^T A g."""
    mean, S4, s, R = _random_gaussians(300, 1, -2.5, 0.5)
    mu3, sig3, temporal, lam_dt2 = oracle.slice_at(mean, S4, t)
    for i in range(300):
        inv = np.linalg.inv(S4[i].numpy())
        A, eta, Z = inv[:3, :3], inv[:3, 3], inv[3, 3]
        g = np.linalg.solve(A, eta)
        dt = t - mean[i, 3].item()
        lam = Z - g @ A @ g
        np.testing.assert_allclose(sig3[i].numpy(), np.linalg.inv(A), rtol=1e-7, atol=1e-12)
        np.testing.assert_allclose(mu3[i].numpy(), mean[i, :3].numpy() - g * dt, rtol=1e-8, atol=1e-10)
        np.testing.assert_allclose(lam, 1.0 / S4[i, 3, 3].item(), rtol=1e-8)
        np.testing.assert_allclose(lam_dt2[i].item(), lam * dt * dt, rtol=1e-8, atol=1e-14)
        np.testing.assert_allclose(temporal[i].item(), np.exp(-0.5 * lam * dt * dt), rtol=1e-8)


def test_density_factorises_into_temporal_times_sliced():
    """G4(x, t) = exp(-1/2 lambda (t-mu_t)^2) exp(-1/2 (x-mu(t))^T Sigma3^{-1} (x-mu(t))) (Eq. 6)."""
    mean, S4, s, R = _random_gaussians(200, 2, -1.5, 0.3)
    rng = np.random.default_rng(3)
    for i in range(200):
        for _ in range(5):
            x = mean[i, :3].numpy() + rng.normal(0, 0.3, 3)
            t = mean[i, 3].item() + rng.normal(0, 0.3)
            mu3, sig3, temporal, _ = oracle.slice_at(mean[i:i + 1], S4[i:i + 1], t)
            d4 = np.concatenate([x, [t]]) - mean[i].numpy()
            full = np.exp(-0.5 * d4 @ np.linalg.solve(S4[i].numpy(), d4))
            d3 = x - mu3[0].numpy()
            fact = temporal.item() * np.exp(-0.5 * d3 @ np.linalg.solve(sig3[0].numpy(), d3))
            np.testing.assert_allclose(fact, full, rtol=1e-8, atol=1e-300)


def test_sliced_covariance_is_psd_and_bounded():
    """Schur complement of an SPD matrix: lambda_min(Sigma3) >= min s^2 and
    W = Sigma4[3,3] lies in [min s^2, max s^2] (Rayleigh quotient)."""
    mean, S4, s, R = _random_gaussians(2000, 4)
    _, sig3, _, _ = oracle.slice_at(mean, S4, 0.5)
    smin2 = (s.min(dim=1).values) ** 2
    smax2 = (s.max(dim=1).values) ** 2
    w = torch.linalg.eigvalsh(sig3)
    assert (w[:, 0] >= smin2 * (1 - 1e-7)).all()
    W = S4[:, 3, 3]
    assert (W >= smin2 * (1 - 1e-12)).all() and (W <= smax2 * (1 + 1e-12)).all()


def test_uncoupled_gaussian_does_not_move():
    """tau = (b03, b13, b23, p) = 0: no space-time coupling, V = 0, so mu(t) = mu_xyz,
    Sigma3 = R3 diag(s_xyz^2) R3^T and lambda = 1 / s_t^2 (Sec. 3.2.1)."""
    rng = np.random.default_rng(5)
    rot = torch.zeros(50, 8, dtype=torch.float64)
    rot[:, :4] = torch.as_tensor(rng.normal(0, 1, (50, 4)))
    s = torch.as_tensor(np.exp(rng.uniform(-3, 0, (50, 4))))
    mean = torch.as_tensor(rng.uniform(-1, 1, (50, 4)))
    R = oracle.rotor_to_matrix(oracle.rotor_normalize(rot))
    mu3, sig3, temporal, lam_dt2 = oracle.slice_at(mean, oracle.covariance4(R, s), 0.25)
    assert torch.allclose(mu3, mean[:, :3], atol=1e-15)
    R3 = R[:, :3, :3]
    ref = R3 @ torch.diag_embed(s[:, :3] ** 2) @ R3.transpose(-1, -2)
    assert torch.allclose(sig3, ref, atol=1e-15)
    assert torch.allclose(lam_dt2, (0.25 - mean[:, 3]) ** 2 / s[:, 3] ** 2, rtol=1e-12)
