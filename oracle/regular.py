"""Regularisers of the optimisation (Sec. 3.3), plain FP64 definitions.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``.

  knn4d        the K nearest neighbours of each 4D mean: Euclidean distance
               after dividing x, y, z by the spatial and t by the temporal
               scene scale; brute force over all pairs, ties to the smaller
               index, the point itself excluded
  speeds       s = V / W of Sigma4 = R S S^T R^T (Sec. 3.2.2: the sliced
               centre moves by (t - mu_t) V / W)
  entropy      L_entropy = 1/N sum -o log o, o = sigmoid(logit)
  consistency  L_consistent4D = 1/N sum_i || s_i - 1/K sum_{j in Omega_i} s_j ||_1
  losses_and_grads  both values and their gradients (torch.autograd), the
               neighbour lists held constant
"""
from __future__ import annotations

import torch

from .rotor import rotor_normalize, rotor_to_matrix
from .slicing import covariance4


def knn4d(means: torch.Tensor, scale_xyz: float, scale_t: float, k: int, chunk: int = 1024):
    """(indices [N,k] int64, squared scaled distances [N,k] float64)."""
    m = torch.as_tensor(means, dtype=torch.float64)
    q = torch.cat([m[:, :3] / scale_xyz, m[:, 3:4] / scale_t], 1)
    n = q.shape[0]
    idx_out, d_out = [], []
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        d2 = ((q[a:b, None, :] - q[None, :, :]) ** 2).sum(-1)
        d2[torch.arange(b - a), torch.arange(a, b)] = float("inf")
        d_sorted, order = torch.sort(d2, dim=1, stable=True)  # equal distances keep index order
        idx_out.append(order[:, :k])
        d_out.append(d_sorted[:, :k])
    return torch.cat(idx_out), torch.cat(d_out)


def speeds(scene: dict) -> torch.Tensor:
    R = rotor_to_matrix(rotor_normalize(scene["rotor"]))
    s4 = covariance4(R, torch.exp(scene["logscale"]))
    return s4[:, :3, 3] / s4[:, 3:4, 3]


def entropy(scene: dict) -> torch.Tensor:
    o = torch.sigmoid(scene["logit"])
    return (-o * torch.log(o)).mean()


def consistency(scene: dict, knn: torch.Tensor) -> torch.Tensor:
    s = speeds(scene)
    r = s - s[knn].mean(1)
    return r.abs().sum(1).mean()


def losses_and_grads(scene: dict, knn, lam_e: float = 1.0, lam_c: float = 1.0) -> dict:
    leaves = {k: torch.as_tensor(v, dtype=torch.float64).clone().requires_grad_(True) for k, v in scene.items()}
    knn = torch.as_tensor(knn, dtype=torch.long)
    le = entropy(leaves)
    lc = consistency(leaves, knn)
    (lam_e * le + lam_c * lc).backward()
    out = {"entropy": le.detach(), "consistency": lc.detach()}
    for k, v in leaves.items():
        out["grad_" + k] = torch.zeros_like(v) if v.grad is None else v.grad.detach()
    return out
