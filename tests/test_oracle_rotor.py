"""Pins for the oracle's rotor normalisation (appendix A.1) and rotor -> matrix
map (appendix A.2) against the geometric-algebra definition u' = r u r^dagger,
computed here by a brute-force Clifford-algebra product independent of the
oracle's 16 closed-form entries."""
import math
import os

import numpy as np
import pytest
import torch

import oracle
from oracle.rotor import rotor_epsilon, rotor_epsilon_grad

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# storage order (s, b01, b02, b12, b03, b13, b23, p) -> blade bitmasks over e0..e3
BLADES = [0b0000, 0b0011, 0b0101, 0b0110, 0b1001, 0b1010, 0b1100, 0b1111]


def _blade_sign(a: int, b: int) -> int:
    """Sign of e_A e_B for an orthonormal Euclidean basis (count transpositions)."""
    a >>= 1
    swaps = 0
    while a:
        swaps += bin(a & b).count("1")
        a >>= 1
    return -1 if swaps & 1 else 1


def _gp(x: dict, y: dict) -> dict:
    out: dict = {}
    for a, ca in x.items():
        for b, cb in y.items():
            k = a ^ b
            out[k] = out.get(k, 0.0) + _blade_sign(a, b) * ca * cb
    return out


def _reverse(x: dict) -> dict:
    out = {}
    for a, c in x.items():
        g = bin(a).count("1")
        out[a] = c * (-1 if (g * (g - 1) // 2) % 2 else 1)
    return out


def sandwich_matrix(r: np.ndarray) -> np.ndarray:
    """Column j = r e_j r^dagger, from the Clifford product (Eq. 'rotor4-rotation')."""
    rv = {BLADES[i]: float(r[i]) for i in range(8)}
    rr = _reverse(rv)
    M = np.zeros((4, 4))
    for j in range(4):
        v = _gp(_gp(rv, {1 << j: 1.0}), rr)
        for i in range(4):
            M[i, j] = v.get(1 << i, 0.0)
        # no non-vector part survives for a normalised rotor
        rest = sum(abs(c) for k, c in v.items() if bin(k).count("1") != 1)
        assert rest < 1e-12
    return M


def _rand_rotors(n, seed):
    rng = np.random.default_rng(seed)
    return torch.as_tensor(rng.normal(0, 1, (n, 8)), dtype=torch.float64)


def test_normalised_rotor_satisfies_both_conditions():
    r = _rand_rotors(2000, 0)
    rn = oracle.rotor_normalize(r)
    assert torch.allclose((rn * rn).sum(-1), torch.ones(2000, dtype=torch.float64), atol=1e-14, rtol=0)
    assert rotor_epsilon(rn).abs().max() < 1e-14
    # r r^dagger = 1 as a multivector (both conditions at once)
    for i in range(20):
        rv = {BLADES[k]: float(rn[i, k]) for k in range(8)}
        p = _gp(rv, _reverse(rv))
        assert abs(p.get(0, 0) - 1) < 1e-13
        assert all(abs(c) < 1e-13 for k, c in p.items() if k != 0)


def test_normalise_is_idempotent():
    rn = oracle.rotor_normalize(_rand_rotors(500, 1))
    assert torch.allclose(oracle.rotor_normalize(rn), rn, atol=1e-15, rtol=0)


def test_root_step_identity_and_printed_root():
    """f(r + delta grad eps) = eps (1 + delta^2) + l^2 delta exactly, and the delta
    used equals the root printed in appendix A.1, (-l^2 + sqrt(l^4-4eps^2))/(2 eps)."""
    r = _rand_rotors(1000, 2)
    eps = rotor_epsilon(r)
    l2 = (r * r).sum(-1)
    for delta in (0.1, -0.37, 1.3):
        lhs = rotor_epsilon(r + delta * rotor_epsilon_grad(r))
        rhs = eps * (1 + delta ** 2) + l2 * delta
        assert torch.allclose(lhs, rhs, atol=1e-12, rtol=0)
    printed = (-l2 + torch.sqrt(l2 * l2 - 4 * eps * eps)) / (2 * eps)
    ours = -2 * eps / (l2 + torch.sqrt(l2 * l2 - 4 * eps * eps))
    m = eps.abs() > 1e-3
    assert torch.allclose(printed[m], ours[m], rtol=1e-10, atol=1e-12)
    # and this delta is the step F_norm takes: epsilon after the step is 0
    r1 = r + ours[:, None] * rotor_epsilon_grad(r)
    assert rotor_epsilon(r1).abs().max() < 1e-12


def test_small_epsilon_step_tends_to_minus_xi():
    """With l^2 = 1 + chi, eps = xi small, delta -> -xi (appendix A.1 sign choice)."""
    r = torch.zeros(1, 8, dtype=torch.float64)
    r[0, 0] = 1.0
    r[0, 7] = 1e-6  # p s = 1e-6
    eps = rotor_epsilon(r)
    rn = oracle.rotor_normalize(r)
    l2 = (r * r).sum(-1)
    delta = -2 * eps / (l2 + torch.sqrt(l2 * l2 - 4 * eps * eps))
    assert abs(delta.item() + eps.item()) < 1e-11
    assert rotor_epsilon(rn).abs().item() < 1e-16


def test_degenerate_rotors_map_to_identity():
    r = torch.zeros(3, 8, dtype=torch.float64)
    r[1, 0] = 1.0
    r[1, 7] = 1.0  # s = p, rest 0: l^4 = 4 eps^2, the step zeroes the rotor
    r[2, 0] = 2.5
    rn = oracle.rotor_normalize(r)
    ident = torch.zeros(8, dtype=torch.float64)
    ident[0] = 1
    assert torch.equal(rn[0], ident)
    assert torch.equal(rn[1], ident)
    assert torch.allclose(rn[2], ident)
    assert torch.allclose(oracle.rotor_to_matrix(rn), torch.eye(4, dtype=torch.float64).expand(3, 4, 4))


def test_matrix_equals_sandwich_product():
    rn = oracle.rotor_normalize(_rand_rotors(200, 3))
    R = oracle.rotor_to_matrix(rn).numpy()
    for i in range(200):
        np.testing.assert_allclose(R[i], sandwich_matrix(rn[i].numpy()), atol=1e-13, rtol=0)


def test_matrix_is_proper_rotation():
    rn = oracle.rotor_normalize(_rand_rotors(2000, 4))
    R = oracle.rotor_to_matrix(rn)
    I = torch.eye(4, dtype=torch.float64)
    assert (R.transpose(-1, -2) @ R - I).abs().max() < 1e-13
    assert (torch.linalg.det(R) - 1).abs().max() < 1e-12


def test_flipped_epsilon_sign_is_not_a_rotation():
    """The summary formula of A.1 flips the b02 b13 and b03 b12 signs; a rotor
    normalised with it does not give an orthogonal A.2 matrix, so the oracle
    uses the sign of the normalisation conditions (reading recorded in docs)."""
    r = _rand_rotors(500, 5)

    def eps_alt(x):
        s, b01, b02, b12, b03, b13, b23, p = [x[..., k] for k in range(8)]
        return p * s - b01 * b23 - b02 * b13 + b03 * b12

    def grad_alt(x):
        s, b01, b02, b12, b03, b13, b23, p = [x[..., k] for k in range(8)]
        return torch.stack([p, -b23, -b13, b03, b12, -b02, -b01, s], -1)

    e = eps_alt(r)
    l2 = (r * r).sum(-1)
    d = -2 * e / (l2 + torch.sqrt(torch.clamp(l2 * l2 - 4 * e * e, min=0)))
    r1 = r + d[:, None] * grad_alt(r)
    r1 = r1 / torch.linalg.norm(r1, dim=-1, keepdim=True)
    R = oracle.rotor_to_matrix(r1)
    err = (R.transpose(-1, -2) @ R - torch.eye(4, dtype=torch.float64)).abs().amax(dim=(-1, -2))
    assert err.max() > 0.1


@pytest.mark.parametrize("plane", range(6))
def test_single_bivector_rotor_is_plane_rotation(plane):
    """r = cos(th) + sin(th) e_ij rotates the (i, j) plane by 2 th: e_i -> cos 2th e_i - sin 2th e_j."""
    pairs = [(0, 1), (0, 2), (1, 2), (0, 3), (1, 3), (2, 3)]  # storage slots 1..6
    i, j = pairs[plane]
    th = 0.3
    r = torch.zeros(8, dtype=torch.float64)
    r[0] = math.cos(th)
    r[1 + plane] = math.sin(th)
    R = oracle.rotor_to_matrix(oracle.rotor_normalize(r)).numpy()
    E = np.eye(4)
    c, s = math.cos(2 * th), math.sin(2 * th)
    E[i, i] = c
    E[j, j] = c
    E[j, i] = -s
    E[i, j] = s
    np.testing.assert_allclose(R, E, atol=1e-14)


def quat_matrix(w, x, y, z):
    """Textbook rotation matrix of the unit quaternion w + x i + y j + z k."""
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


def test_spatial_rotor_reduces_to_quaternion():
    """b03 = b13 = b23 = p = 0 (Sec. 3.2.1): R = diag(R3, 1) with R3 the
    quaternion rotation of (w, x, y, z) = (s, -b12, b02, -b01)."""
    rng = np.random.default_rng(6)
    for _ in range(50):
        r = np.zeros(8)
        r[:4] = rng.normal(0, 1, 4)
        rn = oracle.rotor_normalize(torch.as_tensor(r)).numpy()
        R = oracle.rotor_to_matrix(torch.as_tensor(rn)).numpy()
        s, b01, b02, b12 = rn[:4]
        Q = quat_matrix(s, -b12, b02, -b01)
        np.testing.assert_allclose(R[:3, :3], Q, atol=1e-14)
        np.testing.assert_allclose(R[3], [0, 0, 0, 1], atol=1e-15)
        np.testing.assert_allclose(R[:, 3], [0, 0, 0, 1], atol=1e-15)


def test_golden_rotor_cases():
    """tests/golden/rotor_cases.txt: rotors with closed-form matrices (plane
    rotations by 2 theta and their compositions); see the file header."""
    path = os.path.join(GOLDEN, "rotor_cases.txt")
    rows = [ln for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) >= 4
    for ln in rows:
        v = np.array([float(x) for x in ln.split()])
        r, Rexp = v[:8], v[8:].reshape(4, 4)
        R = oracle.rotor_to_matrix(oracle.rotor_normalize(torch.as_tensor(r))).numpy()
        np.testing.assert_allclose(R, Rexp, atol=1e-12)
