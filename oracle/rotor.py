"""4D rotor normalisation and rotor -> rotation matrix (paper appendix A.1, A.2).

Storage order of the 8 rotor components (main text, Eq. 4 of Sec. 3.2.1):
    (s, b01, b02, b12, b03, b13, b23, p)
for r = s + b01 e01 + b02 e02 + b12 e12 + b03 e03 + b13 e13 + b23 e23 + p e0123,
axes e0..e3 = x, y, z, t. The appendix lists the components in another order;
the arithmetic below uses the named components, so the order only matters for
storage.
"""
from __future__ import annotations

import torch

_S, _B01, _B02, _B12, _B03, _B13, _B23, _P = range(8)


def _parts(r: torch.Tensor):
    return (r[..., _S], r[..., _B01], r[..., _B02], r[..., _B12],
            r[..., _B03], r[..., _B13], r[..., _B23], r[..., _P])


def rotor_epsilon(r: torch.Tensor) -> torch.Tensor:
    """epsilon = p s - b01 b23 + b02 b13 - b03 b12: the e0123 part of r r^dagger
    divided by two (appendix A.1, the two normalisation conditions). The summary
    at the end of A.1 prints the last two signs flipped; that form does not make
    the A.2 matrix orthogonal, this one does (checked by the tests)."""
    s, b01, b02, b12, b03, b13, b23, p = _parts(r)
    return p * s - b01 * b23 + b02 * b13 - b03 * b12


def rotor_epsilon_grad(r: torch.Tensor) -> torch.Tensor:
    """Gradient of epsilon w.r.t. the 8 components (appendix A.1), in storage order."""
    s, b01, b02, b12, b03, b13, b23, p = _parts(r)
    return torch.stack([p, -b23, b13, -b03, -b12, b02, -b01, s], dim=-1)


def rotor_normalize(r: torch.Tensor) -> torch.Tensor:
    """F_norm of appendix A.1, in the paper's order of steps:

    1. epsilon = f(r), l^2 = sum of squares of the 8 components;
    2. one exact root step of f along its gradient: r := r + delta grad(epsilon),
       with delta the root of (1 + delta^2) epsilon + l^2 delta = 0 that tends
       to 0 with epsilon, i.e. (-l^2 + sqrt(l^4 - 4 epsilon^2)) / (2 epsilon);
       it is evaluated in the algebraically equal form
       -2 epsilon / (l^2 + sqrt(l^4 - 4 epsilon^2)), which is finite at
       epsilon = 0 (delta = 0 there);
    3. divide by the norm of the updated rotor.

    A rotor whose updated norm vanishes (e.g. the zero rotor, or s = p with all
    other components 0, where l^4 = 4 epsilon^2) maps to the identity rotor.
    """
    eps = rotor_epsilon(r)
    l2 = (r * r).sum(-1)
    disc = torch.clamp(l2 * l2 - 4.0 * eps * eps, min=0.0)
    delta = -2.0 * eps / torch.where(l2 > 0, l2 + torch.sqrt(disc), torch.ones_like(l2))
    r1 = r + delta[..., None] * rotor_epsilon_grad(r)
    n2 = (r1 * r1).sum(-1)
    ok = n2 > 1e-20
    safe = torch.where(ok, n2, torch.ones_like(n2))
    rn = r1 / torch.sqrt(safe)[..., None]
    ident = torch.zeros_like(r)
    ident[..., _S] = 1.0
    return torch.where(ok[..., None], rn, ident)


def rotor_to_matrix(r: torch.Tensor) -> torch.Tensor:
    """F_map of appendix A.2: the 4x4 matrix R with R u = r u r^dagger for a
    normalised rotor, entry by entry as the appendix gives them (R^{ij} is row
    i, column j; R acts on column vectors)."""
    s, b01, b02, b12, b03, b13, b23, p = _parts(r)
    sq = lambda a: a * a  # noqa: E731
    r00 = -sq(b01) - sq(b02) - sq(b03) + sq(b12) + sq(b13) + sq(b23) - sq(p) + sq(s)
    r01 = 2 * (b01 * s - b02 * b12 - b03 * b13 + b23 * p)
    r02 = 2 * (b01 * b12 + b02 * s - b03 * b23 - b13 * p)
    r03 = 2 * (b01 * b13 + b02 * b23 + b03 * s + b12 * p)
    r10 = 2 * (-b01 * s - b02 * b12 - b03 * b13 - b23 * p)
    r11 = -sq(b01) + sq(b02) + sq(b03) - sq(b12) - sq(b13) + sq(b23) - sq(p) + sq(s)
    r12 = 2 * (-b01 * b02 + b03 * p + b12 * s - b13 * b23)
    r13 = 2 * (-b01 * b03 - b02 * p + b12 * b23 + b13 * s)
    r20 = 2 * (b01 * b12 - b02 * s - b03 * b23 + b13 * p)
    r21 = 2 * (-b01 * b02 - b03 * p - b12 * s - b13 * b23)
    r22 = sq(b01) - sq(b02) + sq(b03) - sq(b12) + sq(b13) - sq(b23) - sq(p) + sq(s)
    r23 = 2 * (b01 * p - b02 * b03 - b12 * b13 + b23 * s)
    r30 = 2 * (b01 * b13 + b02 * b23 - b03 * s - b12 * p)
    r31 = 2 * (-b01 * b03 + b02 * p + b12 * b23 - b13 * s)
    r32 = 2 * (-b01 * p - b02 * b03 - b12 * b13 - b23 * s)
    r33 = sq(b01) + sq(b02) - sq(b03) + sq(b12) - sq(b13) - sq(b23) - sq(p) + sq(s)
    rows = [
        torch.stack([r00, r01, r02, r03], -1),
        torch.stack([r10, r11, r12, r13], -1),
        torch.stack([r20, r21, r22, r23], -1),
        torch.stack([r30, r31, r32, r33], -1),
    ]
    return torch.stack(rows, -2)
