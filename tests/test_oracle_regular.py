"""Pins of the oracle's regularisers (Sec. 3.3): the brute-force 4D KNN
against scipy's k-d tree; the entropy loss at closed-form points; the
consistency loss recomputed from speeds obtained independently by slicing
at two times (the sliced centre moves by (t - mu_t) V / W); the gradients
against central differences."""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import regular as oreg

scipy_spatial = pytest.importorskip("scipy.spatial")


def _scene(n=300, seed=8):
    g = synth.gaussians(n, seed, mean_lo=-2.0, mean_hi=2.0, ls_xyz=(-2.0, 0.4), ls_t=(-1.5, 0.4))
    return oracle.to_f64(g)


def test_knn_matches_a_kd_tree():
    sc = _scene()
    m = sc["mean"]
    sx, st = 4.0, 1.0
    idx, d2 = oreg.knn4d(m, sx, st, 8)
    q = np.concatenate([m[:, :3].numpy() / sx, m[:, 3:].numpy() / st], 1)
    dd, ii = scipy_spatial.cKDTree(q).query(q, k=9)
    assert np.array_equal(ii[:, 0], np.arange(len(q)))  # the point itself first
    assert np.array_equal(idx.numpy(), ii[:, 1:])
    assert np.allclose(d2.numpy(), dd[:, 1:] ** 2, rtol=1e-12, atol=0)


def test_knn_ties_go_to_the_smaller_index():
    m = torch.zeros((6, 4), dtype=torch.float64)
    m[:, 0] = torch.tensor([0.0, 1.0, -1.0, 2.0, -2.0, 3.0])
    idx, d2 = oreg.knn4d(m, 1.0, 1.0, 2)
    assert idx[0].tolist() == [1, 2]  # equal distance 1: index 1 before 2
    assert idx[3].tolist() == [1, 5]


def test_entropy_closed_form():
    sc = _scene(n=4)
    sc["logit"][:] = 0.0
    out = oreg.losses_and_grads(sc, torch.zeros((4, 1), dtype=torch.long), lam_e=1.0, lam_c=0.0)
    assert abs(float(out["entropy"]) - 0.5 * math.log(2.0)) < 1e-15
    g = -(math.log(0.5) + 1.0) * 0.25 / 4
    assert torch.allclose(out["grad_logit"], torch.full((4,), g, dtype=torch.float64), atol=1e-16)


def test_consistency_from_sliced_speeds():
    sc = _scene(n=120, seed=9)
    idx, _ = oreg.knn4d(sc["mean"], 4.0, 1.0, 8)
    R = oracle.rotor_to_matrix(oracle.rotor_normalize(sc["rotor"]))
    s4 = oracle.covariance4(R, torch.exp(sc["logscale"]))
    mu0 = oracle.slice_at(sc["mean"], s4, 0.2)[0]
    mu1 = oracle.slice_at(sc["mean"], s4, 0.7)[0]
    v = ((mu1 - mu0) / 0.5).numpy()
    r = v - v[idx.numpy()].mean(1)
    want = np.abs(r).sum(1).mean()
    got = float(oreg.consistency(sc, idx))
    assert abs(got - want) < 1e-9 * max(1.0, abs(want))
    static = dict(sc)
    static["rotor"] = sc["rotor"].clone()
    static["rotor"][:, 4:] = 0.0  # no space-time coupling: every speed is zero
    assert float(oreg.consistency(static, idx)) < 1e-12


def test_gradients_against_central_differences():
    sc = _scene(n=40, seed=10)
    idx, _ = oreg.knn4d(sc["mean"], 4.0, 1.0, 4)
    out = oreg.losses_and_grads(sc, idx, 0.7, 1.3)

    def f(s):
        return float(0.7 * oreg.entropy(s) + 1.3 * oreg.consistency(s, idx))

    rng = np.random.default_rng(0)
    for name in ("rotor", "logscale", "logit"):
        flat = sc[name].reshape(-1)
        for k in rng.choice(flat.numel(), 6, replace=False):
            h = 1e-6 * max(1.0, abs(float(flat[k])))
            sp = {a: b.clone() for a, b in sc.items()}
            sm = {a: b.clone() for a, b in sc.items()}
            sp[name].reshape(-1)[k] += h
            sm[name].reshape(-1)[k] -= h
            fd = (f(sp) - f(sm)) / (2 * h)
            an = float(out["grad_" + name].reshape(-1)[k])
            assert abs(fd - an) <= 1e-5 * (abs(an) + 1e-3), (name, k, fd, an)
