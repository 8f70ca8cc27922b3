"""Pins of the learned-guess oracle (oracle/mlp.py).

* BF16 rounding against PyTorch's own float32 -> bfloat16 conversion (a library
  routine) and the ties-to-even cases written out;
* loss gradients against central finite differences of the loss;
* Adam's first step against its closed form (m_hat = g, v_hat = g^2);
* the features against their definition evaluated by hand on a 2-subspace case;
* folding the converged angles loses nothing the occupations depend on.
"""
import numpy as np
import pytest
import torch

from oracle import mlp, pnof7
from synthetic import pairing_columns


def test_bf16_round_matches_torch_and_ties_to_even():
    rng = np.random.default_rng(1)
    x = (rng.standard_normal(10000) * np.exp(rng.uniform(-20, 20, 10000))).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16_round(x), ref)
    assert mlp.bf16_round(np.float32(1.0 + 2.0 ** -8)) == 1.0              # tie -> even (down)
    assert mlp.bf16_round(np.float32(1.0 + 3 * 2.0 ** -8)) == 1.0 + 2.0 ** -6  # tie -> even (up)


def _params(rng, F=7, H=5, O=3):
    return [rng.standard_normal(sh) * 0.5 for sh in mlp.param_shapes(F, H, O)]


def test_loss_gradients_match_finite_differences():
    rng = np.random.default_rng(2)
    F, H, O = 7, 5, 3
    P = _params(rng, F, H, O)
    X = rng.standard_normal((11, F))
    T = rng.standard_normal((11, O))
    mean, inv = rng.standard_normal(F), rng.uniform(0.5, 2.0, F)
    loss, G = mlp.loss_and_grads(P, X, T, mean, inv, round_weights=False)
    h = 1e-6
    for i, p in enumerate(P):
        for idx in np.ndindex(p.shape):
            Pp = [q.copy() for q in P]
            Pm = [q.copy() for q in P]
            Pp[i][idx] += h
            Pm[i][idx] -= h
            lp, _ = mlp.loss_and_grads(Pp, X, T, mean, inv, round_weights=False)
            lm, _ = mlp.loss_and_grads(Pm, X, T, mean, inv, round_weights=False)
            assert abs((lp - lm) / (2 * h) - G[i][idx]) < 1e-8


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(3)
    P = _params(rng)
    G = [rng.standard_normal(p.shape) for p in P]
    Z = [np.zeros_like(p) for p in P]
    lr, wd = 1e-2, 1e-3
    P1, M1, V1 = mlp.adam_step(P, G, Z, Z, 1, lr, weight_decay=wd)
    for i, (p, g, p1) in enumerate(zip(P, G, P1)):
        expect = p - lr * g / (np.abs(g) + 1e-8) - (lr * wd * p if i % 2 == 0 else 0.0)
        assert np.allclose(p1, expect, rtol=0, atol=1e-15)


def test_features_by_hand():
    sub, rank = pairing_columns(2, 2)  # columns: 0, 1 strong; weak of g=1 at 2, 4; of g=0 at 3, 5
    m = 6
    J = np.arange(m * m, dtype=float).reshape(m, m)
    J = J + J.T
    K = 0.5 * J + np.eye(m)
    Hd = np.arange(m, dtype=float) * 10
    X = mlp.subspace_features(J, K, Hd, sub, rank, 2, 2)
    n0 = np.where(rank < 0, 0.98, 0.01)
    # subspace 0: strong 0, weak rank 0 at column 3, rank 1 at column 5; outside = {1, 2, 4}
    out = [1, 2, 4]
    mf0 = sum(n0[q] * (2 * J[0, q] - K[0, q]) for q in out)
    mf3 = sum(n0[q] * (2 * J[3, q] - K[3, q]) for q in out)
    assert np.allclose(X[0, :3], [0.0, J[0, 0], mf0])
    assert np.allclose(X[0, 3:7], [30.0, J[3, 3], K[0, 3], mf3])
    assert X[0, 7] == 50.0 and X[0, 9] == K[0, 5]


def test_fold_keeps_the_occupations():
    rng = np.random.default_rng(4)
    NI, Ng = 5, 4
    sub, rank = pairing_columns(NI, Ng)
    gamma = rng.uniform(-7.0, 7.0, NI * Ng)
    Y = mlp.fold_angles(gamma, NI, Ng)
    assert Y.min() >= 0.0 and Y.max() <= np.pi / 2
    n1 = pnof7.occupations(gamma, NI, Ng, sub, rank)
    n2 = pnof7.occupations(mlp.unfold_angles(Y), NI, Ng, sub, rank)
    assert np.allclose(n1, n2, atol=1e-14)
