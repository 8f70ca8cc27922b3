"""The learned gamma warm start: features, network, loss gradients, Adam (oracle).

Test infrastructure only; see the package docstring.

The paper has no learned part; the network is this project's warm start for the
occupation optimisation of Sec. 2 ("Occupancy Optimization with RI").  It maps
features of one pairing subspace g to the converged angles of that subspace.

Features of subspace g (strong orbital s, weak orbitals w_0..w_{N_g-1} in rank
order), with n0 the standard-guess occupations (strong 0.98, weak 0.02 / N_g)
and mf_p = sum_{q outside g} n0_q (2 J_pq - K_pq) the mean field of the other
subspaces on orbital p:
  [H_ss, J_ss, mf_s,  then per weak w: H_ww, J_ww, K_sw, mf_w]   (3 + 4 N_g values).
Targets: the N_g angles of the subspace (strong angle, then the N_g - 1 weak
angles) folded into [0, pi/2] (the occupations depend on cos^2 and sin^2 only).

Network: z-scored features -> 64 tanh -> 64 tanh -> N_g, weights stored as BF16
values (this module rounds them to nearest-even BF16), biases FP32; loss = mean
squared error over the batch and outputs; Adam (beta1 0.9, beta2 0.999,
eps 1e-8) with decoupled weight decay on the weight matrices.  Everything
here is FP64 arithmetic on those values.
"""
from __future__ import annotations

import numpy as np


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round FP32 values to the nearest BF16 value (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return (r.astype(np.uint32)).view(np.float32).astype(np.float64)


def subspace_features(J, K, Hd, subspace, weak_rank, n_strong, n_weak_per):
    """Feature rows [N_I, 3 + 4 N_g] (definition in the module docstring)."""
    n0 = np.where(np.asarray(weak_rank) < 0, 0.98, 0.02 / n_weak_per)
    X = np.zeros((n_strong, 3 + 4 * n_weak_per))
    for g in range(n_strong):
        members = [int(np.where((subspace == g) & (weak_rank == r))[0][0]) for r in range(-1, n_weak_per)]
        outside = np.asarray(subspace) != g
        s = members[0]
        mf = [float(np.sum(n0[outside] * (2.0 * J[p, outside] - K[p, outside]))) for p in members]
        X[g, 0:3] = [Hd[s], J[s, s], mf[0]]
        for i, w in enumerate(members[1:]):
            X[g, 3 + 4 * i: 7 + 4 * i] = [Hd[w], J[w, w], K[s, w], mf[i + 1]]
    return X


def fold_angles(gamma, n_strong, n_weak_per):
    """Converged angles -> targets [N_I, N_g] in [0, pi/2]."""
    a = np.arccos(np.minimum(1.0, np.abs(np.cos(np.asarray(gamma, dtype=np.float64)))))
    Y = np.zeros((n_strong, n_weak_per))
    Y[:, 0] = a[:n_strong]
    Y[:, 1:] = a[n_strong:].reshape(n_strong, n_weak_per - 1)
    return Y


def unfold_angles(Y, clip=0.0):
    """Network outputs [N_I, N_g] -> gamma (N_I strong angles, then the weak ones),
    clipped to [clip, pi/2 - clip]."""
    Y = np.clip(np.asarray(Y, dtype=np.float64), clip, np.pi / 2 - clip)
    return np.concatenate([Y[:, 0], Y[:, 1:].reshape(-1)])


def param_shapes(n_in, n_hidden, n_out):
    return [(n_hidden, n_in), (n_hidden,), (n_hidden, n_hidden), (n_hidden,), (n_out, n_hidden), (n_out,)]


def unpack(flat, n_in, n_hidden, n_out):
    out, o = [], 0
    for sh in param_shapes(n_in, n_hidden, n_out):
        k = int(np.prod(sh))
        out.append(np.asarray(flat[o:o + k], dtype=np.float64).reshape(sh))
        o += k
    return out


def forward(P, X, mean, inv_std, round_weights=True):
    """Activations (Z, A1, A2, Y) for feature rows X; P = [W1, b1, W2, b2, W3, b3]."""
    W1, b1, W2, b2, W3, b3 = P
    if round_weights:
        W1, W2, W3 = bf16_round(W1), bf16_round(W2), bf16_round(W3)
    Z = (np.asarray(X, dtype=np.float64) - mean) * inv_std
    A1 = np.tanh(Z @ W1.T + b1)
    A2 = np.tanh(A1 @ W2.T + b2)
    Y = A2 @ W3.T + b3
    return Z, A1, A2, Y


def loss_and_grads(P, X, T, mean, inv_std, round_weights=True):
    """MSE loss and its gradients with respect to [W1, b1, W2, b2, W3, b3]
    (through the BF16 weight values when round_weights)."""
    W1, b1, W2, b2, W3, b3 = P
    if round_weights:
        W1, W2, W3 = bf16_round(W1), bf16_round(W2), bf16_round(W3)
    Z, A1, A2, Y = forward([W1, b1, W2, b2, W3, b3], X, mean, inv_std, round_weights=False)
    D = Y - T
    loss = float(np.mean(D * D))
    dY = 2.0 * D / D.size
    gW3 = dY.T @ A2
    gb3 = dY.sum(axis=0)
    dZ2 = (dY @ W3) * (1.0 - A2 * A2)
    gW2 = dZ2.T @ A1
    gb2 = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ W2) * (1.0 - A1 * A1)
    gW1 = dZ1.T @ Z
    gb1 = dZ1.sum(axis=0)
    return loss, [gW1, gb1, gW2, gb2, gW3, gb3]


def adam_step(P, G, M, V, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=1e-4):
    """One Adam update (step counts from 1); weight decay lr * wd * W on the matrices only."""
    newP, newM, newV = [], [], []
    for i, (p, g, m, v) in enumerate(zip(P, G, M, V)):
        m = beta1 * m + (1.0 - beta1) * g
        v = beta2 * v + (1.0 - beta2) * g * g
        mh = m / (1.0 - beta1 ** step)
        vh = v / (1.0 - beta2 ** step)
        upd = lr * mh / (np.sqrt(vh) + eps)
        if i % 2 == 0:
            upd = upd + lr * weight_decay * p
        newP.append(p - upd)
        newM.append(m)
        newV.append(v)
    return newP, newM, newV
