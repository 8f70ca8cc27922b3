"""Pins of the orbital-rotation oracle (oracle/orbopt.py).

* a small rotation step lowers E by the first-order amount predicted from the
  rotation gradient dE/dkappa_qp = 4 (lambda_qp - lambda_pq), itself pinned by
  finite differences in test_oracle_pnof7 (a wrong sign or scale of the step
  fails this);
* the rotated orbitals stay orthonormal in the overlap metric (C^T S C = I);
* the trust-radius driver never raises E.
"""
import numpy as np
import pytest

from oracle import integrals as I, orbopt, ri
from synthetic import pairing_columns
from tests.workloads import make_workload


@pytest.fixture(scope="module")
def sq():
    w = make_workload("square4")
    s = w.system
    B, L, G = ri.setup(s)
    H = I.core_hamiltonian(s)
    sub, rank = pairing_columns(s.n_strong, s.n_weak_per)
    return w, B, H, I.nuclear_repulsion(s), sub, rank


def test_small_step_lowers_energy_by_the_first_order_amount(sq):
    w, B, H, enuc, sub, rank = sq
    s = w.system
    E0, lam = orbopt.energy_lambda(s, B, H, enuc, w.C, w.gamma, sub, rank)
    G = lam - lam.T
    gmax = np.abs(G).max()
    r = 1e-4
    C1 = orbopt.rotation_step(w.C, lam, r)
    E1, _ = orbopt.energy_lambda(s, B, H, enuc, C1, w.gamma, sub, rank)
    iu = np.triu_indices(s.nbf, 1)
    predicted = -4.0 * r / gmax * np.sum(G[iu] ** 2)
    assert E1 < E0
    assert abs((E1 - E0) - predicted) <= 1e-2 * abs(predicted)
    S = I.overlap(s)
    assert np.abs(C1.T @ S @ C1 - np.eye(s.nbf)).max() < 1e-13


def test_driver_never_raises_energy(sq):
    w, B, H, enuc, sub, rank = sq
    s = w.system
    E0, lam = orbopt.energy_lambda(s, B, H, enuc, w.C, w.gamma, sub, rank)
    C, E, gmax, it = orbopt.optimize(s, w.C, w.gamma, sub, rank, max_iter=15)
    assert E < E0
    g0 = np.abs(lam - lam.T).max()
    assert gmax < g0


def test_flambda_step_is_the_identity_at_a_stationary_point(sq):
    """lambda symmetric (a stationary point): F^lambda is diagonal, and with an
    ascending diagonal the step keeps every orbital (up to its sign)."""
    w, B, H, enuc, sub, rank = sq
    nb = w.system.nbf
    rng = np.random.default_rng(4)
    X = rng.standard_normal((nb, nb))
    lam = X + X.T
    D = np.sort(rng.uniform(-3.0, 3.0, nb))
    C1, eps = orbopt.flambda_step(w.C, lam, D, bound=0.1)
    # the rotation in orbital space is C^T S C1 (orbitals orthonormal in the overlap metric)
    np.testing.assert_allclose(np.abs(C1.T @ I.overlap(w.system) @ w.C), np.eye(nb), atol=1e-12)
    np.testing.assert_allclose(eps, D, atol=1e-12)


def test_flambda_step_descends_by_the_first_order_amount(sq):
    """With small off-diagonal elements and an ascending diagonal the eigenvectors are
    U = I + kappa with kappa_qp = F_qp / (D_pp - D_qq), so E changes by
    4 sum_{q>p} (lambda_qp - lambda_pq) U_qp to first order, and the change is a
    descent (a reversed F^lambda off-diagonal would climb)."""
    w, B, H, enuc, sub, rank = sq
    s = w.system
    nb = s.nbf
    E0, lam = orbopt.energy_lambda(s, B, H, enuc, w.C, w.gamma, sub, rank)
    G = lam - lam.T
    D = np.arange(nb, dtype=np.float64)          # ascending, unit gaps
    bound = 1e-5 * np.abs(G).max()
    C1, eps = orbopt.flambda_step(w.C, lam, D, bound)
    U = w.C.T @ I.overlap(s) @ C1
    U = U * np.sign(np.diag(U))[None, :]         # eigenvector signs as near the identity
    E1, _ = orbopt.energy_lambda(s, B, H, enuc, w.C @ U, w.gamma, sub, rank)
    il = np.tril_indices(nb, -1)
    predicted = 4.0 * np.sum(G[il] * U[il])
    assert predicted < 0.0 and E1 < E0
    assert abs((E1 - E0) - predicted) <= 2e-2 * abs(predicted)
    np.testing.assert_allclose(U.T @ U, np.eye(nb), atol=1e-12)
