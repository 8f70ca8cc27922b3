"""Pins of the orbital-rotation oracle (oracle/orbopt.py).

* a small rotation step lowers E by the first-order amount predicted from the
  rotation gradient dE/dkappa_qp = 4 (lambda_qp - lambda_pq), itself pinned by
  finite differences in test_oracle_pnof7 (a wrong sign or scale of the step
  fails this);
* the rotated orbitals stay orthonormal;
* the trust-radius driver never raises E.
"""
import numpy as np
import pytest

from oracle import integrals as I, orbopt, ri
from synthetic import make_workload, pairing_columns


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
    assert np.abs(C1.T @ C1 - np.eye(s.nbf)).max() < 1e-13


def test_driver_never_raises_energy(sq):
    w, B, H, enuc, sub, rank = sq
    s = w.system
    E0, lam = orbopt.energy_lambda(s, B, H, enuc, w.C, w.gamma, sub, rank)
    C, E, gmax, it = orbopt.optimize(s, w.C, w.gamma, sub, rank, max_iter=15)
    assert E < E0
    g0 = np.abs(lam - lam.T).max()
    assert gmax < g0
