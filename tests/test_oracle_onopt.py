"""Pins of the occupation-optimisation oracle (oracle/onopt.py).

* the analytic dE/dn and dE/dgamma against central finite differences of the
  energy (a route that does not use the derivative formulas);
* the occupation Jacobian conserves each subspace's sum (sum_p n_p = 1 per
  subspace, so its derivative vanishes);
* the optimiser's closed-form special case: with J = K = 0 the energy is linear
  in n, and its minimum puts each subspace's weak share on its lowest-H weak
  orbital and the strong orbital at n = 1 or 1/2 (the bounds of the map);
* a real case (square4): the optimiser ends at a stationary point below the
  standard guess.
"""
import numpy as np
import pytest

from oracle import integrals as I, onopt, pnof7, ri
from synthetic import pairing_columns
from tests.workloads import make_workload


def _random_problem(rng, n_strong=3, n_weak=3):
    sub, rank = pairing_columns(n_strong, n_weak)
    m = n_strong * (1 + n_weak)
    X = rng.standard_normal((m, m))
    J = X @ X.T / m + np.eye(m)
    Y = rng.standard_normal((m, m))
    K = 0.3 * (Y @ Y.T) / m
    np.fill_diagonal(K, np.diag(J))  # J_pp = K_pp
    H = rng.standard_normal(m)
    gamma = rng.uniform(0.1, 1.4, n_strong * n_weak)
    return sub, rank, m, J, K, H, gamma


def test_energy_dn_matches_finite_differences():
    rng = np.random.default_rng(11)
    sub, rank, m, J, K, H, gamma = _random_problem(rng)
    n = pnof7.occupations(gamma, 3, 3, sub, rank)

    def E(nv):
        A, Bc = pnof7.coupling(nv, sub, rank)
        return pnof7.energy(nv, H, J, K, A, Bc, 0.0)
    g = onopt.energy_dn(n, H, J, K, sub, rank)
    for p in range(m):
        # step relative to the distance from the bounds: the sqrt(n) terms curve
        # strongly for small occupations
        h = 1e-5 * min(n[p], 1.0 - n[p])
        e = np.zeros(m)
        e[p] = h
        fd = (E(n + e) - E(n - e)) / (2 * h)
        assert abs(fd - g[p]) <= 1e-7 * max(1.0, abs(g[p])), (p, fd, g[p])


def test_jacobian_conserves_subspace_sums_and_matches_fd():
    rng = np.random.default_rng(12)
    sub, rank, m, J, K, H, gamma = _random_problem(rng, 2, 4)
    D = onopt.occupations_jacobian(gamma, 2, 4, sub, rank)
    for g in range(2):
        assert np.abs(D[sub == g].sum(axis=0)).max() < 1e-14
    h = 1e-6
    for k in range(gamma.shape[0]):
        e = np.zeros_like(gamma)
        e[k] = h
        fd = (pnof7.occupations(gamma + e, 2, 4, sub, rank) - pnof7.occupations(gamma - e, 2, 4, sub, rank)) / (2 * h)
        assert np.abs(fd - D[:, k]).max() < 1e-9


def test_energy_gradient_matches_finite_differences():
    rng = np.random.default_rng(13)
    sub, rank, m, J, K, H, gamma = _random_problem(rng)
    E0, g = onopt.energy_and_gradient(gamma, 3, 3, sub, rank, H, J, K, 1.5)
    h = 1e-6
    for k in range(gamma.shape[0]):
        e = np.zeros_like(gamma)
        e[k] = h
        Ep, _ = onopt.energy_and_gradient(gamma + e, 3, 3, sub, rank, H, J, K, 1.5)
        Em, _ = onopt.energy_and_gradient(gamma - e, 3, 3, sub, rank, H, J, K, 1.5)
        assert abs((Ep - Em) / (2 * h) - g[k]) <= 1e-7 * max(1.0, abs(g[k]))


def test_standard_guess_occupations():
    sub, rank = pairing_columns(4, 3)
    g0 = onopt.standard_guess(4, 3)
    n = pnof7.occupations(g0, 4, 3, sub, rank)
    assert np.allclose(n[rank < 0], 0.98)
    assert np.allclose(n[rank >= 0], 0.02 / 3)


def test_optimizer_closed_form_without_two_electron_terms():
    rng = np.random.default_rng(14)
    n_strong, n_weak = 3, 3
    sub, rank = pairing_columns(n_strong, n_weak)
    m = n_strong * (1 + n_weak)
    H = rng.uniform(-2.0, 2.0, m)
    Z = np.zeros((m, m))
    g0 = onopt.standard_guess(n_strong, n_weak)
    gam, E, n, it, gmax = onopt.optimize(g0, n_strong, n_weak, sub, rank, H, Z, Z, 0.0, gtol=1e-10)
    expect = 0.0
    for g in range(n_strong):
        Hs = H[(sub == g) & (rank < 0)][0]
        Hw = H[(sub == g) & (rank >= 0)].min()
        expect += 2.0 * Hs if Hs < Hw else (Hs + Hw)
    assert E == pytest.approx(expect, abs=1e-8)


def test_optimizer_on_square4_reaches_a_stationary_point_below_the_guess():
    w = make_workload("square4")
    s = w.system
    B, L, G = ri.setup(s)
    m = s.n_omega
    rows = ri.all_rows(B, w.C, m)
    H = I.core_hamiltonian(s)
    Hd = np.einsum("mp,mn,np->p", w.C[:, :m], H, w.C[:, :m])
    sub, rank = pairing_columns(s.n_strong, s.n_weak_per)
    g0 = onopt.standard_guess(s.n_strong, s.n_weak_per)
    E0, _ = onopt.energy_and_gradient(g0, s.n_strong, s.n_weak_per, sub, rank, Hd, rows["J"], rows["K"],
                                      I.nuclear_repulsion(s))
    gam, E, n, it, gmax = onopt.optimize(g0, s.n_strong, s.n_weak_per, sub, rank, Hd, rows["J"], rows["K"],
                                         I.nuclear_repulsion(s))
    assert E < E0
    assert gmax < 1e-6
    for g in range(s.n_strong):
        assert n[sub == g].sum() == pytest.approx(1.0, abs=1e-14)
