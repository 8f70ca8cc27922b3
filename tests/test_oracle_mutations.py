"""Plausible mistakes planted in the oracle (on the CPU) are caught by its pins.

Each case swaps one oracle function for a subtly wrong variant (a dropped
term, a wrong sign, a transposed operand) and checks that the corresponding
pin from the other test files fails.
"""
import numpy as np
import pytest

from oracle import brute, integrals as I, pnof7, rhf, ri
from synthetic.systems import pairing_columns
from tests.workloads import make_workload


@pytest.fixture(scope="module")
def sq():
    w = make_workload("square4")
    B, L, G = ri.setup(w.system)
    return w, B


def test_transposed_half_transform_fails_brute_force(sq):
    w, B = sq
    m = w.system.n_omega
    C = w.C
    good = ri.all_rows(B, C, m)["K"]
    # C used untransposed: rows of C taken as orbitals
    bad_bh = np.einsum("pm,Pmn->Ppn", C[:m, :], B)
    bad = ri.jk_mo(ri.full_transform(bad_bh, C.T), ri.diagonal(bad_bh, C.T))[1]
    eri = brute.fitted_eri4(B)
    ref = brute.conventional_jk(eri, C, m)[1]
    assert np.allclose(good, ref, atol=1e-12)
    assert not np.allclose(bad, ref, atol=1e-6)


def test_exchange_with_wrong_orbital_fails_tie_to_mo_exchange(sq):
    w, B = sq
    m = w.system.n_omega
    r = ri.all_rows(B, w.C, m)
    bh = r["bh"]
    # K^(q) built from the next orbital's slice (an off-by-one in q)
    bad_k = np.einsum("Pqm,Pqn->qmn", np.roll(bh, 1, axis=1), np.roll(bh, 1, axis=1))
    C = w.C[:, :m]
    good = np.einsum("mp,qmn,np->pq", C, r["Kao"], C)
    bad = np.einsum("mp,qmn,np->pq", C, bad_k, C)
    assert np.allclose(good, r["K"], atol=1e-12)
    assert not np.allclose(bad, r["K"], atol=1e-6)


def test_wrong_cross_coefficient_fails_closed_shell_pin(sq, monkeypatch):
    w, B = sq
    s = w.system
    H = I.core_hamiltonian(s)
    e_nuc = I.nuclear_repulsion(s)
    sub, rank = pairing_columns(s.n_strong, s.n_weak_per)
    gam = w.gamma.copy()
    gam[: s.n_strong] = 0.0
    m = s.n_omega
    n = pnof7.occupations(gam, s.n_strong, s.n_weak_per, sub, rank)
    r = ri.all_rows(B, w.C, m)
    Hd = np.einsum("mp,mn,np->p", w.C[:, :m], H, w.C[:, :m])
    A, Bc = pnof7.coupling(n, sub, rank)
    e_rhf = rhf.closed_shell_energy(B, H, w.C[:, : s.n_strong], e_nuc)
    assert abs(pnof7.energy(n, Hd, r["J"], r["K"], A, Bc, e_nuc) - e_rhf) < 1e-10
    A_bad = np.where(np.equal.outer(sub, sub), A, 0.5 * A)   # drop the factor 2 of 2 J_pq across pairs
    assert abs(pnof7.energy(n, Hd, r["J"], r["K"], A_bad, Bc, e_nuc) - e_rhf) > 1e-3


def test_wrong_weak_weak_sign_fails_two_electron_pin():
    w = make_workload("square4")
    B, L, G = ri.setup(w.system)
    H = I.core_hamiltonian(w.system)
    ng = 5
    sub, rank = pairing_columns(1, ng)
    n = pnof7.occupations(np.array([0.4, 0.3, 0.9, 0.2, 1.2]), 1, ng, sub, rank)
    m = 1 + ng
    C = w.C[:, :m]
    r = ri.all_rows(B, w.C, m)
    Hd = np.einsum("mp,mn,np->p", C, H, C)
    D, Pi = pnof7.delta_pi(n, sub, rank)
    weak = rank >= 0
    Pi_bad = Pi.copy()
    Pi_bad[np.ix_(weak, weak)] *= np.where(np.eye(weak.sum()) > 0, 1.0, -1.0)
    mo = brute.mo_eri4(brute.fitted_eri4(B), C)
    c = np.where(rank < 0, 1.0, -1.0) * np.sqrt(n)
    e_wf = 2.0 * np.sum(c * c * Hd) + np.einsum("p,q,pqpq->", c, c, mo)
    good = pnof7.energy_eq_pnof(n, Hd, r["J"], r["K"], D, Pi, 0.0)
    bad = pnof7.energy_eq_pnof(n, Hd, r["J"], r["K"], D, Pi_bad, 0.0)
    assert abs(good - e_wf) < 1e-12
    assert abs(bad - e_wf) > 1e-6


def test_dropped_kinetic_term_fails_textbook_pin():
    # T without the -2 mu R^2 term disagrees with the S&O value T12 = 0.2365.
    from tests.test_oracle_integrals import _toy_system
    al = np.array([0.109818, 0.405771, 2.22766]) * 1.24 ** 2
    d = np.array([0.444635, 0.535328, 0.154329])
    s = _toy_system([[0, 0, 0], [0, 0, 1.4]], [1, 1], [0, 0, 0, 1, 1, 1], np.concatenate([al, al]))
    p, mu, r2, kab, P, nn = I._pair_data(s)
    bad = nn * mu * 3.0 * (np.pi / p) ** 1.5 * kab
    D = np.zeros((6, 2)); D[:3, 0] = d; D[3:, 1] = d
    assert abs((D.T @ I.kinetic(s) @ D)[0, 1] - 0.2365) < 1e-4
    assert abs((D.T @ bad @ D)[0, 1] - 0.2365) > 1e-2


def test_wrong_sign_weak_weak_gradient_fails_finite_differences(monkeypatch):
    from oracle import onopt
    rng = np.random.default_rng(21)
    sub, rank = pairing_columns(2, 3)
    m = 8
    X = rng.standard_normal((m, m))
    J = X @ X.T / m + np.eye(m)
    K = 0.3 * J
    np.fill_diagonal(K, np.diag(J))
    H = rng.standard_normal(m)
    gamma = rng.uniform(0.2, 1.3, 6)

    def fd_ok():
        E0, g = onopt.energy_and_gradient(gamma, 2, 3, sub, rank, H, J, K, 0.0)
        h = 1e-6
        for k in range(gamma.shape[0]):
            e = np.zeros_like(gamma)
            e[k] = h
            Ep, _ = onopt.energy_and_gradient(gamma + e, 2, 3, sub, rank, H, J, K, 0.0)
            Em, _ = onopt.energy_and_gradient(gamma - e, 2, 3, sub, rank, H, J, K, 0.0)
            if abs((Ep - Em) / (2 * h) - g[k]) > 1e-7 * max(1.0, abs(g[k])):
                return False
        return True

    assert fd_ok()
    good = onopt.energy_dn

    def bad(n, Hd, J_, K_, sub_, rank_):
        # the within-subspace sign taken as +1 for weak-weak pairs too
        g = good(n, Hd, J_, K_, sub_, rank_)
        for p in range(n.shape[0]):
            for q in range(n.shape[0]):
                if q != p and sub_[q] == sub_[p] and rank_[p] >= 0 and rank_[q] >= 0:
                    g[p] -= 2.0 * K_[p, q] * np.sqrt(n[q] / n[p])
        return g
    monkeypatch.setattr(onopt, "energy_dn", bad)
    assert not fd_ok()


def _flambda_fixture():
    from oracle import orbopt
    w = make_workload("square4")
    s = w.system
    B, L, G = ri.setup(s)
    H = I.core_hamiltonian(s)
    sub, rank = pairing_columns(s.n_strong, s.n_weak_per)
    return orbopt, w, s, B, H, I.nuclear_repulsion(s), sub, rank


def test_reversed_flambda_off_diagonal_fails_descent_pin(monkeypatch):
    """F_qp = lambda_pq - lambda_qp (the gradient's sign flipped): the step that the
    descent pin of test_oracle_orbopt requires to lower E raises it instead."""
    orbopt, w, s, B, H, enuc, sub, rank = _flambda_fixture()
    nb = s.nbf
    E0, lam = orbopt.energy_lambda(s, B, H, enuc, w.C, w.gamma, sub, rank)
    D = np.arange(nb, dtype=np.float64)
    bound = 1e-5 * np.abs(lam - lam.T).max()
    good = orbopt.flambda_matrix
    monkeypatch.setattr(orbopt, "flambda_matrix", lambda lam_, diag, b: good(lam_.T, diag, b))
    C1, _ = orbopt.flambda_step(w.C, lam, D, bound)
    U = w.C.T @ C1
    U = U * np.sign(np.diag(U))[None, :]
    E1, _ = orbopt.energy_lambda(s, B, H, enuc, w.C @ U, w.gamma, sub, rank)
    assert E1 > E0


def test_descending_eigenvector_order_fails_stationary_pin(monkeypatch):
    """Eigenvectors taken in decreasing order of eigenvalue (aufbau reversed): at a
    stationary point the step no longer keeps the orbitals."""
    orbopt, w, s, B, H, enuc, sub, rank = _flambda_fixture()
    nb = s.nbf
    rng = np.random.default_rng(4)
    S = rng.standard_normal((nb, nb))
    lam = S + S.T
    D = np.sort(rng.uniform(-3.0, 3.0, nb))

    def reversed_step(C, lam_, diag, bound):
        eps, U = np.linalg.eigh(orbopt.flambda_matrix(lam_, diag, bound))
        return C @ U[:, ::-1], eps[::-1]

    monkeypatch.setattr(orbopt, "flambda_step", reversed_step)
    C1, eps = orbopt.flambda_step(w.C, lam, D, bound=0.1)
    assert not np.allclose(np.abs(C1.T @ w.C), np.eye(nb), atol=1e-6)
    assert not np.allclose(eps, D, atol=1e-6)


def test_full_weight_exchange_fails_printed_h2_scf():
    """F = H + J - K (the exchange's 1/2 dropped, a plausible slip): the SCF no
    longer reproduces the printed minimal-basis H2 energies."""
    import json
    import os
    from tests.test_oracle_rhf import GOLDEN, _h2_sto3g
    g = json.load(open(os.path.join(GOLDEN, "sto3g_h2_scf.json")))
    S, H, eri, enuc = _h2_sto3g()
    good = rhf.jk_exact(eri)

    def bad(D):
        Jd, Kd = good(D)
        return Jd, 2.0 * Kd

    r = rhf.scf(H, S, bad, 1, enuc)
    assert abs(r["E"] - g["E_total"]) > 10 * g["tolerance"] or abs(r["eps"][0] - g["eps1"]) > 10 * g["tolerance"]
