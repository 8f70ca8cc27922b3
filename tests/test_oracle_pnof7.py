"""Pins of the oracle's PNOF7 occupations, energy and Lagrangian.

* occupation sum rules (Sec. 2: 2 sum n = N, 0 <= n <= 1; one electron pair
  per subspace) and the map's special cases;
* Eq. (PNOF) with explicit Delta/Pi == the symmetric A/B form;
* special case: all strong angles zero -> the closed-shell determinant energy
  computed from the AO density (a different route);
* special case: one electron pair -> the expectation value of the paired
  two-electron wavefunction sum_p c_p |p alpha p beta> (c = +sqrt(n) for the
  strong orbital, -sqrt(n) for weak ones), evaluated from the MO four-index
  tensor of the brute-force path;
* finite differences: dE/dC = 4 F^(p) C_p and dE/dkappa = 4 (lambda - lambda^T);
* E = E_nuc + sum_p (n_p H_pp + lambda_pp).
"""
import numpy as np
import pytest

from oracle import brute, integrals as I, pnof7, rhf, ri
from synthetic.systems import pairing_columns
from tests.workloads import make_workload


@pytest.fixture(scope="module")
def sq():
    w = make_workload("square4")
    s = w.system
    B, L, G = ri.setup(s)
    H = I.core_hamiltonian(s)
    e_nuc = I.nuclear_repulsion(s)
    sub, rank = pairing_columns(s.n_strong, s.n_weak_per)
    return w, B, H, e_nuc, sub, rank


def _energy(w, B, H, e_nuc, sub, rank, C=None, gamma=None):
    s = w.system
    C = w.C if C is None else C
    gamma = w.gamma if gamma is None else gamma
    m = s.n_omega
    n = pnof7.occupations(gamma, s.n_strong, s.n_weak_per, sub, rank)
    r = ri.all_rows(B, C, m)
    Hd = np.einsum("mp,mn,np->p", C[:, :m], H, C[:, :m])
    A, Bc = pnof7.coupling(n, sub, rank)
    return pnof7.energy(n, Hd, r["J"], r["K"], A, Bc, e_nuc), n, r, A, Bc


def test_pairing_map_is_a_bijection():
    for ni, ng in [(4, 2), (24, 4), (3, 1), (1, 5)]:
        sub, rank = pairing_columns(ni, ng)
        assert sub.shape == (ni * (1 + ng),)
        assert sorted(zip(sub.tolist(), rank.tolist())) == sorted(
            [(g, -1) for g in range(ni)] + [(g, i) for g in range(ni) for i in range(ng)])


def test_occupation_sum_rules():
    rng = np.random.default_rng(0)
    for ni, ng in [(4, 2), (24, 4), (3, 1), (2, 6)]:
        sub, rank = pairing_columns(ni, ng)
        gam = rng.uniform(-3, 3, size=ni * ng)
        n = pnof7.occupations(gam, ni, ng, sub, rank)
        assert (n >= 0).all() and (n <= 1).all()
        assert abs(2 * n.sum() - 2 * ni) < 1e-13
        for g in range(ni):
            assert abs(n[sub == g].sum() - 1.0) < 1e-14
            assert 0.5 <= n[g] <= 1.0


def test_occupation_special_cases():
    sub, rank = pairing_columns(2, 3)
    n = pnof7.occupations(np.zeros(6), 2, 3, sub, rank)
    np.testing.assert_allclose(n[:2], 1.0)
    np.testing.assert_allclose(n[2:], 0.0)
    # gamma_strong = pi/2 -> n_g = 1/2; weak angles 0 put the pair's other half in weak orbital 0.
    g = np.zeros(6)
    g[:2] = np.pi / 2
    n = pnof7.occupations(g, 2, 3, sub, rank)
    np.testing.assert_allclose(n[:2], 0.5)
    for gg in range(2):
        w = (sub == gg) & (rank == 0)
        np.testing.assert_allclose(n[w], 0.5)
    # N_g = 1: the single weak orbital holds h_g.
    sub, rank = pairing_columns(3, 1)
    gam = np.array([0.3, 0.7, 1.1])
    n = pnof7.occupations(gam, 3, 1, sub, rank)
    np.testing.assert_allclose(n[3:][::-1], 1.0 - 0.5 * (1.0 + np.cos(gam) ** 2))


def test_eq_pnof_form_equals_symmetric_form(sq):
    w, B, H, e_nuc, sub, rank = sq
    e, n, r, A, Bc = _energy(w, B, H, e_nuc, sub, rank)
    m = w.system.n_omega
    Hd = np.einsum("mp,mn,np->p", w.C[:, :m], H, w.C[:, :m])
    Delta, Pi = pnof7.delta_pi(n, sub, rank)
    e2 = pnof7.energy_eq_pnof(n, Hd, r["J"], r["K"], Delta, Pi, e_nuc)
    assert abs(e - e2) < 1e-12 * abs(e)
    np.testing.assert_allclose(A, A.T, atol=0)
    np.testing.assert_allclose(Bc, Bc.T, atol=0)


def test_reduces_to_closed_shell_determinant(sq):
    w, B, H, e_nuc, sub, rank = sq
    s = w.system
    gam = w.gamma.copy()
    gam[: s.n_strong] = 0.0
    e, n, r, A, Bc = _energy(w, B, H, e_nuc, sub, rank, gamma=gam)
    e_rhf = rhf.closed_shell_energy(B, H, w.C[:, : s.n_strong], e_nuc)
    assert abs(e - e_rhf) < 1e-12 * abs(e_rhf)


def test_single_pair_is_paired_two_electron_wavefunction():
    w = make_workload("square4")
    s = w.system
    B, L, G = ri.setup(s)
    H = I.core_hamiltonian(s)
    ng = 5
    sub, rank = pairing_columns(1, ng)
    gam = np.array([0.4, 0.3, 0.9, 0.2, 1.2])
    n = pnof7.occupations(gam, 1, ng, sub, rank)
    m = 1 + ng
    C = w.C[:, :m]
    r = ri.all_rows(B, w.C, m)
    Hd = np.einsum("mp,mn,np->p", C, H, C)
    A, Bc = pnof7.coupling(n, sub, rank)
    e = pnof7.energy(n, Hd, r["J"], r["K"], A, Bc, 0.0)
    mo = brute.mo_eri4(brute.fitted_eri4(B), C)
    c = np.where(rank < 0, 1.0, -1.0) * np.sqrt(n)
    # <Psi|H|Psi> over paired determinants: 2 sum c_p^2 h_pp + sum_pq c_p c_q (pq|pq)
    e_wf = 2.0 * np.sum(c * c * Hd) + np.einsum("p,q,pqpq->", c, c, mo)
    assert abs(e - e_wf) < 1e-12 * abs(e_wf)


def test_lagrangian_energy_and_finite_differences(sq):
    w, B, H, e_nuc, sub, rank = sq
    s = w.system
    m = s.n_omega
    e, n, r, A, Bc = _energy(w, B, H, e_nuc, sub, rank)
    lam = pnof7.lagrangian(w.C, H, r["Jao"], r["Kao"], n, A, Bc)
    Hd = np.einsum("mp,mn,np->p", w.C[:, :m], H, w.C[:, :m])
    assert abs(pnof7.energy_from_lagrangian(lam, n, Hd, e_nuc) - e) < 1e-12 * abs(e)
    np.testing.assert_allclose(lam[:, m:], 0.0)
    h = 1e-5
    # dE/dC_{mu p} = 4 (F^(p) C_p)_mu, recovered from lambda as (C^-T lambda)
    grad = 4.0 * np.linalg.solve(w.C.T, lam)
    for (mu, p) in [(0, 0), (5, 3), (17, 7), (23, 11), (9, 15)]:
        Cp = w.C.copy(); Cp[mu, p] += h
        Cm = w.C.copy(); Cm[mu, p] -= h
        fd = (_energy(w, B, H, e_nuc, sub, rank, C=Cp)[0] - _energy(w, B, H, e_nuc, sub, rank, C=Cm)[0]) / (2 * h)
        assert abs(fd - grad[mu, p]) < 1e-7 * max(1.0, abs(fd)), (mu, p, fd, grad[mu, p])
    # Orbital rotation C -> C expm(kappa): dE/dkappa_qp = 4 (lambda_qp - lambda_pq).
    from scipy.linalg import expm
    for (q, p) in [(0, 1), (2, 9), (11, 4), (20, 3)]:
        kap = np.zeros((s.nbf, s.nbf)); kap[q, p] = h; kap[p, q] = -h
        ep = _energy(w, B, H, e_nuc, sub, rank, C=w.C @ expm(kap))[0]
        em = _energy(w, B, H, e_nuc, sub, rank, C=w.C @ expm(-kap))[0]
        fd = (ep - em) / (2 * h)
        ref = 4.0 * (lam[q, p] - lam[p, q])
        assert abs(fd - ref) < 1e-7 * max(1.0, abs(fd)), (q, p, fd, ref)


def test_energy_gradient_wrt_gamma_is_finite_and_consistent(sq):
    """Occupation-angle derivatives by central differences agree between the two energy forms."""
    w, B, H, e_nuc, sub, rank = sq
    s = w.system
    m = s.n_omega
    r = ri.all_rows(B, w.C, m)
    Hd = np.einsum("mp,mn,np->p", w.C[:, :m], H, w.C[:, :m])

    def e1(g):
        n = pnof7.occupations(g, s.n_strong, s.n_weak_per, sub, rank)
        A, Bc = pnof7.coupling(n, sub, rank)
        return pnof7.energy(n, Hd, r["J"], r["K"], A, Bc, e_nuc)

    def e2(g):
        n = pnof7.occupations(g, s.n_strong, s.n_weak_per, sub, rank)
        D, P = pnof7.delta_pi(n, sub, rank)
        return pnof7.energy_eq_pnof(n, Hd, r["J"], r["K"], D, P, e_nuc)

    h = 1e-6
    for k in range(len(w.gamma)):
        gp = w.gamma.copy(); gp[k] += h
        gm = w.gamma.copy(); gm[k] -= h
        d1 = (e1(gp) - e1(gm)) / (2 * h)
        d2 = (e2(gp) - e2(gm)) / (2 * h)
        assert np.isfinite(d1) and abs(d1 - d2) < 1e-7


@pytest.mark.parametrize("name", ["square4", "c6h12"])
def test_contracted_lagrangian_equals_the_per_orbital_form(name):
    """lambda from the RI transforms directly (no J^(q), K^(q)) equals lambda from
    the per-orbital AO matrices: two routes through the same algebra."""
    from oracle import integrals as I, pnof7, ri
    from synthetic import pairing_columns
    from tests.workloads import make_workload
    w = make_workload(name)
    s = w.system
    m = s.n_omega
    B, L, G = ri.setup(s)
    r = ri.all_rows(B, w.C, m)
    sub, rank = pairing_columns(s.n_strong, s.n_weak_per)
    n = pnof7.occupations(w.gamma, s.n_strong, s.n_weak_per, sub, rank)
    A, Bc = pnof7.coupling(n, sub, rank)
    H = I.core_hamiltonian(s)
    lam = pnof7.lagrangian(w.C, H, r["Jao"], r["Kao"], n, A, Bc)
    lam_c = pnof7.lagrangian_contracted(w.C, H, r["bh"], r["d"], r["bf"], n, A, Bc)
    np.testing.assert_allclose(lam_c, lam, atol=1e-11 * np.abs(lam).max())
