"""Pins of the oracle's RI algebra (factored path vs brute force and invariants).

P1  factored RI (Tables 2-3) == conventional Table 1 applied to the fitted
    four-index tensor of Eq. (AOERI), with an explicit O(N^5) transform.
P2  invariants: J, K symmetric; J_pp = K_pp; K_pq >= 0; fitted ERI PSD;
    J_pq = C_p^T J^(q) C_p and K_pq = C_p^T K^(q) C_p (ties J/K to J^(q)/K^(q)).
P5  Cholesky-fitted B and the symmetric G^-1/2 fitting give the same results.
RI  Coulomb-metric fitting is variational: exact - fitted is PSD in pair space.
"""
import numpy as np
import pytest

from oracle import brute, integrals as I, ri
from synthetic.systems import System, random_orthogonal
from tests.workloads import make_workload


def _two_atom():
    return System(name="two", atom_xyz=np.array([[0.0, 0.0, 0.0], [0.0, 0.3, 1.6]]),
                  atom_charge=np.array([1.0, 1.0]),
                  bf_atom=np.array([0, 0, 0, 1, 1, 1], np.int32),
                  bf_alpha=np.array([0.2, 1.1, 4.0, 0.35, 1.4, 6.0]),
                  aux_atom=np.array([0] * 8 + [1] * 8, np.int32),
                  aux_alpha=np.concatenate([0.25 * 2.3 ** np.arange(8), 0.3 * 2.1 ** np.arange(8)]),
                  n_strong=1, n_weak_per=2)


@pytest.fixture(scope="module")
def square():
    w = make_workload("square4")
    B, L, G = ri.setup(w.system)
    return w, B, L, G


def _check_against_brute(B, C, n_om, tol):
    rows = ri.all_rows(B, C, n_om)
    eri = brute.fitted_eri4(B)
    J, K, Jao, Kao = brute.conventional_jk(eri, C, n_om)
    scale = max(1.0, np.abs(eri).max())
    np.testing.assert_allclose(rows["J"], J, atol=tol * scale)
    np.testing.assert_allclose(rows["K"], K, atol=tol * scale)
    np.testing.assert_allclose(rows["Jao"], Jao, atol=tol * scale)
    np.testing.assert_allclose(rows["Kao"], Kao, atol=tol * scale)
    mo = brute.mo_eri4(eri, C[:, :n_om])
    np.testing.assert_allclose(rows["J"], np.einsum("ppqq->pq", mo), atol=tol * scale)
    np.testing.assert_allclose(rows["K"], np.einsum("pqpq->pq", mo), atol=tol * scale)
    np.testing.assert_allclose(rows["bf"].transpose(1, 2, 0).reshape(n_om * n_om, -1)
                               @ rows["bf"].transpose(1, 2, 0).reshape(n_om * n_om, -1).T,
                               mo.reshape(n_om * n_om, n_om * n_om), atol=tol * scale)


def test_factored_equals_brute_force_two_atom():
    s = _two_atom()
    B, L, G = ri.setup(s)
    C = random_orthogonal(s.nbf, np.random.default_rng(3))
    _check_against_brute(B, C, 5, 1e-12)


def test_factored_equals_brute_force_square(square):
    w, B, L, G = square
    _check_against_brute(B, w.C, w.system.n_omega, 1e-12)


def test_cholesky_and_fitted_tensor(square):
    w, B, L, G = square
    np.testing.assert_allclose(L @ L.T, G, atol=1e-13)
    assert np.allclose(np.triu(L, 1), 0.0)
    e3 = I.eri3(w.system)
    nx, nb, _ = e3.shape
    ref = e3.reshape(nx, -1).T @ np.linalg.solve(G, e3.reshape(nx, -1))
    got = B.reshape(nx, -1).T @ B.reshape(nx, -1)
    np.testing.assert_allclose(got, ref, atol=1e-10 * np.abs(ref).max())


def test_invariants(square):
    w, B, L, G = square
    m = w.system.n_omega
    r = ri.all_rows(B, w.C, m)
    J, K = r["J"], r["K"]
    np.testing.assert_allclose(J, J.T, atol=1e-13)
    np.testing.assert_allclose(K, K.T, atol=1e-13)
    np.testing.assert_allclose(np.diag(J), np.diag(K), atol=1e-13)
    assert (K >= -1e-15).all()
    C = w.C[:, :m]
    np.testing.assert_allclose(np.einsum("mp,qmn,np->pq", C, r["Jao"], C), J, atol=1e-12)
    np.testing.assert_allclose(np.einsum("mp,qmn,np->pq", C, r["Kao"], C), K, atol=1e-12)
    np.testing.assert_allclose(r["Jao"], r["Jao"].transpose(0, 2, 1), atol=1e-13)
    np.testing.assert_allclose(r["Kao"], r["Kao"].transpose(0, 2, 1), atol=1e-13)
    eri = brute.fitted_eri4(B).reshape(w.system.nbf ** 2, -1)
    ev = np.linalg.eigvalsh(eri)
    assert ev.min() > -1e-12 * ev.max()
    # J^(q) is the AO Coulomb matrix of the density C_q C_q^T built directly from B.
    q = 3
    Dq = np.outer(w.C[:, q], w.C[:, q])
    Jq = np.einsum("Pmn,Pls,ls->mn", B, B, Dq)
    np.testing.assert_allclose(r["Jao"][q], Jq, atol=1e-12)
    Kq = np.einsum("Pml,ls,Psn->mn", B, Dq, B)
    np.testing.assert_allclose(r["Kao"][q], Kq, atol=1e-12)


def test_rotation_invariance_cholesky_vs_symmetric(square):
    w, B, L, G = square
    Bs = ri.fitted_tensor_symmetric(I.eri3(w.system), G)
    m = w.system.n_omega
    r1 = ri.all_rows(B, w.C, m)
    r2 = ri.all_rows(Bs, w.C, m)
    for key in ("J", "K", "Jao", "Kao"):
        np.testing.assert_allclose(r1[key], r2[key], atol=1e-9)


def test_ri_fit_is_variational(square):
    w, B, L, G = square
    exact = I.eri4(w.system).reshape(w.system.nbf ** 2, -1)
    fitted = brute.fitted_eri4(B).reshape(w.system.nbf ** 2, -1)
    ev = np.linalg.eigvalsh(exact - fitted)
    assert ev.min() > -1e-10 * np.abs(exact).max()
    # The fit error is small but nonzero for s-only fitting functions.
    rel = np.abs(exact - fitted).max() / np.abs(exact).max()
    assert 1e-8 < rel < 0.2


def test_metric_not_positive_definite_raises():
    G = np.array([[1.0, 2.0], [2.0, 1.0]])
    with pytest.raises(ri.MetricNotPositiveDefinite):
        ri.metric_cholesky(G)
    G = np.array([[1.0, 1.0], [1.0, 1.0 + 1e-16]])
    with pytest.raises(ri.MetricNotPositiveDefinite):
        ri.metric_cholesky(G)


def test_transforms_edge_cases(square):
    w, B, L, G = square
    # One orbital and a sign flip of an orbital (J/K invariant to MO signs).
    r1 = ri.all_rows(B, w.C, 1)
    C2 = w.C.copy()
    C2[:, 0] *= -1.0
    r2 = ri.all_rows(B, C2, 1)
    np.testing.assert_allclose(r1["J"], r2["J"], atol=1e-14)
    np.testing.assert_allclose(r1["K"], r2["K"], atol=1e-14)
    np.testing.assert_allclose(r1["Kao"], r2["Kao"], atol=1e-14)
    # Identity orbitals: b^P_pq is B itself.
    nb = w.system.nbf
    r3 = ri.all_rows(B, np.eye(nb), nb)
    np.testing.assert_allclose(r3["bf"], B, atol=1e-15)


def test_cholesky_orthonormal_basis_leaves_every_result_unchanged():
    """The digit-plane engine computes in the basis chi' = chi L^-T (S = L L^T): orbitals
    C' = L^T C, fitted tensor B'^P = L^-1 B^P L^-T, H' = L^-1 H L^-T.  The RI algebra is
    invariant under it: b^P_pq, J, K and lambda are the same, J^(q), K^(q) and b_half
    come back as L X' L^T and b' L^T; C' is orthogonal when C^T S C = I."""
    from oracle import pnof7
    from synthetic import pairing_columns
    w = make_workload("square4")
    s = w.system
    B, L, G = ri.setup(s)
    S, H = I.overlap(s), I.core_hamiltonian(s)
    Ls = np.linalg.cholesky(S)
    Li = np.linalg.inv(Ls)
    Bp = np.einsum("ij,Pjk,lk->Pil", Li, B, Li)
    Cp = Ls.T @ w.C
    Hp = Li @ H @ Li.T
    np.testing.assert_allclose(Cp.T @ Cp, np.eye(s.nbf), atol=1e-12)
    m = s.n_omega
    r = ri.all_rows(B, w.C, m)
    rp = ri.all_rows(Bp, Cp, m)
    for key in ("d", "bf", "J", "K"):
        np.testing.assert_allclose(rp[key], r[key], atol=1e-12)
    np.testing.assert_allclose(np.einsum("Ppn,mn->Ppm", rp["bh"], Ls), r["bh"], atol=1e-12)
    for key in ("Jao", "Kao"):
        np.testing.assert_allclose(np.einsum("ij,qjk,lk->qil", Ls, rp[key], Ls), r[key], atol=1e-12)
    sub, rank = pairing_columns(s.n_strong, s.n_weak_per)
    n = pnof7.occupations(w.gamma, s.n_strong, s.n_weak_per, sub, rank)
    A, Bc = pnof7.coupling(n, sub, rank)
    lam = pnof7.lagrangian(w.C, H, r["Jao"], r["Kao"], n, A, Bc)
    lamp = pnof7.lagrangian(Cp, Hp, rp["Jao"], rp["Kao"], n, A, Bc)
    np.testing.assert_allclose(lamp, lam, atol=1e-11)


def test_ghost_centre_auxiliary_set_fits_the_basis_products():
    """The "ring_fit" auxiliary set (ghost centres between the atoms) brings the RI
    error of the Hartree-Fock energy of a C3H6 ring from ~0.1 Eh (functions on the
    atoms only, which cannot represent a product of functions on two atoms) to the
    order of the paper's RI errors (Sec. 4, Table 4: 2.2e-4 Eh on average for the
    cycloalkanes).  The ghost centres carry no charge and no basis function, so the
    one-electron integrals and the nuclear repulsion are those of the plain ring."""
    from oracle import rhf
    from synthetic.systems import make_system
    plain = make_system("ring", n_c=3, seed=2)
    fit = make_system("ring_fit", n_c=3, seed=2)
    np.testing.assert_array_equal(fit.atom_xyz[:plain.n_atoms], plain.atom_xyz)
    np.testing.assert_array_equal(fit.bf_alpha, plain.bf_alpha)
    assert fit.n_electrons == plain.n_electrons and fit.naux > plain.naux
    S, H = I.overlap(plain), I.core_hamiltonian(plain)
    e_nuc = I.nuclear_repulsion(plain)
    assert I.nuclear_repulsion(fit) == pytest.approx(e_nuc, abs=1e-12)
    np.testing.assert_allclose(I.core_hamiltonian(fit), H, atol=1e-12)
    n_occ = plain.n_electrons // 2
    E_exact = rhf.scf(H, S, rhf.jk_exact(I.eri4(plain)), n_occ, e_nuc, tol=1e-8)["E"]
    errors = {}
    for s in (plain, fit):
        B, _, _ = ri.setup(s)
        errors[s.name] = rhf.scf(H, S, rhf.jk_ri(B), n_occ, e_nuc, tol=1e-8)["E"] - E_exact
    assert errors[plain.name] > 0.05
    assert 0.0 < errors[fit.name] < 2e-3
