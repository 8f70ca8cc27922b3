"""Pins of the oracle's modified Cholesky fit (Sec. 2, G = P L D L^T P^T with the
Cheng-Higham correction of D's blocks).

* The Bunch-Kaufman factors equal LAPACK's symmetric-indefinite factorisation
  (scipy.linalg.ldl): same permutation, same L and D, on random indefinite
  matrices and on the Coulomb metrics of the synthetic systems.
* P L D L^T P^T reconstructs G; every 2x2 block of D is indefinite.
* With nothing raised, the modified fit gives the J / K of the plain Cholesky
  fit (the two b differ by an orthogonal rotation of the auxiliary index).
* With eigenvalues raised, the fit is the exact RI fit with the corrected metric
  G~ = P L D~ L^T P^T, and G~ - G is positive semi-definite.
* On an auxiliary set made linearly dependent by near-duplicate functions the
  plain Cholesky fails, and the modified fit reproduces the J / K of the set
  without the duplicates (the fitting space is the same).
"""
import numpy as np
import pytest
import scipy.linalg as sl

from oracle import integrals as I, modchol, ri
from synthetic import with_near_duplicate_aux
from tests.workloads import make_workload


def _random_symmetric(n, seed):
    A = np.random.default_rng(seed).standard_normal((n, n))
    return A + A.T


@pytest.mark.parametrize("n,seed", [(8, 1), (40, 2), (130, 3)])
def test_bunch_kaufman_matches_lapack_random(n, seed):
    A = _random_symmetric(n, seed)
    perm, L, starts, sizes, D, _ = modchol.bunch_kaufman(A)
    lu, d, p = sl.ldl(A, lower=True)
    np.testing.assert_array_equal(perm, p)
    np.testing.assert_allclose(L, lu[p], atol=1e-12 * np.abs(L).max())
    np.testing.assert_allclose(D, d, atol=1e-12 * np.abs(A).max())
    assert (sizes == 2).sum() > 0  # an indefinite matrix exercises the 2x2 pivots


@pytest.mark.parametrize("name", ["square4", "c6h12"])
def test_bunch_kaufman_matches_lapack_metric(name):
    G = I.metric(make_workload(name).system)
    perm, L, starts, sizes, D, _ = modchol.bunch_kaufman(G)
    lu, d, p = sl.ldl(G, lower=True)
    np.testing.assert_array_equal(perm, p)
    np.testing.assert_allclose(L, lu[p], atol=1e-11)
    np.testing.assert_allclose(D, d, atol=1e-12 * np.abs(G).max())
    assert (perm != np.arange(len(G))).any()  # the metric does pivot


@pytest.mark.parametrize("n,seed", [(40, 5), (130, 6)])
def test_factors_reconstruct_and_pivot_blocks_are_indefinite(n, seed):
    A = _random_symmetric(n, seed)
    perm, L, starts, sizes, D, _ = modchol.bunch_kaufman(A)
    np.testing.assert_allclose(L @ D @ L.T, A[np.ix_(perm, perm)], atol=1e-12 * n * np.abs(A).max())
    np.testing.assert_array_equal(np.triu(L, 1), 0.0)
    np.testing.assert_array_equal(np.diag(L), 1.0)
    for k, s in zip(starts, sizes):
        if s == 2:
            assert np.linalg.det(D[k:k + 2, k:k + 2]) < 0.0
            np.testing.assert_array_equal(L[k + 1, k], 0.0)


@pytest.mark.parametrize("name", ["square4", "c6h12"])
def test_modified_fit_equals_cholesky_fit_when_nothing_is_raised(name):
    w = make_workload(name)
    s = w.system
    G, X = I.metric(s), I.eri3(s)
    B, f = modchol.fitted_tensor_modified(X, G, 1e-10)
    assert f["raised"] == 0
    B0, _, _ = ri.setup(s, eri3=X, G=G)
    r, r0 = ri.all_rows(B, w.C, s.n_omega), ri.all_rows(B0, w.C, s.n_omega)
    for key in ("J", "K", "Jao", "Kao"):
        np.testing.assert_allclose(r[key], r0[key], atol=1e-12 * max(1.0, np.abs(r0[key]).max()))


def test_raised_eigenvalues_give_the_fit_of_the_corrected_metric():
    s = make_workload("square4").system
    G, X = I.metric(s), I.eri3(s)
    tol = 1e-3
    B, f = modchol.fitted_tensor_modified(X, G, tol)
    assert f["raised"] > 0
    delta = tol * np.diag(G).max()
    for k, sz in zip(f["starts"], f["sizes"]):
        assert np.linalg.eigvalsh(f["Dt"][k:k + sz, k:k + sz]).min() >= delta * (1 - 1e-12)
    Gt = modchol.corrected_metric(f)
    assert np.linalg.eigvalsh(Gt - G).min() > -1e-12 * np.abs(G).max()
    nx, nb, _ = X.shape
    Xm = X.reshape(nx, nb * nb)
    fitted = B.reshape(nx, -1).T @ B.reshape(nx, -1)          # sum_P b^P b^P
    exact = Xm.T @ np.linalg.solve(Gt, Xm)                     # (mu nu|.) G~^-1 (.|l s)
    np.testing.assert_allclose(fitted, exact, atol=1e-10 * np.abs(exact).max())


@pytest.mark.parametrize("rel", [1e-6, 1e-9])
def test_redundant_auxiliary_set(rel):
    w = make_workload("square4")
    s = w.system
    sd = with_near_duplicate_aux(s, 8, rel)
    G, X = I.metric(sd), I.eri3(sd)
    with pytest.raises(ri.MetricNotPositiveDefinite):
        ri.metric_cholesky(G)
    B, f = modchol.fitted_tensor_modified(X, G, 1e-8)
    assert f["raised"] >= 1
    B0, _, _ = ri.setup(s)
    r, r0 = ri.all_rows(B, w.C, s.n_omega), ri.all_rows(B0, w.C, s.n_omega)
    for key in ("J", "K", "Jao", "Kao"):
        np.testing.assert_allclose(r[key], r0[key], atol=1e-9 * max(1.0, np.abs(r0[key]).max()))
