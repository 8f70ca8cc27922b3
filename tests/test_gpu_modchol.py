"""GPU parity of the modified Cholesky fit (donof_ri_init_ex with
DONOF_RI_METRIC_MODIFIED) against the FP64 oracle.

* Nothing raised (tol 1e-10): the engine's J, K, E and lambda equal the oracle's
  (the plain Cholesky fit, to which they are invariant), its pivot counts equal
  the oracle's Bunch-Kaufman counts, and the L it keeps equals the oracle's L.
* Eigenvalues raised (tol 1e-3): J / K equal the oracle's corrected fit.
* A redundant auxiliary set: plain Cholesky init reports E_METRIC_NOT_PD, the
  modified one succeeds with the J / K of the set without the duplicates.
* The digit-plane (SLICE4) path on the modified fit keeps its 1e-7 J / K bar.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _oracle_rows(system, C, B):
    from oracle import ri
    return ri.all_rows(B, C, system.n_omega)


@pytest.mark.parametrize("name", ["square4", "c6h12"])
def test_modified_fit_nothing_raised(name):
    from paper_2012_15662_gb300 import binding as bd
    from oracle import integrals as I, modchol, pnof7, ri
    from tests.workloads import make_workload
    w = make_workload(name)
    s = w.system
    eng = bd.Engine(s, bd.DONOF_RI_FP64, metric=bd.DONOF_RI_METRIC_MODIFIED, metric_tol=1e-10)
    n2, nraised, nswap = bd.donof_ri_metric_info(eng.ctx)
    G, X = I.metric(s), I.eri3(s)
    perm, L, starts, sizes, D, swaps = modchol.bunch_kaufman(G)
    assert (n2, nraised, nswap) == (int((sizes == 2).sum()), 0, swaps)
    Lg = np.empty((s.naux, s.naux))
    eng_fetch(eng, bd.DONOF_RI_FETCH_METRIC, Lg)
    np.testing.assert_allclose(Lg, L, atol=1e-12 * max(1.0, np.abs(L).max()))
    eng.transform(w.C, bd.DONOF_RI_FULL)
    J, K = eng.jk_mo()
    eng.jk_ao(want=False)
    E, lam = eng.energy_lagrangian(w.gamma)
    eng.close()
    B0, _, _ = ri.setup(s, eri3=X, G=G)
    r = _oracle_rows(s, w.C, B0)
    np.testing.assert_allclose(J, r["J"], atol=1e-10 * np.abs(r["J"]).max())
    np.testing.assert_allclose(K, r["K"], atol=1e-10 * np.abs(r["K"]).max())
    H = I.core_hamiltonian(s)
    m = s.n_omega
    sub, rank = eng.subspace, eng.weak_rank
    n = pnof7.occupations(w.gamma, s.n_strong, s.n_weak_per, sub, rank)
    A, Bc = pnof7.coupling(n, sub, rank)
    Hd = np.einsum("mp,mn,np->p", w.C[:, :m], H, w.C[:, :m])
    E_ref = pnof7.energy(n, Hd, r["J"], r["K"], A, Bc, I.nuclear_repulsion(s))
    lam_ref = pnof7.lagrangian(w.C, H, r["Jao"], r["Kao"], n, A, Bc)
    assert abs(E - E_ref) <= 1e-10 * max(1.0, abs(E_ref))
    np.testing.assert_allclose(lam, lam_ref, atol=1e-10 * np.abs(lam_ref).max())


def eng_fetch(eng, what, dst):
    from paper_2012_15662_gb300 import binding as bd
    bd.donof_ri_fetch(eng.ctx, what, dst)


def test_modified_fit_with_raised_eigenvalues():
    from paper_2012_15662_gb300 import binding as bd
    from oracle import integrals as I, modchol
    from tests.workloads import make_workload
    w = make_workload("square4")
    s = w.system
    tol = 1e-3
    eng = bd.Engine(s, bd.DONOF_RI_FP64, metric=bd.DONOF_RI_METRIC_MODIFIED, metric_tol=tol)
    B, f = modchol.fitted_tensor_modified(I.eri3(s), I.metric(s), tol)
    n2, nraised, nswap = bd.donof_ri_metric_info(eng.ctx)
    assert nraised == f["raised"] > 0
    assert n2 == int((f["sizes"] == 2).sum())
    assert nswap == f["nswap"]
    eng.transform(w.C, bd.DONOF_RI_FULL)
    J, K = eng.jk_mo()
    Bg = np.empty((s.naux, s.nbf, s.nbf))
    eng_fetch(eng, bd.DONOF_RI_FETCH_B, Bg)
    eng.close()
    r = _oracle_rows(s, w.C, B)
    np.testing.assert_allclose(J, r["J"], atol=1e-10 * np.abs(r["J"]).max())
    np.testing.assert_allclose(K, r["K"], atol=1e-10 * np.abs(r["K"]).max())
    # same pivots, same blocks: the fitted tensor itself agrees
    np.testing.assert_allclose(Bg, B, atol=1e-10 * np.abs(B).max())


@pytest.mark.parametrize("rel", [1e-6, 1e-9])
def test_redundant_auxiliary_set(rel):
    from paper_2012_15662_gb300 import binding as bd
    from oracle import ri
    from synthetic import with_near_duplicate_aux
    from tests.workloads import make_workload
    w = make_workload("square4")
    s = w.system
    sd = with_near_duplicate_aux(s, 8, rel)
    with pytest.raises(bd.DonofError) as ei:
        bd.Engine(sd, bd.DONOF_RI_FP64)
    assert ei.value.status == bd.DONOF_RI_E_METRIC_NOT_PD
    eng = bd.Engine(sd, bd.DONOF_RI_FP64, metric=bd.DONOF_RI_METRIC_MODIFIED, metric_tol=1e-8)
    assert bd.donof_ri_metric_info(eng.ctx)[1] >= 1
    eng.transform(w.C, bd.DONOF_RI_FULL)
    J, K = eng.jk_mo()
    eng.close()
    B0, _, _ = ri.setup(s)
    r = _oracle_rows(s, w.C, B0)
    np.testing.assert_allclose(J, r["J"], atol=1e-8 * np.abs(r["J"]).max())
    np.testing.assert_allclose(K, r["K"], atol=1e-8 * np.abs(r["K"]).max())


def test_slice4_on_the_modified_fit():
    from paper_2012_15662_gb300 import binding as bd
    from oracle import ri
    from tests.workloads import make_workload
    w = make_workload("c6h12")
    s = w.system
    eng = bd.Engine(s, bd.DONOF_RI_SLICE4, metric=bd.DONOF_RI_METRIC_MODIFIED, metric_tol=1e-10)
    eng.transform(w.C, bd.DONOF_RI_FULL)
    J, K = eng.jk_mo()
    eng.close()
    B0, _, _ = ri.setup(s)
    r = _oracle_rows(s, w.C, B0)
    assert np.abs(J - r["J"]).max() < 1e-7
    assert np.abs(K - r["K"]).max() < 1e-7


def test_init_ex_rejects_bad_options():
    from paper_2012_15662_gb300 import binding as bd
    from tests.workloads import make_workload
    s = make_workload("square4").system
    for metric, tol in ((7, 1e-8), (bd.DONOF_RI_METRIC_MODIFIED, 0.0), (bd.DONOF_RI_METRIC_MODIFIED, 1.5)):
        with pytest.raises(bd.DonofError) as ei:
            bd.Engine(s, bd.DONOF_RI_FP64, metric=metric, metric_tol=tol)
        assert ei.value.status == bd.DONOF_RI_E_ARG
