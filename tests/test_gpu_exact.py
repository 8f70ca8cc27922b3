"""Exact four-centre J / K on the device (donof_ri_exact_jk), the conventional
algorithm the paper's RI -> exact restart returns to.

* square4: J, K, J^(q), K^(q) against the oracle's conventional algorithm on its
  exact s-type integrals (oracle.brute.conventional_jk on oracle.integrals.eri4),
  then the energy and Lagrangian that follow on the exact integrals, and the
  occupation optimisation on exact J / K reaching the oracle optimiser's minimum;
* C6H12 at full size: the exact results against the RI ones through what the
  Coulomb-metric fit guarantees: the fitted four-index tensor lies below the
  exact one in pair space, so J_exact - J_RI is positive semi-definite and
  K_exact - K_RI is non-negative element by element; J, K symmetric, J_pp = K_pp.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import brute, integrals as I, onopt, pnof7  # noqa: E402
from synthetic import pairing_columns  # noqa: E402
from tests.workloads import make_workload  # noqa: E402


def test_exact_square4_matches_conventional_oracle():
    from paper_2012_15662_gb300 import binding as bd
    w = make_workload("square4")
    s = w.system
    m = s.n_omega
    eng = bd.Engine(s, bd.DONOF_RI_FP64)
    J = np.empty((m, m))
    K = np.empty((m, m))
    bd.donof_ri_exact_jk(eng.ctx, bd.Engine.colmajor(w.C), J, K)
    E, lam = eng.energy_lagrangian(w.gamma)
    eri = I.eri4(s)
    Jo, Ko, Jao, Kao = brute.conventional_jk(eri, w.C, m)
    scale = np.abs(Jo).max()
    np.testing.assert_allclose(J, Jo, atol=1e-12 * scale)
    np.testing.assert_allclose(K, Ko, atol=1e-12 * scale)
    sub, rank = pairing_columns(s.n_strong, s.n_weak_per)
    n = pnof7.occupations(w.gamma, s.n_strong, s.n_weak_per, sub, rank)
    A, Bc = pnof7.coupling(n, sub, rank)
    H = I.core_hamiltonian(s)
    Hd = np.einsum("mp,mn,np->p", w.C[:, :m], H, w.C[:, :m])
    enuc = I.nuclear_repulsion(s)
    E_ref = pnof7.energy(n, Hd, Jo, Ko, A, Bc, enuc)
    lam_ref = pnof7.lagrangian(w.C, H, Jao, Kao, n, A, Bc)
    assert abs(E - E_ref) <= 1e-11 * max(1.0, abs(E_ref))
    np.testing.assert_allclose(lam, lam_ref, atol=1e-11 * np.abs(lam_ref).max())
    # occupation optimisation on the exact J / K (the restart's outer step)
    g0 = onopt.standard_guess(s.n_strong, s.n_weak_per)
    g, Eg, grad, it, reason = eng.optimize_occupations(g0, max_iter=5000, gtol=1e-9, etol=0.0)
    g_o, E_o = onopt.optimize(g0, s.n_strong, s.n_weak_per, sub, rank, Hd, Jo, Ko, enuc)[:2]
    assert abs(Eg - E_o) <= 1e-8 * max(1.0, abs(E_o))
    eng.close()


def test_exact_c6h12_against_the_ri_fit():
    from paper_2012_15662_gb300 import binding as bd
    w = make_workload("c6h12")
    s = w.system
    m = s.n_omega
    eng = bd.Engine(s, bd.DONOF_RI_FP64)
    eng.transform(w.C, bd.DONOF_RI_FULL)
    J_ri, K_ri = eng.jk_mo()
    eng.jk_ao(want=False)
    E_ri, _ = eng.energy_lagrangian(w.gamma)
    J = np.empty((m, m))
    K = np.empty((m, m))
    bd.donof_ri_exact_jk(eng.ctx, bd.Engine.colmajor(w.C), J, K)
    E_ex, lam = eng.energy_lagrangian(w.gamma)
    eng.close()
    scale = np.abs(J).max()
    np.testing.assert_allclose(J, J.T, atol=1e-12 * scale)
    np.testing.assert_allclose(K, K.T, atol=1e-12 * scale)
    np.testing.assert_allclose(np.diag(J), np.diag(K), atol=1e-12 * scale)
    assert np.linalg.eigvalsh(J - J_ri).min() >= -1e-10 * scale
    assert (K - K_ri).min() >= -1e-12 * scale
    # the fit is good: RI errors small against the integrals themselves
    assert np.abs(J - J_ri).max() <= 1e-2 * scale
    assert np.isfinite(E_ex) and np.isfinite(lam).all() and E_ex != E_ri


def test_exact_rejects_other_precisions():
    from paper_2012_15662_gb300 import binding as bd
    w = make_workload("square4")
    eng = bd.Engine(w.system, bd.DONOF_RI_SLICE4)
    with pytest.raises(bd.DonofError) as e:
        bd.donof_ri_exact_jk(eng.ctx, bd.Engine.colmajor(w.C))
    assert e.value.status == bd.DONOF_RI_E_UNSUPPORTED
    eng.close()
