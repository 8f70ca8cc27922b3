"""Degenerate and ragged cases of the engine against the oracle.

* Closed shell: all strong angles 0 (n_g = 1, every weak n = 0, Phi = 0).  Eq.
  (PNOF) then collapses to the closed-shell determinant energy, which the oracle
  computes by a different route (from the AO density, oracle/rhf.py); the engine's
  energy must match it (FP64: to rounding; SLICE4: within 1e-6 Eh).
* Pairing shapes other than the workloads': N_g = 1 (one weak orbital per
  subspace, no weak angles) and N_g = 3, on a C5H10 ring whose sizes are ragged for
  every tile (nbf 120, naux 420, N_Omega 40 / 80): J, K, J^(q), K^(q), E and lambda
  of the SLICE4 engine within the bars, and the occupation optimiser's energy.
* Odd sizes: the same ring without its last 3 basis and 5 auxiliary functions
  (nbf 117, naux 415): every row of the digit passes ends in a lone column.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import integrals as I, onopt, pnof7, rhf, ri  # noqa: E402
from synthetic import (draw_gamma, make_system, orthonormal_orbitals, pairing_columns,   # noqa: E402
                       random_orthogonal, standard_gamma, without_basis_functions)
from tests.workloads import make_workload  # noqa: E402


@pytest.mark.parametrize("prec", ["fp64", "slice4"])
def test_closed_shell_energy_is_the_determinant_energy(prec):
    from paper_2012_15662_gb300 import binding as bd
    w = make_workload("c6h12")
    s = w.system
    eng = bd.Engine(s, bd.DONOF_RI_FP64 if prec == "fp64" else bd.DONOF_RI_SLICE4)
    eng.transform(w.C, bd.DONOF_RI_HALF)
    eng.jk_ao(want=False)
    E, lam = eng.energy_lagrangian(np.zeros(s.n_strong * s.n_weak_per))
    eng.close()
    B, L, G = ri.setup(s)
    Ed = rhf.closed_shell_energy(B, I.core_hamiltonian(s), w.C[:, :s.n_strong], I.nuclear_repulsion(s))
    tol = 1e-9 * abs(Ed) if prec == "fp64" else 1e-6
    assert abs(E - Ed) <= tol
    # only the occupied orbitals carry lambda columns at n = (1, 0)
    assert np.abs(lam[:, s.n_strong:s.n_omega]).max() <= (1e-12 if prec == "fp64" else 1e-7)


@pytest.mark.parametrize("n_weak", [1, 3])
def test_pairing_shapes_on_a_ragged_ring(n_weak):
    from paper_2012_15662_gb300 import binding as bd
    s = make_system("ring", n_c=5, seed=77, jitter=0.02, n_weak_per=n_weak)
    rng = np.random.default_rng(177)
    C = orthonormal_orbitals(I.overlap(s), random_orthogonal(s.nbf, rng))
    gamma = draw_gamma(s.n_strong, s.n_weak_per, rng)
    m = s.n_omega
    B, L, G = ri.setup(s)
    r = ri.all_rows(B, C, m)
    H = I.core_hamiltonian(s)
    sub, rank = pairing_columns(s.n_strong, s.n_weak_per)
    n = pnof7.occupations(gamma, s.n_strong, s.n_weak_per, sub, rank)
    A, Bc = pnof7.coupling(n, sub, rank)
    Hd = np.einsum("mp,mn,np->p", C[:, :m], H, C[:, :m])
    enuc = I.nuclear_repulsion(s)
    Eo = pnof7.energy(n, Hd, r["J"], r["K"], A, Bc, enuc)
    lamo = pnof7.lagrangian(C, H, r["Jao"], r["Kao"], n, A, Bc)
    eng = bd.Engine(s, bd.DONOF_RI_SLICE4)
    eng.transform(C, bd.DONOF_RI_FULL)
    J, K = eng.jk_mo()
    Jao, Kao = eng.jk_ao()
    E, lam = eng.energy_lagrangian(gamma)
    assert np.abs(J - r["J"]).max() <= 1e-7 and np.abs(K - r["K"]).max() <= 1e-7
    assert np.abs(Jao - r["Jao"]).max() <= 1e-7 and np.abs(Kao - r["Kao"]).max() <= 1e-7
    assert abs(E - Eo) <= 1e-6 and np.abs(lam - lamo).max() <= 1e-6
    g0 = standard_gamma(s.n_strong, s.n_weak_per)
    gam, Eopt, grad, it, reason = eng.optimize_occupations(g0, max_iter=20000, gtol=1e-8, etol=1e-14)
    eng.close()
    go, Eopt_o, no, _, _ = onopt.optimize(g0, s.n_strong, s.n_weak_per, sub, rank, Hd, r["J"], r["K"], enuc,
                                          gtol=1e-9)
    assert reason in (0, 3) and abs(Eopt - Eopt_o) <= 1e-8 * abs(Eopt_o) + 1e-6


@pytest.mark.parametrize("prec", ["slice4", "tf32x3"])
def test_odd_sizes(prec):
    from paper_2012_15662_gb300 import binding as bd
    s = without_basis_functions(make_system("ring", n_c=5, seed=77, jitter=0.02, n_weak_per=3), 3, 5)
    assert s.nbf % 2 == 1 and s.naux % 2 == 1
    rng = np.random.default_rng(178)
    C = orthonormal_orbitals(I.overlap(s), random_orthogonal(s.nbf, rng))
    gamma = draw_gamma(s.n_strong, s.n_weak_per, rng)
    m = s.n_omega
    B, L, G = ri.setup(s)
    r = ri.all_rows(B, C, m)
    H = I.core_hamiltonian(s)
    sub, rank = pairing_columns(s.n_strong, s.n_weak_per)
    n = pnof7.occupations(gamma, s.n_strong, s.n_weak_per, sub, rank)
    A, Bc = pnof7.coupling(n, sub, rank)
    Hd = np.einsum("mp,mn,np->p", C[:, :m], H, C[:, :m])
    Eo = pnof7.energy(n, Hd, r["J"], r["K"], A, Bc, I.nuclear_repulsion(s))
    lamo = pnof7.lagrangian(C, H, r["Jao"], r["Kao"], n, A, Bc)
    eng = bd.Engine(s, bd.DONOF_RI_SLICE4 if prec == "slice4" else bd.DONOF_RI_TF32X3)
    eng.transform(C, bd.DONOF_RI_FULL)
    J, K = eng.jk_mo()
    Jao, Kao = eng.jk_ao()
    E, lam = eng.energy_lagrangian(gamma)
    eng.close()
    if prec == "slice4":  # the digit path's absolute bars
        assert np.abs(J - r["J"]).max() <= 1e-7 and np.abs(K - r["K"]).max() <= 1e-7
        assert np.abs(Jao - r["Jao"]).max() <= 1e-7 and np.abs(Kao - r["Kao"]).max() <= 1e-7
        assert abs(E - Eo) <= 1e-6 and np.abs(lam - lamo).max() <= 1e-6
    else:  # split TF32 with FP32 accumulation: 2e-5 of each result's largest element
        for got, ref in ((J, r["J"]), (K, r["K"]), (Jao, r["Jao"]), (Kao, r["Kao"]), (lam, lamo)):
            assert np.abs(got - ref).max() <= 2e-5 * np.abs(ref).max()
        assert abs(E - Eo) <= 1e-6 * abs(Eo)
