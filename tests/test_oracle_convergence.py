"""The oracle's outer / inner scheme to convergence (oracle/orbopt.converge) and the
paper's RI -> exact restart (Sec. 4 and the Abstract: a converged PNOF7-RI
calculation restarted with four-centre integrals converges in at most two outer
iterations), on square4 from its Hartree-Fock orbitals (oracle/rhf.scf).

Pins: the converged state is a stationary point (max |lambda - lambda^T| <= 1e-4
and the energy is below the Hartree-Fock one, which is PNOF7's closed-shell
limit); the exact restart takes at most two outer iterations and ends lower than
the RI energy evaluated with exact integrals at the RI solution (the restart
only descends), and the RI error lies in the range the fit's variational
property allows (E_RI > E_exact: the Coulomb-metric fit underestimates the
Coulomb-type terms)."""
import numpy as np
import pytest

from oracle import integrals as I, orbopt, rhf, ri
from synthetic import pairing_columns, standard_gamma
from tests.workloads import make_workload


@pytest.fixture(scope="module")
def runs():
    w = make_workload("square4")
    s = w.system
    B, L, G = ri.setup(s)
    H, S, enuc = I.core_hamiltonian(s), I.overlap(s), I.nuclear_repulsion(s)
    hf = rhf.scf(H, S, rhf.jk_ri(B), s.n_strong, enuc, tol=1e-9)
    sub, rank = pairing_columns(s.n_strong, s.n_weak_per)
    g0 = standard_gamma(s.n_strong, s.n_weak_per)
    r = orbopt.converge(s, hf["C"], g0, hf["eps"], sub, rank, B=B)
    eri = I.eri4(s)
    x = orbopt.converge(s, r["C"], r["gamma"], r["diag"], sub, rank, eri=eri)
    return s, hf, r, x, eri, sub, rank


def test_ri_run_converges_below_hartree_fock(runs):
    s, hf, r, x, eri, sub, rank = runs
    assert r["converged"]
    assert r["history"][-1]["gmax"] <= 1e-4
    assert r["E"] < hf["E"] - 1e-3
    E = [h["E"] for h in r["history"]]
    assert all(b <= a + 1e-12 for a, b in zip(E, E[1:]))


def test_exact_restart_takes_at_most_two_outer_iterations(runs):
    s, hf, r, x, eri, sub, rank = runs
    assert x["converged"] and x["outer"] <= 2
    assert x["history"][-1]["gmax"] <= 1e-4
    # the RI solution evaluated with exact integrals is the restart's start: it only descends
    from oracle import pnof7
    m = s.n_omega
    ex = orbopt.exact_rows(eri, r["C"], m)
    H = I.core_hamiltonian(s)
    n = pnof7.occupations(r["gamma"], s.n_strong, s.n_weak_per, sub, rank)
    A, Bc = pnof7.coupling(n, sub, rank)
    Hd = np.einsum("mp,mn,np->p", r["C"][:, :m], H, r["C"][:, :m])
    E_start = pnof7.energy(n, Hd, ex["J"], ex["K"], A, Bc, I.nuclear_repulsion(s))
    assert x["E"] <= E_start + 1e-12
    assert 0.0 < r["E"] - x["E"] < 0.05


def test_exact_rows_equal_the_conventional_algorithm(runs):
    """orbopt.exact_rows (einsum route) against brute.conventional_jk (Table 1 with the
    projectors P^q, a loop per orbital) on the exact four-index integrals."""
    from oracle import brute
    s, hf, r, x, eri, sub, rank = runs
    m = s.n_omega
    a = orbopt.exact_rows(eri, r["C"], m)
    J, K, Jao, Kao = brute.conventional_jk(eri, r["C"], m)
    for got, want in ((a["J"], J), (a["K"], K), (a["Jao"], Jao), (a["Kao"], Kao)):
        np.testing.assert_allclose(got, want, atol=1e-12)
