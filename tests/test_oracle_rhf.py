"""Pins of the oracle's closed-shell SCF (oracle.rhf.scf), the Hartree-Fock NO
guess of Sec. 4:

* minimal-basis H2 (STO-3G at R = 1.4 bohr, exact four-centre integrals): the
  orbital, electronic and total energies printed by Szabo & Ostlund
  (tests/golden/sto3g_h2_scf.json);
* on square4 with RI integrals: the converged energy equals the determinant
  energy of closed_shell_energy (pinned separately against PNOF7 at full
  occupation), the orbitals are S-orthonormal, the Roothaan-Hall commutator
  vanishes, and small occupied-virtual rotations raise the energy (a minimum).
"""
import json
import os

import numpy as np
import pytest
from scipy.linalg import expm

from oracle import integrals as I, rhf, ri
from tests.workloads import make_workload
from synthetic.systems import System

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _h2_sto3g():
    g = json.load(open(os.path.join(GOLDEN, "sto3g_h2.json")))
    zeta, R = g["zeta"], g["R_bohr"]
    alphas = np.array(g["sto3g_1s_exponents_zeta1"]) * zeta ** 2
    coef = np.array(g["sto3g_1s_coefficients"])
    s = System(name="h2", atom_xyz=np.array([[0.0, 0.0, 0.0], [0.0, 0.0, R]]), atom_charge=np.array([1.0, 1.0]),
               bf_atom=np.array([0, 0, 0, 1, 1, 1], dtype=np.int32), bf_alpha=np.concatenate([alphas, alphas]),
               aux_atom=np.array([0], dtype=np.int32), aux_alpha=np.array([1.0]), n_strong=1, n_weak_per=1)
    D = np.zeros((6, 2))
    D[:3, 0] = coef
    D[3:, 1] = coef
    S = D.T @ I.overlap(s) @ D
    H = D.T @ I.core_hamiltonian(s) @ D
    eri = np.einsum("abcd,ai,bj,ck,dl->ijkl", I.eri4(s), D, D, D, D)
    return S, H, eri, I.nuclear_repulsion(s)


def test_minimal_basis_h2_matches_the_printed_scf():
    g = json.load(open(os.path.join(GOLDEN, "sto3g_h2_scf.json")))
    S, H, eri, enuc = _h2_sto3g()
    assert enuc == pytest.approx(1.0 / g["R_bohr"], rel=1e-14)
    r = rhf.scf(H, S, rhf.jk_exact(eri), 1, enuc)
    tol = g["tolerance"]
    assert r["commutator"] <= 1e-10
    assert abs(r["eps"][0] - g["eps1"]) <= tol and abs(r["eps"][1] - g["eps2"]) <= tol
    assert abs((r["E"] - enuc) - g["E0_electronic"]) <= tol
    assert abs(r["E"] - g["E_total"]) <= tol


@pytest.fixture(scope="module")
def sq_scf():
    w = make_workload("square4")
    s = w.system
    B, L, G = ri.setup(s)
    H = I.core_hamiltonian(s)
    S = I.overlap(s)
    enuc = I.nuclear_repulsion(s)
    r = rhf.scf(H, S, rhf.jk_ri(B), s.n_strong, enuc)
    return s, B, H, S, enuc, r


def test_ri_scf_is_a_converged_closed_shell_determinant(sq_scf):
    s, B, H, S, enuc, r = sq_scf
    C = r["C"]
    assert r["commutator"] <= 1e-10 and r["iterations"] < 100
    np.testing.assert_allclose(C.T @ S @ C, np.eye(s.nbf), atol=1e-10)
    assert np.all(np.diff(r["eps"]) >= 0.0)
    E_det = rhf.closed_shell_energy(B, H, C[:, :s.n_strong], enuc)
    assert r["E"] == pytest.approx(E_det, abs=1e-10)


def test_ri_scf_energy_is_a_minimum(sq_scf):
    s, B, H, S, enuc, r = sq_scf
    C, no, nb = r["C"], s.n_strong, s.nbf
    rng = np.random.default_rng(11)
    for _ in range(5):
        kappa = np.zeros((nb, nb))
        kappa[no:, :no] = 1e-3 * rng.standard_normal((nb - no, no))
        kappa = kappa - kappa.T
        C1 = C @ expm(kappa)                     # stays S-orthonormal
        E1 = rhf.closed_shell_energy(B, H, C1[:, :no], enuc)
        assert E1 > r["E"]


def test_pnof7_at_hf_orbitals(sq_scf):
    """At the SCF orbitals PNOF7 with every strong orbital full (gamma = 0) is the
    SCF energy; optimising the occupations from the standard guess then gives a
    small negative correlation energy (gamma = 0 is itself a feasible point)."""
    from oracle import onopt, pnof7
    from synthetic import pairing_columns
    s, B, H, S, enuc, r = sq_scf
    m = s.n_omega
    C = r["C"]
    rows = ri.all_rows(B, C, m)
    Hd = np.einsum("mp,mn,np->p", C[:, :m], H, C[:, :m])
    sub, rank = pairing_columns(s.n_strong, s.n_weak_per)
    g0 = np.zeros(s.n_strong * s.n_weak_per)
    n0 = pnof7.occupations(g0, s.n_strong, s.n_weak_per, sub, rank)
    A, Bc = pnof7.coupling(n0, sub, rank)
    assert pnof7.energy(n0, Hd, rows["J"], rows["K"], A, Bc, enuc) == pytest.approx(r["E"], abs=1e-10)
    _, E_opt, _, _, _ = onopt.optimize(onopt.standard_guess(s.n_strong, s.n_weak_per), s.n_strong, s.n_weak_per,
                                       sub, rank, Hd, rows["J"], rows["K"], enuc)
    assert -1.0 < E_opt - r["E"] < 0.0
