"""Closed-shell determinant energy from the AO density, and the closed-shell
Hartree-Fock orbitals of the NO guess (oracle, FP64).

Test infrastructure only; see the package docstring.

When every strong orbital is fully occupied (all strong angles zero, so
n_g = 1 and every weak n = 0, Phi = 0) the PNOF7 energy of Eq. (PNOF)
collapses to the energy of the closed-shell determinant built from the first
N_I orbitals.  That energy is computed here by a different route, from the AO
density D = 2 C_occ C_occ^T and RI Coulomb / exchange matrices built from D:
  J[D]_{mu nu} = sum_P B^P_{mu nu} sum_{l s} B^P_{l s} D_{l s}
  K[D]_{mu nu} = sum_P sum_{l s} B^P_{mu l} D_{l s} B^P_{s nu}
  E = E_nuc + 1/2 sum_{mu nu} D_{mu nu} (2 H_{mu nu} + J[D]_{mu nu} - K[D]_{mu nu} / 2)
Pins of the SCF (tests/test_oracle_rhf.py): the printed minimal-basis H2 result,
its energy against closed_shell_energy, convergence and the minimum.
"""
from __future__ import annotations

import numpy as np


def closed_shell_energy(B: np.ndarray, H: np.ndarray, C_occ: np.ndarray, e_nuc: float) -> float:
    D = 2.0 * C_occ @ C_occ.T
    nx, nb, _ = B.shape
    Bf = B.reshape(nx, nb * nb)
    Jd = (Bf.T @ (Bf @ D.reshape(-1))).reshape(nb, nb)
    Kd = np.einsum("Pml,ls,Psn->mn", B, D, B, optimize=True)
    F = H + Jd - 0.5 * Kd
    return float(e_nuc + 0.5 * np.sum(D * (H + F)))


# ---------------------------------------------------------------------------
# Closed-shell Hartree-Fock orbitals: the NO guess of Sec. 4 (the guess MOs
# come from a Hartree-Fock calculation).  Roothaan-Hall equations in the overlap
# metric, F C = S C eps with F = H + J[D] - K[D] / 2 and D = 2 C_occ C_occ^T,
# iterated from the core-Hamiltonian guess with Pulay's DIIS (direct inversion
# in the iterative subspace: the Fock matrix extrapolated from the last few with
# coefficients that minimise the norm of the combined error F D S - S D F,
# subject to their sum being one).
# ---------------------------------------------------------------------------
def jk_ri(B: np.ndarray):
    """J[D], K[D] from the fitted three-index tensor (the RI route, as above)."""
    nx, nb, _ = B.shape
    Bf = B.reshape(nx, nb * nb)

    def jk(D):
        Jd = (Bf.T @ (Bf @ D.reshape(-1))).reshape(nb, nb)
        Kd = np.einsum("Pml,ls,Psn->mn", B, D, B, optimize=True)
        return Jd, Kd

    return jk


def jk_exact(eri: np.ndarray):
    """J[D]_mn = sum_ls (mn|ls) D_ls, K[D]_mn = sum_ls (ml|ns) D_ls from four-index integrals."""

    def jk(D):
        return np.einsum("mnls,ls->mn", eri, D), np.einsum("mlns,ls->mn", eri, D)

    return jk


def scf(H: np.ndarray, S: np.ndarray, jk, n_occ: int, e_nuc: float, max_iter: int = 200, tol: float = 1e-10,
        n_diis: int = 8) -> dict:
    """Closed-shell SCF.  Returns dict(C: all orbitals, S-orthonormal, by ascending
    eps; eps; E (total energy); iterations; commutator: max |F D S - S D F| of the
    last Fock matrix)."""
    from scipy.linalg import eigh
    eps, C = eigh(H, S)
    Fs, errs = [], []
    E, it, com = 0.0, 0, np.inf
    for it in range(1, max_iter + 1):
        Cocc = C[:, :n_occ]
        D = 2.0 * Cocc @ Cocc.T
        Jd, Kd = jk(D)
        F = H + Jd - 0.5 * Kd
        E = float(e_nuc + 0.5 * np.sum(D * (H + F)))
        err = F @ D @ S - S @ D @ F
        com = float(np.abs(err).max())
        if com <= tol:
            eps, C = eigh(F, S)
            break
        Fs.append(F)
        errs.append(err)
        Fs, errs = Fs[-n_diis:], errs[-n_diis:]
        m = len(Fs)
        A = -np.ones((m + 1, m + 1))
        A[m, m] = 0.0
        for i in range(m):
            for j in range(m):
                A[i, j] = np.sum(errs[i] * errs[j])
        rhs = np.zeros(m + 1)
        rhs[m] = -1.0
        c = np.linalg.lstsq(A, rhs, rcond=None)[0][:m]
        eps, C = eigh(sum(ci * Fi for ci, Fi in zip(c, Fs)), S)
    return dict(C=C, eps=eps, E=E, iterations=it, commutator=com)
