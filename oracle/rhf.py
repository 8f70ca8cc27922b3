"""Closed-shell determinant energy from the AO density (oracle, FP64).

Test infrastructure only; see the package docstring.

When every strong orbital is fully occupied (all strong angles zero, so
n_g = 1 and every weak n = 0, Phi = 0) the PNOF7 energy of Eq. (PNOF)
collapses to the energy of the closed-shell determinant built from the first
N_I orbitals.  That energy is computed here by a different route, from the AO
density D = 2 C_occ C_occ^T and RI Coulomb / exchange matrices built from D:
  J[D]_{mu nu} = sum_P B^P_{mu nu} sum_{l s} B^P_{l s} D_{l s}
  K[D]_{mu nu} = sum_P sum_{l s} B^P_{mu l} D_{l s} B^P_{s nu}
  E = E_nuc + 1/2 sum_{mu nu} D_{mu nu} (2 H_{mu nu} + J[D]_{mu nu} - K[D]_{mu nu} / 2)
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
