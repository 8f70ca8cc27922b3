"""Four-index brute force (oracle, FP64; small systems only).

Test infrastructure only; see the package docstring.

Builds the fitted AO four-index tensor of Eq. (AOERI),
  (mu nu|l s)_RI = sum_P B^P_{mu nu} B^P_{l s},
and applies the conventional algorithm of Table 1 / Eqs. (Jpq), (Pmat),
(Kpq) to it with an explicit O(N^5) transform:
  J^(q)_{mu nu} = sum_{l s} P^q_{l s} (mu nu|l s),  K^(q)_{mu s} = sum_{nu l} P^q_{nu l} (mu nu|s l),
  J_pq = sum_{mu nu} P^p_{mu nu} J^(q)_{mu nu},      K_pq = sum_{mu s} P^p_{mu s} K^(q)_{mu s},
with P^p_{mu nu} = C_{mu p} C_{nu p}.  Agreement with the factored RI path of
`ri` is the paper's own equivalence between Table 1 and Tables 2-3.
"""
from __future__ import annotations

import numpy as np


def fitted_eri4(B: np.ndarray) -> np.ndarray:
    nx, nb, _ = B.shape
    Bf = B.reshape(nx, nb * nb)
    return (Bf.T @ Bf).reshape(nb, nb, nb, nb)


def conventional_jk(eri: np.ndarray, C: np.ndarray, n_om: int):
    """Table 1 on a given AO four-index tensor; returns J, K, Jao, Kao."""
    nb = C.shape[0]
    Jao = np.zeros((n_om, nb, nb))
    Kao = np.zeros((n_om, nb, nb))
    for q in range(n_om):
        Pq = np.outer(C[:, q], C[:, q])                       # Eq. (Pmat)
        Jao[q] = np.einsum("ls,mnls->mn", Pq, eri)            # Table 1 step 2 (J)
        Kao[q] = np.einsum("nl,mnsl->ms", Pq, eri)            # Table 1 step 2 (K)
    J = np.zeros((n_om, n_om))
    K = np.zeros((n_om, n_om))
    for p in range(n_om):
        Pp = np.outer(C[:, p], C[:, p])
        for q in range(n_om):
            J[p, q] = np.sum(Pp * Jao[q])                     # Eq. (Jpq)
            K[p, q] = np.sum(Pp * Kao[q])                     # Eq. (Kpq)
    return J, K, Jao, Kao


def mo_eri4(eri: np.ndarray, C: np.ndarray) -> np.ndarray:
    """(pq|rs) = sum C_mp C_nq C_lr C_ss (mn|ls), one index at a time (O(N^5))."""
    t = np.einsum("mnls,mp->pnls", eri, C)
    t = np.einsum("pnls,nq->pqls", t, C)
    t = np.einsum("pqls,lr->pqrs", t, C)
    return np.einsum("pqrs,st->pqrt", t, C)
