"""Resolution-of-the-identity J/K algebra of the paper (oracle, FP64).

Test infrastructure only; see the package docstring.

Each function is the plain definition of one step of Sec. 2 ("Occupancy
Optimization with RI" and "Orbital Optimization with RI"), written with
numpy library primitives and no blocking or fusion:

  Eq. (AOERI)        (mu nu|s l) = sum_kl (mu nu|k) G^-1_kl (l|s l)
  metric factor      G = L L^T (plain Cholesky), B^P = sum_Q (L^-1)_PQ (Q|mu nu)
                     (the paper solves P L D^1/2 b^T = (mu nu|k); with a
                     positive-definite G and no pivoting this is the same b
                     up to an orthogonal rotation of the P index, to which
                     every J/K result is invariant)
  Table 2/3 step 2   b^P_{p nu} = sum_mu C_{mu p} B^P_{mu nu}         (half)
  Table 3 step 3     b^P_{pp}   = sum_nu C_{nu p} b^P_{p nu}          (diagonal)
  Table 2 step 3     b^P_{pq}   = sum_nu C_{nu q} b^P_{p nu}          (full)
  Table 2 step 4     J_pq = sum_P b^P_pp b^P_qq,  K_pq = sum_P (b^P_pq)^2
  Table 3 step 4     J^(q)_{mu nu} = sum_P b^P_qq B^P_{mu nu}
  Table 3 step 3 (K) K^(q)_{mu nu} = sum_P b^P_{q mu} b^P_{q nu}

Array conventions (numpy, row-major):
  B   [naux, nbf, nbf]       B[P, mu, nu]
  C   [nbf, nbf]             C[mu, p] (column p is orbital p)
  bh  [naux, n_om, nbf]      bh[P, p, nu] = b^P_{p nu}
  d   [naux, n_om]           d[P, p] = b^P_pp
  bf  [naux, n_om, n_om]     bf[P, p, q] = b^P_pq
  Jao [n_om, nbf, nbf]       Jao[q] = J^(q);  Kao likewise
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import solve_triangular


class MetricNotPositiveDefinite(ValueError):
    pass


def metric_cholesky(G: np.ndarray, rel_pivot_min: float = 1e-14) -> np.ndarray:
    """Lower Cholesky factor L of the Coulomb metric, G = L L^T.

    Raises MetricNotPositiveDefinite when a pivot falls below
    rel_pivot_min * max(diag(G)) (the plain factorisation the engine uses in
    place of the paper's modified LDL^T of Sec. 2).
    """
    try:
        L = np.linalg.cholesky(G)
    except np.linalg.LinAlgError as exc:
        raise MetricNotPositiveDefinite(str(exc)) from exc
    piv = np.diag(L) ** 2
    if piv.min() < rel_pivot_min * np.max(np.diag(G)):
        raise MetricNotPositiveDefinite(f"pivot {piv.min():.3e} below threshold")
    return L


def fitted_tensor(eri3: np.ndarray, L: np.ndarray) -> np.ndarray:
    """B^P_{mu nu} = sum_Q (L^-1)_{PQ} (Q|mu nu) by a forward triangular solve."""
    nx, nb, _ = eri3.shape
    X = solve_triangular(L, eri3.reshape(nx, nb * nb), lower=True)
    return X.reshape(nx, nb, nb)


def fitted_tensor_symmetric(eri3: np.ndarray, G: np.ndarray) -> np.ndarray:
    """B'^P = sum_Q (G^-1/2)_{PQ} (Q|mu nu): the symmetric approach of Sec. 2."""
    w, V = np.linalg.eigh(G)
    Ginvh = (V / np.sqrt(w)[None, :]) @ V.T
    nx, nb, _ = eri3.shape
    return (Ginvh @ eri3.reshape(nx, nb * nb)).reshape(nx, nb, nb)


def half_transform(B: np.ndarray, C: np.ndarray, n_om: int) -> np.ndarray:
    """b^P_{p nu} = sum_mu C_{mu p} B^P_{mu nu} for p < n_om; returns bh[P, p, nu]."""
    Ct = C[:, :n_om].T                      # [p, mu]
    return np.einsum("pm,Pmn->Ppn", Ct, B, optimize=True)


def diagonal(bh: np.ndarray, C: np.ndarray) -> np.ndarray:
    """b^P_pp = sum_nu C_{nu p} b^P_{p nu}; returns d[P, p]."""
    n_om = bh.shape[1]
    return np.einsum("Ppn,np->Pp", bh, C[:, :n_om], optimize=True)


def full_transform(bh: np.ndarray, C: np.ndarray) -> np.ndarray:
    """b^P_pq = sum_nu C_{nu q} b^P_{p nu}; returns bf[P, p, q]."""
    n_om = bh.shape[1]
    return np.einsum("Ppn,nq->Ppq", bh, C[:, :n_om], optimize=True)


def jk_mo(bf: np.ndarray, d: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """J_pq = sum_P b^P_pp b^P_qq and K_pq = sum_P (b^P_pq)^2."""
    J = d.T @ d
    K = np.einsum("Ppq,Ppq->pq", bf, bf, optimize=True)
    return J, K


def jk_ao(B: np.ndarray, bh: np.ndarray, d: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Per-orbital AO matrices J^(q) = sum_P b^P_qq B^P and
    K^(q)_{mu nu} = sum_P b^P_{q mu} b^P_{q nu}; returns (Jao, Kao)."""
    nx, nb, _ = B.shape
    Jao = (d.T @ B.reshape(nx, nb * nb)).reshape(-1, nb, nb)
    Xq = np.ascontiguousarray(bh.transpose(1, 2, 0))      # [q, mu, P] = b^P_{q mu}
    Kao = np.matmul(Xq, Xq.transpose(0, 2, 1))           # K^(q) = X_q X_q^T
    return Jao, Kao


def setup(system, eri3=None, G=None):
    """Integrals -> Cholesky -> B for a system; returns (B, L, G)."""
    from . import integrals
    if G is None:
        G = integrals.metric(system)
    if eri3 is None:
        eri3 = integrals.eri3(system)
    L = metric_cholesky(G)
    return fitted_tensor(eri3, L), L, G


def all_rows(B: np.ndarray, C: np.ndarray, n_om: int) -> dict:
    """Every J/K row of the hot path for one orbital matrix."""
    bh = half_transform(B, C, n_om)
    d = diagonal(bh, C)
    bf = full_transform(bh, C)
    J, K = jk_mo(bf, d)
    Jao, Kao = jk_ao(B, bh, d)
    return dict(bh=bh, d=d, bf=bf, J=J, K=K, Jao=Jao, Kao=Kao)
