"""PNOF7 occupations, energy and orthonormality Lagrangian (oracle, FP64).

Test infrastructure only; see the package docstring.

Energy, Eq. (PNOF) of Sec. 2 (singlet, real orbitals so L_pq = K_pq):
  E = 2 sum_p n_p H_pp + sum_qp Pi_qp K_pq + sum_qp (n_q n_p - Delta_qp)(2 J_pq - K_pq)
plus the nuclear repulsion.  The paper does not print PNOF7's Delta and Pi;
they are read from the PNOF7 functional it cites (PNOF7-2017):
  * Delta_qp = n_q n_p when p and q share a pairing subspace (p = q included),
    0 otherwise;
  * within a subspace: Pi_pp = n_p, and for p != q
    Pi_qp = -sqrt(n_q n_p) when one of them is the strong orbital,
    Pi_qp = +sqrt(n_q n_p) when both are weak;
  * across subspaces: Pi_qp = -Phi_q Phi_p with Phi_p = sqrt(n_p (1 - n_p)).
Only orbitals of the pairing space (Sec. 2, "electron-pairing constraints",
N_Omega <= N_b) carry occupation.

Occupations from the unconstrained angles gamma (the paper names the
gamma-variables of DoNOF but not their map; the DoNOF form is used): for
subspace g with strong orbital g and N_g weak orbitals,
  n_g = (1 + cos^2 gamma_g) / 2,   h_g = 1 - n_g,
  n_{g,i} = h_g alpha_i,  alpha_1 = cos^2 gamma_{g,1},
  alpha_i = prod_{j<i} sin^2 gamma_{g,j} cos^2 gamma_{g,i},
  alpha_{N_g} = prod_{j<N_g} sin^2 gamma_{g,j},
so sum over the subspace is 1 and 2 sum_p n_p = N.  gamma holds the N_I
strong angles, then N_g - 1 weak angles per subspace (subspace-major).

Lagrangian (Sec. 2, "Orbital Optimization with RI"; the paper defines lambda
through the orthonormality constraints without printing a formula): with
the symmetric coefficients A, B of E = E_nuc + 2 sum n_p H_pp
+ sum_pq (A_pq J_pq - B_pq K_pq),
  F^(p) = n_p H + sum_q (A_pq J^(q) - B_pq K^(q)),
  lambda_qp = C_q^T F^(p) C_p   (q over all orbitals, p in the pairing space;
                                 0 for p outside it),
so dE/dC_{mu p} = 4 (F^(p) C_p)_mu, dE/dkappa_qp = 4 (lambda_qp - lambda_pq)
for C -> C exp(kappa), and E = E_nuc + sum_p (n_p H_pp + lambda_pp).
"""
from __future__ import annotations

import numpy as np


def occupations(gamma: np.ndarray, n_strong: int, n_weak_per: int,
                subspace: np.ndarray, weak_rank: np.ndarray) -> np.ndarray:
    """n_p for the N_Omega pairing-space orbitals from the angles gamma."""
    n_om = n_strong * (1 + n_weak_per)
    n = np.zeros(n_om)
    gamma = np.asarray(gamma, dtype=np.float64)
    for g in range(n_strong):
        ng = 0.5 * (1.0 + np.cos(gamma[g]) ** 2)
        hg = 1.0 - ng
        wang = gamma[n_strong + g * (n_weak_per - 1): n_strong + (g + 1) * (n_weak_per - 1)]
        alpha = np.empty(n_weak_per)
        carry = 1.0
        for i in range(n_weak_per):
            if i < n_weak_per - 1:
                alpha[i] = carry * np.cos(wang[i]) ** 2
                carry *= np.sin(wang[i]) ** 2
            else:
                alpha[i] = carry
        for p in range(n_om):
            if subspace[p] != g:
                continue
            n[p] = ng if weak_rank[p] < 0 else hg * alpha[weak_rank[p]]
    return n


def delta_pi(n: np.ndarray, subspace: np.ndarray, weak_rank: np.ndarray):
    """PNOF7 Delta and Pi matrices over the pairing space (Eq. PNOF)."""
    m = n.shape[0]
    phi = np.sqrt(n * (1.0 - n))
    Delta = np.zeros((m, m))
    Pi = np.zeros((m, m))
    for q in range(m):
        for p in range(m):
            if subspace[p] == subspace[q]:
                Delta[q, p] = n[q] * n[p]
                if p == q:
                    Pi[q, p] = n[p]
                elif weak_rank[p] < 0 or weak_rank[q] < 0:
                    Pi[q, p] = -np.sqrt(n[q] * n[p])
                else:
                    Pi[q, p] = np.sqrt(n[q] * n[p])
            else:
                Pi[q, p] = -phi[q] * phi[p]
    return Delta, Pi


def energy_eq_pnof(n, Hmo_diag, J, K, Delta, Pi, e_nuc) -> float:
    """E = E_nuc + 2 sum n_p H_pp + sum Pi_qp K_pq + sum (n_q n_p - Delta_qp)(2J_pq - K_pq)."""
    m = n.shape[0]
    e = e_nuc + 2.0 * np.sum(n * Hmo_diag[:m])
    e += np.sum(Pi * K[:m, :m])
    e += np.sum((np.outer(n, n) - Delta) * (2.0 * J[:m, :m] - K[:m, :m]))
    return float(e)


def coupling(n: np.ndarray, subspace: np.ndarray, weak_rank: np.ndarray):
    """Symmetric A, B with E - E_nuc - 2 sum n H_pp = sum_pq (A_pq J_pq - B_pq K_pq).

    Obtained from Eq. (PNOF) with J_pp = K_pp folded into A:
      A_pp = n_p, B_pp = 0; same subspace p != q: A = 0, B = -Pi_pq;
      different subspaces: A = 2 n_p n_q, B = n_p n_q + Phi_p Phi_q.
    """
    Delta, Pi = delta_pi(n, subspace, weak_rank)
    m = n.shape[0]
    A = np.zeros((m, m))
    Bc = np.zeros((m, m))
    for p in range(m):
        for q in range(m):
            if p == q:
                A[p, q] = n[p]
            elif subspace[p] == subspace[q]:
                Bc[p, q] = -Pi[p, q]
            else:
                A[p, q] = 2.0 * (n[p] * n[q] - Delta[p, q])
                Bc[p, q] = (n[p] * n[q] - Delta[p, q]) - Pi[p, q]
    return A, Bc


def energy(n, Hmo_diag, J, K, A, Bc, e_nuc) -> float:
    """E = E_nuc + 2 sum_p n_p H_pp + sum_pq (A_pq J_pq - B_pq K_pq)."""
    m = n.shape[0]
    return float(e_nuc + 2.0 * np.sum(n * Hmo_diag[:m])
                 + np.sum(A * J[:m, :m]) - np.sum(Bc * K[:m, :m]))


def lagrangian(C, H, Jao, Kao, n, A, Bc) -> np.ndarray:
    """lambda_qp = C_q^T F^(p) C_p, F^(p) = n_p H + sum_q (A_pq J^(q) - B_pq K^(q)).

    Returns lambda [nbf, nbf] (column p; zero for p outside the pairing space).
    """
    nb = C.shape[0]
    m = n.shape[0]
    lam = np.zeros((nb, nb))
    for p in range(m):
        F = n[p] * H + np.einsum("q,qmn->mn", A[p], Jao) - np.einsum("q,qmn->mn", Bc[p], Kao)
        lam[:, p] = C.T @ (F @ C[:, p])
    return lam


def lagrangian_contracted(C, H, bh, d, bf, n, A, Bc) -> np.ndarray:
    """The same lambda without the per-orbital AO matrices (contracted form).

    With b^P_{p mu} (bh), b^P_pp (d) and b^P_qp (bf) of the RI transforms,
      J^(q) C_p = sum_P b^P_qq b^P_{p .},   K^(q) C_p = sum_P b^P_{q .} b^P_qp,
    so F^(p) C_p = n_p H C_p + sum_P w_pP b^P_{p .} - sum_P sum_q B_pq b^P_qp b^P_{q .}
    with w_pP = sum_q A_pq b^P_qq, and lambda_qp = C_q^T F^(p) C_p.
    """
    nb = C.shape[0]
    m = n.shape[0]
    w = A @ d.T                                             # w[p, P]
    YJ = np.einsum("pP,Ppm->mp", w, bh)                     # sum_P w_pP b^P_{p mu}
    YK = np.einsum("pq,Pqm,Pqp->mp", Bc, bh, bf)            # sum_P sum_q B_pq b^P_{q mu} b^P_qp
    Y = (H @ C[:, :m]) * n[None, :] + YJ - YK               # F^(p) C_p, columns p
    lam = np.zeros((nb, nb))
    lam[:, :m] = C.T @ Y
    return lam


def energy_from_lagrangian(lam, n, Hmo_diag, e_nuc) -> float:
    """E = E_nuc + sum_p (n_p H_pp + lambda_pp)."""
    m = n.shape[0]
    return float(e_nuc + np.sum(n * Hmo_diag[:m]) + np.trace(lam[:m, :m]))
