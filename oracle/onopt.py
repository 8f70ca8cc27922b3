"""Occupation (gamma) optimisation for fixed orbitals (oracle, FP64).

Test infrastructure only; see the package docstring.

Sec. 2, "Occupancy Optimization with RI": for fixed orbitals J and K are
computed once, and the energy is minimised over the auxiliary variables gamma
that parametrise the occupations (the constrained problem in n becomes an
unconstrained one in gamma).  The paper names neither the optimiser nor the
gradient; this module writes out the gradient of Eq. (PNOF) by the chain rule,
  dE/dgamma_k = sum_p (dE/dn_p) (dn_p/dgamma_k),
and minimises with scipy's L-BFGS (a library routine standing for "an
unconstrained minimiser").  The guess is the standard one described with the
paper's calculations (Sec. 4: gamma^0 from a Fermi-Dirac-like distribution of
occupations); its reading here: every strong orbital at n = 0.98 and the weak
share of each subspace split equally over its weak orbitals.

Notation as in pnof7.py: subspace g has strong orbital g (n_g = (1 + cos^2
gamma_g)/2) and N_g weak orbitals with n_{g,i} = (1 - n_g) alpha_i, alpha from
the N_g - 1 weak angles w_{g,j} of the subspace.
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import minimize

from . import pnof7


def energy_dn(n, Hmo_diag, J, K, subspace, weak_rank):
    """dE/dn_p of E(n) = E_nuc + 2 sum n_p H_pp + sum_pq (A_pq(n) J_pq - B_pq(n) K_pq)
    for symmetric J, K, with A, B the PNOF7 coupling of pnof7.coupling:
      2 H_pp + J_pp
      - sum_{q in g(p), q != p} s_pq K_pq sqrt(n_q / n_p)       (s = +1 if p or q strong, -1 otherwise)
      + sum_{q not in g(p)} (4 n_q J_pq - 2 n_q K_pq - 2 Phi'_p Phi_q K_pq),
    Phi = sqrt(n (1 - n)), Phi' = (1 - 2 n) / (2 Phi)."""
    m = n.shape[0]
    phi = np.sqrt(n * (1.0 - n))
    # At n_p = 0 or 1 the sqrt terms have infinite slope (E is not differentiable
    # in n there); those terms are taken as 0, which is what the chain rule gives
    # wherever dn_p/dgamma vanishes with them.
    with np.errstate(divide="ignore", invalid="ignore"):
        dphi = np.where(phi > 0, (1.0 - 2.0 * n) / (2.0 * phi), 0.0)
    g = np.zeros(m)
    for p in range(m):
        v = 2.0 * Hmo_diag[p] + J[p, p]
        for q in range(m):
            if q == p:
                continue
            if subspace[q] == subspace[p]:
                s = 1.0 if (weak_rank[p] < 0 or weak_rank[q] < 0) else -1.0
                if n[p] > 0.0:
                    v -= s * K[p, q] * np.sqrt(n[q] / n[p])
            else:
                v += 4.0 * n[q] * J[p, q] - 2.0 * n[q] * K[p, q] - 2.0 * dphi[p] * phi[q] * K[p, q]
        g[p] = v
    return g


def occupations_jacobian(gamma, n_strong, n_weak_per, subspace, weak_rank):
    """dn_p/dgamma_k [N_Omega, N_I N_g] of the map in pnof7.occupations."""
    gamma = np.asarray(gamma, dtype=np.float64)
    n_om = n_strong * (1 + n_weak_per)
    ng_ang = n_weak_per - 1
    D = np.zeros((n_om, gamma.shape[0]))
    for g in range(n_strong):
        cg = np.cos(gamma[g]) ** 2
        hg = 1.0 - 0.5 * (1.0 + cg)
        dh = 0.5 * np.sin(2.0 * gamma[g])          # d h_g / d gamma_g
        w = gamma[n_strong + g * ng_ang: n_strong + (g + 1) * ng_ang]
        # alpha_i and d alpha_i / d w_j
        alpha = np.empty(n_weak_per)
        dalpha = np.zeros((n_weak_per, ng_ang))
        for i in range(n_weak_per):
            tail = np.cos(w[i]) ** 2 if i < ng_ang else 1.0
            prod = np.prod(np.sin(w[:i]) ** 2) if i > 0 else 1.0
            alpha[i] = prod * tail
            for j in range(min(i, ng_ang)):
                others = np.prod([np.sin(w[k]) ** 2 for k in range(i) if k != j]) if i > 1 else 1.0
                dalpha[i, j] = others * np.sin(2.0 * w[j]) * tail
            if i < ng_ang:
                dalpha[i, i] = -prod * np.sin(2.0 * w[i])
        for p in range(n_om):
            if subspace[p] != g:
                continue
            if weak_rank[p] < 0:
                D[p, g] = -dh
            else:
                i = weak_rank[p]
                D[p, g] = dh * alpha[i]
                for j in range(ng_ang):
                    D[p, n_strong + g * ng_ang + j] = hg * dalpha[i, j]
    return D


def energy_and_gradient(gamma, n_strong, n_weak_per, subspace, weak_rank, Hmo_diag, J, K, e_nuc):
    """E(gamma) and dE/dgamma (chain rule through the occupations)."""
    n = pnof7.occupations(gamma, n_strong, n_weak_per, subspace, weak_rank)
    A, Bc = pnof7.coupling(n, subspace, weak_rank)
    E = pnof7.energy(n, Hmo_diag, J, K, A, Bc, e_nuc)
    dEdn = energy_dn(n, Hmo_diag, J, K, subspace, weak_rank)
    D = occupations_jacobian(gamma, n_strong, n_weak_per, subspace, weak_rank)
    return E, D.T @ dEdn


def standard_guess(n_strong, n_weak_per, n_strong_occ=0.98):
    """gamma^0: strong n = n_strong_occ, the weak share split equally (cos^2 w_i = 1/(N_g - i))."""
    g0 = np.arccos(np.sqrt(2.0 * n_strong_occ - 1.0))
    w = [np.arccos(np.sqrt(1.0 / (n_weak_per - i))) for i in range(n_weak_per - 1)]
    return np.concatenate([np.full(n_strong, g0), np.tile(np.array(w, dtype=np.float64), n_strong)])


def optimize(gamma0, n_strong, n_weak_per, subspace, weak_rank, Hmo_diag, J, K, e_nuc,
             gtol=1e-8, maxiter=2000):
    """Minimise E over gamma from gamma0; returns (gamma, E, n, iterations, max|grad|)."""
    def f(x):
        E, g = energy_and_gradient(x, n_strong, n_weak_per, subspace, weak_rank, Hmo_diag, J, K, e_nuc)
        return E, g
    res = minimize(f, np.asarray(gamma0, dtype=np.float64), jac=True, method="L-BFGS-B",
                   options={"gtol": gtol, "ftol": 1e-15, "maxiter": maxiter, "maxcor": 8})
    E, g = f(res.x)
    n = pnof7.occupations(res.x, n_strong, n_weak_per, subspace, weak_rank)
    return res.x, E, n, int(res.nit), float(np.abs(g).max())
