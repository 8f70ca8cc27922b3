"""Orbital optimisation for fixed occupations (oracle, FP64).

Test infrastructure only; see the package docstring.

Sec. 2, "Orbital Optimization with RI": the energy is minimised over real
orthonormal orbitals at fixed occupations, with J^(q), K^(q) recomputed at every
inner iteration and the Lagrangian lambda driving the step.  The paper's own
step, the iterative diagonalisation of a symmetric matrix F^lambda built from
lambda (flambda_matrix, flambda_step), is stated here with the plain driver:
the orbitals rotate as C -> C expm(kappa) with kappa a steepest-descent step on
the rotation gradient
  dE/dkappa_qp = 4 (lambda_qp - lambda_pq)          (pinned in test_oracle_pnof7)
of length controlled by a trust radius: kappa = -r G / max|G|, G = lambda -
lambda^T; a step that raises E is rejected and halves r, an accepted one grows r
by 1.5 (up to r_max).
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import expm

from . import integrals as I, pnof7, ri


def rotation_step(C: np.ndarray, lam: np.ndarray, radius: float) -> np.ndarray:
    """C expm(kappa) with kappa = -radius (lam - lam^T) / max|lam - lam^T|."""
    G = lam - lam.T
    gmax = np.abs(G).max()
    if gmax == 0.0:
        return C.copy()
    return C @ expm(-radius * G / gmax)


def flambda_matrix(lam: np.ndarray, diag: np.ndarray, bound: float) -> np.ndarray:
    """The symmetric matrix F^lambda of the iterative-diagonalisation step.

    Off-diagonal F_qp = lambda_qp - lambda_pq for q > p, mirrored (the orbital
    gradient, which vanishes at a stationary point); every off-diagonal element
    larger than `bound` in magnitude is scaled by the smallest power of 1/10 that
    brings it to `bound` or below (the paper gives no scaling rule; DoNOF damps the
    large elements this way); the diagonal is `diag` (the aufbau ordering: the
    previous step's eigenvalues, lambda_pp at the first step).
    """
    G = lam - lam.T
    F = np.tril(G, -1)
    F = F + F.T
    a = np.abs(F)
    k = np.where(a > bound, np.ceil(np.log10(np.maximum(a, 1e-300) / bound)), 0.0)
    F = F * 10.0 ** (-k)
    F[np.diag_indices_from(F)] = diag
    return F


def flambda_step(C: np.ndarray, lam: np.ndarray, diag: np.ndarray, bound: float):
    """One step of the paper's orbital optimisation (Sec. 2, "Orbital Optimization
    with RI"): diagonalise F^lambda and rotate the orbitals onto its eigenvectors,
    taken in increasing order of eigenvalue (aufbau).  Returns (C U, eigenvalues)."""
    eps, U = np.linalg.eigh(flambda_matrix(lam, diag, bound))
    return C @ U, eps


def energy_lambda(system, B, H, e_nuc, C, gamma, subspace, weak_rank):
    """(E, lambda) of Eq. (PNOF) and the Lagrangian at orbitals C and angles gamma."""
    m = system.n_omega
    r = ri.all_rows(B, C, m)
    n = pnof7.occupations(gamma, system.n_strong, system.n_weak_per, subspace, weak_rank)
    A, Bc = pnof7.coupling(n, subspace, weak_rank)
    lam = pnof7.lagrangian(C, H, r["Jao"], r["Kao"], n, A, Bc)
    Hd = np.einsum("mp,mn,np->p", C[:, :m], H, C[:, :m])
    return pnof7.energy_from_lagrangian(lam, n, Hd, e_nuc), lam


def optimize(system, C0, gamma, subspace, weak_rank, max_iter=500, gtol=1e-6, radius=0.05, r_max=0.3):
    """Trust-radius steepest descent on the orbitals; returns (C, E, max|lam - lam^T|, iterations)."""
    B, L, G = ri.setup(system)
    H = I.core_hamiltonian(system)
    e_nuc = I.nuclear_repulsion(system)
    C = C0.copy()
    E, lam = energy_lambda(system, B, H, e_nuc, C, gamma, subspace, weak_rank)
    it = 0
    for it in range(1, max_iter + 1):
        g = np.abs(lam - lam.T).max()
        if g <= gtol:
            break
        Cn = rotation_step(C, lam, radius)
        En, lamn = energy_lambda(system, B, H, e_nuc, Cn, gamma, subspace, weak_rank)
        if En < E:
            C, E, lam = Cn, En, lamn
            radius = min(1.5 * radius, r_max)
        else:
            radius *= 0.5
    return C, E, float(np.abs(lam - lam.T).max()), it


# ---------------------------------------------------------------------------
# The paper's outer / inner scheme to convergence (Sec. 2, Fig. 1: occupations for
# fixed orbitals, then orbitals for fixed occupations, repeated), with the F^lambda
# step for the orbitals.  Readings (the paper gives the step, not its controls):
# the aufbau diagonal of the first step is the starting orbitals' energies (the
# Hartree-Fock eigenvalues), later ones the previous step's eigenvalues, every gap
# of the ascending diagonal raised to at least `gapmin` (orbitals degenerate in
# energy but in different pairing subspaces would otherwise be mixed by 45
# degrees); the damping bound starts at 0.1 max|lambda - lambda^T| of each inner
# loop, grows by 1.5 (to at most 1) after an accepted step and halves after a
# rejected one; an inner loop ends when max|lambda - lambda^T| <= gtol, when a step
# lowers E by at most 1e-10 |E|, or after max_inner steps; the scheme has converged
# when an outer iteration changes E by less than etol with max|lambda - lambda^T|
# <= gtol.
# ---------------------------------------------------------------------------
def exact_rows(eri: np.ndarray, C: np.ndarray, n_om: int) -> dict:
    """J, K, J^(q), K^(q) from four-index integrals (mu nu|l s) (the conventional route)."""
    Cm = C[:, :n_om]
    Jao = np.einsum("mnls,lq,sq->qmn", eri, Cm, Cm, optimize=True)
    Kao = np.einsum("mlns,lq,sq->qmn", eri, Cm, Cm, optimize=True)
    J = np.einsum("qmn,mp,np->pq", Jao, Cm, Cm, optimize=True)
    K = np.einsum("qmn,mp,np->pq", Kao, Cm, Cm, optimize=True)
    return dict(J=J, K=K, Jao=Jao, Kao=Kao)


def _gap_floor(d: np.ndarray, gapmin: float) -> np.ndarray:
    out = d.copy()
    for k in range(1, out.size):
        out[k] = max(out[k], out[k - 1] + gapmin)
    return out


def converge(system, C0, gamma0, diag0, subspace, weak_rank, B=None, eri=None, etol=1e-6, gtol=1e-4,
             max_outer=60, max_inner=100, gapmin=0.01):
    """Outer / inner iterations from (C0, gamma0) with the F^lambda step, on RI integrals
    (B) or, when eri is given, on exact four-index integrals.  Returns dict(C, gamma,
    diag, E, outer, inner_total, converged, history)."""
    from . import onopt
    m = system.n_omega
    H = I.core_hamiltonian(system)
    e_nuc = I.nuclear_repulsion(system)

    def rows(C):
        return exact_rows(eri, C, m) if eri is not None else ri.all_rows(B, C, m)

    def energy_lam(C, g):
        r = rows(C)
        n = pnof7.occupations(g, system.n_strong, system.n_weak_per, subspace, weak_rank)
        A, Bc = pnof7.coupling(n, subspace, weak_rank)
        lam = pnof7.lagrangian(C, H, r["Jao"], r["Kao"], n, A, Bc)
        Hd = np.einsum("mp,mn,np->p", C[:, :m], H, C[:, :m])
        return pnof7.energy_from_lagrangian(lam, n, Hd, e_nuc), lam

    C, g, diag = C0.copy(), np.array(gamma0, dtype=np.float64), np.array(diag0, dtype=np.float64)
    hist, E_prev, total, converged = [], None, 0, False
    for outer in range(1, max_outer + 1):
        r = rows(C)
        Hd = np.einsum("mp,mn,np->p", C[:, :m], H, C[:, :m])
        g, E_on = onopt.optimize(g, system.n_strong, system.n_weak_per, subspace, weak_rank, Hd, r["J"], r["K"],
                                 e_nuc, gtol=1e-8)[:2]
        E, lam = energy_lam(C, g)
        bound = 0.1 * max(np.abs(lam - lam.T).max(), 1e-12)
        inner = 0
        for inner in range(1, max_inner + 1):
            if np.abs(lam - lam.T).max() <= gtol:
                inner -= 1
                break
            Cn, eps = flambda_step(C, lam, _gap_floor(diag, gapmin), bound)
            En, lamn = energy_lam(Cn, g)
            if En < E:
                dec = E - En
                C, E, lam, diag = Cn, En, lamn, eps
                bound = min(1.5 * bound, 1.0)
                if dec <= 1e-10 * abs(E):
                    break
            else:
                bound *= 0.5
        total += inner
        gm = float(np.abs(lam - lam.T).max())
        hist.append(dict(outer=outer, E_occ=E_on, E=E, inner=inner, gmax=gm))
        if E_prev is not None and abs(E - E_prev) < etol and gm <= gtol:
            converged = True
            break
        E_prev = E
    return dict(C=C, gamma=g, diag=diag, E=hist[-1]["E"], outer=len(hist), inner_total=total,
                converged=converged, history=hist)
