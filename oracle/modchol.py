"""Modified Cholesky factorisation of the Coulomb metric (oracle, FP64).

Test infrastructure only; see the package docstring.

Sec. 2, "Occupancy Optimization with RI": the metric G_kl = (k|l) may be
numerically ill conditioned, so the paper factorises it as
    G = P L D L^T P^T
with P a permutation, L unit lower triangular and D block diagonal with 1x1
and 2x2 blocks (Bunch and Kaufman's symmetric pivoting), corrects the
eigenvalues of each block of D that are negative or too small (Cheng and
Higham), giving D~, and obtains the fitted tensor from
    P L D~^(1/2) b^T = (mu nu|k),
with D~^(1/2) the symmetric square root of each block.

Readings (the paper gives neither constant):
  * pivoting: Bunch-Kaufman partial pivoting with alpha = (1 + sqrt 17) / 8,
    columns taken left to right, as in LAPACK's symmetric-indefinite
    factorisation (pinned against scipy.linalg.ldl in the tests);
  * correction: every eigenvalue of a D block below delta = tol * max_k G_kk
    is replaced by delta; tol is the caller's.  With a positive-definite G
    whose blocks all stay above delta nothing changes, and b is the plain
    Cholesky fit up to an orthogonal rotation of the auxiliary index.

Written with numpy primitives (outer products, 2x2 inverses, eigh of a 2x2
block, a unit-triangular solve), in the order of the algorithm.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import solve_triangular

ALPHA = (1.0 + np.sqrt(17.0)) / 8.0


def bunch_kaufman(G: np.ndarray):
    """P^T G P = L D L^T by Bunch-Kaufman partial pivoting.

    Returns (perm, L, starts, sizes, D, nswap): G[perm][:, perm] = L D L^T, L unit
    lower triangular, D block diagonal with blocks of size 1 or 2 starting at
    `starts`; nswap counts the symmetric interchanges."""
    A = np.array(G, dtype=np.float64, copy=True)
    n = A.shape[0]
    perm = np.arange(n)
    L = np.eye(n)
    D = np.zeros((n, n))
    starts, sizes = [], []

    nswap = [0]

    def interchange(i, j, k):
        # symmetric interchange of indices i, j >= k in A; rows of the finished part of L
        if i == j:
            return
        nswap[0] += 1
        A[[i, j], :] = A[[j, i], :]
        A[:, [i, j]] = A[:, [j, i]]
        L[[i, j], :k] = L[[j, i], :k]
        perm[[i, j]] = perm[[j, i]]

    k = 0
    while k < n:
        akk = abs(A[k, k])
        if k + 1 < n:
            col = np.abs(A[k + 1:, k])
            imax = k + 1 + int(np.argmax(col))
            colmax = col[imax - k - 1]
        else:
            imax, colmax = k, 0.0
        size, piv = 1, k
        if max(akk, colmax) == 0.0 or akk >= ALPHA * colmax:
            size, piv = 1, k
        else:
            # largest off-diagonal element of row / column imax in the active matrix
            rowvals = np.concatenate([np.abs(A[imax, k:imax]), np.abs(A[imax + 1:, imax])])
            rowmax = rowvals.max()
            if akk * rowmax >= ALPHA * colmax * colmax:
                size, piv = 1, k
            elif abs(A[imax, imax]) >= ALPHA * rowmax:
                size, piv = 1, imax
            else:
                size, piv = 2, imax
        if size == 1:
            interchange(k, piv, k)
            d = A[k, k]
            D[k, k] = d
            if d != 0.0 and k + 1 < n:
                a = A[k + 1:, k].copy()
                l = a / d
                A[k + 1:, k + 1:] -= np.outer(l, a)
                L[k + 1:, k] = l
        else:
            interchange(k + 1, piv, k)
            E = A[k:k + 2, k:k + 2].copy()
            D[k:k + 2, k:k + 2] = E
            if k + 2 < n:
                Cb = A[k + 2:, k:k + 2].copy()
                Lb = Cb @ np.linalg.inv(E)
                A[k + 2:, k + 2:] -= Lb @ Cb.T
                L[k + 2:, k:k + 2] = Lb
        starts.append(k)
        sizes.append(size)
        k += size
    return perm, L, np.array(starts), np.array(sizes), D, nswap[0]


def corrected_blocks(D: np.ndarray, starts, sizes, delta: float):
    """Cheng-Higham: per block, eigenvalues below delta raised to delta.
    Returns (D~, D~^(-1/2), number of eigenvalues raised)."""
    n = D.shape[0]
    Dt = np.zeros((n, n))
    Dmh = np.zeros((n, n))
    raised = 0
    for k, s in zip(starts, sizes):
        blk = D[k:k + s, k:k + s]
        lam, Q = np.linalg.eigh(blk)
        raised += int(np.sum(lam < delta))
        lam = np.maximum(lam, delta)
        Dt[k:k + s, k:k + s] = (Q * lam) @ Q.T
        Dmh[k:k + s, k:k + s] = (Q / np.sqrt(lam)) @ Q.T
    return Dt, Dmh, raised


def fitted_tensor_modified(eri3: np.ndarray, G: np.ndarray, tol: float):
    """b from P L D~^(1/2) b^T = (mu nu|k); returns (B [naux, nbf, nbf], factors dict)."""
    nx, nb, _ = eri3.shape
    perm, L, starts, sizes, D, nswap = bunch_kaufman(G)
    delta = tol * float(np.max(np.diag(G)))
    Dt, Dmh, raised = corrected_blocks(D, starts, sizes, delta)
    X = eri3.reshape(nx, nb * nb)[perm]                    # P^T (mu nu|k)
    Z = solve_triangular(L, X, lower=True, unit_diagonal=True)
    B = (Dmh @ Z).reshape(nx, nb, nb)
    return B, dict(perm=perm, L=L, D=D, Dt=Dt, starts=starts, sizes=sizes, raised=raised, delta=delta,
                   nswap=nswap)


def corrected_metric(f: dict) -> np.ndarray:
    """G~ = P L D~ L^T P^T, the matrix whose inverse the corrected fit applies."""
    n = f["L"].shape[0]
    M = f["L"] @ f["Dt"] @ f["L"].T
    Gt = np.empty((n, n))
    Gt[np.ix_(f["perm"], f["perm"])] = M
    return Gt
