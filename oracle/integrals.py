"""Closed-form integrals over normalised s-type Gaussians (oracle, FP64).

Test infrastructure only; see the package docstring.

The paper evaluates (mu nu|k), (k|l) and four-centre ERIs once at the start
(Table 2 step 0, Table 3 step 0, Sec. 3).  The synthetic systems use s-type
Gaussians g_a(r) = N_a exp(-a |r-A|^2), with N_a = (2a/pi)^(3/4) for the
orbital basis and the Coulomb normalisation N_k = (2k/pi)^(3/4) sqrt(k/(4 pi))
(unit (k|k)) for the auxiliary basis, for which every integral has a textbook
closed form through the Boys function F0(T) = 1/2 sqrt(pi/T) erf(sqrt(T)).

With p = a + b, mu = ab/p, P = (aA + bB)/p and K_ab = exp(-mu |A-B|^2):
  S_ab      = N_a N_b (pi/p)^(3/2) K_ab
  T_ab      = N_a N_b mu (3 - 2 mu R_AB^2) (pi/p)^(3/2) K_ab
  V_ab      = -sum_C Z_C N_a N_b (2 pi/p) K_ab F0(p |P-C|^2)
  (ab|c)    = N_a N_b N_c 2 pi^(5/2) / (p c sqrt(p+c)) K_ab F0(pc/(p+c) |P-C|^2)
  (c|d)     = N_c N_d 2 pi^(5/2) / (c d sqrt(c+d)) F0(cd/(c+d) |C-D|^2)
  (ab|cd)   = N_a N_b N_c N_d 2 pi^(5/2) / (p q sqrt(p+q)) K_ab K_cd
              F0(pq/(p+q) |P-Q|^2)
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

PI = np.pi
TWO_PI_52 = 2.0 * PI ** 2.5


def boys_f0(t: np.ndarray) -> np.ndarray:
    """Boys function of order 0: F0(T) = int_0^1 exp(-T x^2) dx.

    F0(T) = 1/2 sqrt(pi/T) erf(sqrt(T)); below T = 1e-8 the Taylor series
    sum_k (-T)^k / (k! (2k+1)) truncated after three terms is used.
    """
    t = np.asarray(t, dtype=np.float64)
    out = np.empty_like(t)
    small = t < 1e-8
    ts = t[small]
    out[small] = 1.0 - ts / 3.0 + ts * ts / 10.0
    tl = t[~small]
    st = np.sqrt(tl)
    out[~small] = 0.5 * np.sqrt(PI / tl) * erf(st)
    return out


def norm_s(alpha: np.ndarray) -> np.ndarray:
    """L2 normalisation of an s Gaussian: (2 alpha / pi)^(3/4)."""
    return (2.0 * np.asarray(alpha) / PI) ** 0.75


def _centres(system, which: str):
    if which == "bf":
        return system.atom_xyz[system.bf_atom], system.bf_alpha
    return system.atom_xyz[system.aux_atom], system.aux_alpha


def _pair_data(system):
    """Gaussian-product data for all basis pairs (a, b): p, P, K_ab, N_a N_b."""
    X, al = _centres(system, "bf")
    a = al[:, None]
    b = al[None, :]
    p = a + b
    mu = a * b / p
    r2 = ((X[:, None, :] - X[None, :, :]) ** 2).sum(-1)
    kab = np.exp(-mu * r2)
    P = (a[..., None] * X[:, None, :] + b[..., None] * X[None, :, :]) / p[..., None]
    nn = norm_s(al)[:, None] * norm_s(al)[None, :]
    return p, mu, r2, kab, P, nn


def overlap(system) -> np.ndarray:
    """S_ab for the orbital basis, [nbf, nbf]."""
    p, mu, r2, kab, P, nn = _pair_data(system)
    return nn * (PI / p) ** 1.5 * kab


def kinetic(system) -> np.ndarray:
    """T_ab = <a| -1/2 nabla^2 |b>, [nbf, nbf]."""
    p, mu, r2, kab, P, nn = _pair_data(system)
    return nn * mu * (3.0 - 2.0 * mu * r2) * (PI / p) ** 1.5 * kab


def nuclear(system) -> np.ndarray:
    """V_ab = -sum_C Z_C <a| 1/|r-C| |b>, [nbf, nbf]."""
    p, mu, r2, kab, P, nn = _pair_data(system)
    v = np.zeros_like(p)
    for zc, c in zip(system.atom_charge, system.atom_xyz):
        rpc2 = ((P - c[None, None, :]) ** 2).sum(-1)
        v -= zc * nn * (2.0 * PI / p) * kab * boys_f0(p * rpc2)
    return v


def core_hamiltonian(system) -> np.ndarray:
    """H = T + V (the paper's one-electron matrix elements H_pp in AO form)."""
    return kinetic(system) + nuclear(system)


def nuclear_repulsion(system) -> float:
    """E_nuc = sum_{A<B} Z_A Z_B / R_AB."""
    e = 0.0
    xyz, z = system.atom_xyz, system.atom_charge
    for i in range(len(z)):
        for j in range(i):
            e += z[i] * z[j] / np.linalg.norm(xyz[i] - xyz[j])
    return float(e)


def norm_aux(alpha: np.ndarray) -> np.ndarray:
    """Coulomb normalisation of an auxiliary s Gaussian, so that (k|k) = 1.

    The L2-normalised function has (k|k) = 4 pi / alpha; scaling by
    sqrt(alpha / (4 pi)) gives unit self-repulsion.  Every RI result is
    invariant to the scaling of the auxiliary functions (it cancels between
    (mu nu|k) and G^-1); unit diagonal keeps the metric's pivots comparable.
    """
    alpha = np.asarray(alpha)
    return norm_s(alpha) * np.sqrt(alpha / (4.0 * PI))


def metric(system) -> np.ndarray:
    """Two-centre Coulomb metric G_kl = (k|l), [naux, naux]."""
    X, c = _centres(system, "aux")
    ci = c[:, None]
    cj = c[None, :]
    r2 = ((X[:, None, :] - X[None, :, :]) ** 2).sum(-1)
    nn = norm_aux(c)[:, None] * norm_aux(c)[None, :]
    return nn * TWO_PI_52 / (ci * cj * np.sqrt(ci + cj)) * boys_f0(ci * cj / (ci + cj) * r2)


def eri3(system, aux_slice: slice | None = None) -> np.ndarray:
    """Three-centre integrals (k|mu nu), [naux(slice), nbf, nbf]."""
    p, mu, r2, kab, P, nn = _pair_data(system)
    Xc, c = _centres(system, "aux")
    if aux_slice is not None:
        Xc, c = Xc[aux_slice], c[aux_slice]
    nc = norm_aux(c)
    out = np.empty((c.shape[0],) + p.shape)
    for k in range(c.shape[0]):
        ck = c[k]
        rpc2 = ((P - Xc[k][None, None, :]) ** 2).sum(-1)
        out[k] = (nn * nc[k] * TWO_PI_52 / (p * ck * np.sqrt(p + ck)) * kab
                  * boys_f0(p * ck / (p + ck) * rpc2))
    return out


def eri4(system) -> np.ndarray:
    """Exact four-centre ERIs (ab|cd), [nbf]*4 (small systems only)."""
    p, mu, r2, kab, P, nn = _pair_data(system)
    n = p.shape[0]
    pf = p.reshape(-1)
    kf = (kab * nn).reshape(-1)
    Pf = P.reshape(-1, 3)
    pi_ = pf[:, None]
    qj = pf[None, :]
    rpq2 = ((Pf[:, None, :] - Pf[None, :, :]) ** 2).sum(-1)
    val = (TWO_PI_52 / (pi_ * qj * np.sqrt(pi_ + qj)) * kf[:, None] * kf[None, :]
           * boys_f0(pi_ * qj / (pi_ + qj) * rpq2))
    return val.reshape(n, n, n, n)
