"""Pins of the oracle's s-type Gaussian integrals against independent routes.

* Boys F0 against direct quadrature of its defining integral.
* Normalisation: S_aa = 1 and (k|k) = 1 for the Coulomb-normalised aux set.
* Coulomb integrals against the classical electrostatics of two spherical
  Gaussian charge clouds, E = Q1 Q2 erf(sqrt(w) R) / R, w = a1 a2/(a1+a2):
  a different algebraic route from the Boys-function formulas.
* Kinetic integrals against 1-D quadrature of the separable Laplacian.
* Textbook values: H2 / STO-3G integrals printed in Szabo & Ostlund.
"""
import json
import os

import numpy as np
import pytest
from scipy.integrate import quad
from scipy.special import erf

from oracle import integrals as I
from synthetic.systems import System
from tests.workloads import make_workload

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _toy_system(xyz, z, bf_atom, bf_alpha, aux_atom=None, aux_alpha=None):
    if aux_atom is None:
        aux_atom, aux_alpha = [0], [1.0]
    return System(name="toy", atom_xyz=np.asarray(xyz, float), atom_charge=np.asarray(z, float),
                  bf_atom=np.asarray(bf_atom, np.int32), bf_alpha=np.asarray(bf_alpha, float),
                  aux_atom=np.asarray(aux_atom, np.int32), aux_alpha=np.asarray(aux_alpha, float),
                  n_strong=1, n_weak_per=1)


def _electrostatic(q1, q2, w, r):
    r = np.asarray(r, float)
    out = np.where(r > 1e-12, q1 * q2 * erf(np.sqrt(w) * np.maximum(r, 1e-300)) / np.maximum(r, 1e-300),
                   q1 * q2 * 2.0 * np.sqrt(w / np.pi))
    return out


def test_boys_f0_against_quadrature():
    for t in [0.0, 1e-12, 1e-9, 1e-7, 1e-3, 0.1, 1.0, 7.5, 30.0, 200.0]:
        ref = quad(lambda x: np.exp(-t * x * x), 0.0, 1.0, epsabs=1e-15, epsrel=1e-14)[0]
        got = I.boys_f0(np.array([t]))[0]
        assert abs(got - ref) < 1e-14, (t, got, ref)


def test_normalisation():
    w = make_workload("square4")
    S = I.overlap(w.system)
    np.testing.assert_allclose(np.diag(S), 1.0, atol=1e-14)
    G = I.metric(w.system)
    np.testing.assert_allclose(np.diag(G), 1.0, atol=1e-13)


def test_symmetries():
    s = make_workload("square4").system
    for M in (I.overlap(s), I.kinetic(s), I.nuclear(s), I.metric(s)):
        np.testing.assert_allclose(M, M.T, atol=1e-14)
    e3 = I.eri3(s)
    np.testing.assert_allclose(e3, e3.transpose(0, 2, 1), atol=1e-14)


def test_coulomb_integrals_against_electrostatics():
    rng = np.random.default_rng(7)
    xyz = rng.uniform(-1.5, 1.5, size=(3, 3))
    s = _toy_system(xyz, [1, 2, 3], [0, 1, 2, 0], [0.3, 1.7, 0.8, 5.0],
                    aux_atom=[0, 1, 2, 2], aux_alpha=[0.4, 2.5, 0.9, 11.0])
    X = s.atom_xyz[s.bf_atom]
    a = s.bf_alpha
    Xk = s.atom_xyz[s.aux_atom]
    k = s.aux_alpha
    Nk = I.norm_aux(k)
    Qk = Nk * (np.pi / k) ** 1.5
    G = I.metric(s)
    for i in range(4):
        for j in range(4):
            w = k[i] * k[j] / (k[i] + k[j])
            ref = _electrostatic(Qk[i], Qk[j], w, np.linalg.norm(Xk[i] - Xk[j]))
            assert abs(G[i, j] - ref) < 1e-13 * max(1.0, abs(ref))
    e3 = I.eri3(s)
    Na = I.norm_s(a)
    V = I.nuclear(s)
    for m in range(4):
        for n in range(4):
            p = a[m] + a[n]
            Kab = np.exp(-a[m] * a[n] / p * np.sum((X[m] - X[n]) ** 2))
            P = (a[m] * X[m] + a[n] * X[n]) / p
            Qab = Na[m] * Na[n] * Kab * (np.pi / p) ** 1.5
            for c in range(4):
                w = p * k[c] / (p + k[c])
                ref = _electrostatic(Qab, Qk[c], w, np.linalg.norm(P - Xk[c]))
                assert abs(e3[c, m, n] - ref) < 1e-13 * max(1.0, abs(ref))
            vref = 0.0
            for zc, cc in zip(s.atom_charge, s.atom_xyz):
                vref -= zc * _electrostatic(Qab, 1.0, p, np.linalg.norm(P - cc))
            assert abs(V[m, n] - vref) < 1e-13 * max(1.0, abs(vref))
    e4 = I.eri4(s)
    for (m, n, l, t) in [(0, 1, 2, 3), (1, 1, 0, 2), (3, 2, 3, 2), (0, 0, 0, 0)]:
        p = a[m] + a[n]
        q = a[l] + a[t]
        P = (a[m] * X[m] + a[n] * X[n]) / p
        Q = (a[l] * X[l] + a[t] * X[t]) / q
        Qab = Na[m] * Na[n] * np.exp(-a[m] * a[n] / p * np.sum((X[m] - X[n]) ** 2)) * (np.pi / p) ** 1.5
        Qcd = Na[l] * Na[t] * np.exp(-a[l] * a[t] / q * np.sum((X[l] - X[t]) ** 2)) * (np.pi / q) ** 1.5
        ref = _electrostatic(Qab, Qcd, p * q / (p + q), np.linalg.norm(P - Q))
        assert abs(e4[m, n, l, t] - ref) < 1e-13 * max(1.0, abs(ref))


def test_kinetic_against_quadrature():
    xyz = [[0.0, 0.0, 0.0], [0.4, -0.7, 1.1]]
    s = _toy_system(xyz, [1, 1], [0, 1], [0.6, 1.9])
    T = I.kinetic(s)
    A, B = s.atom_xyz
    a, b = s.bf_alpha
    x = np.linspace(-14.0, 14.0, 400001)

    def ov(d):
        return np.trapezoid(np.exp(-a * (x - A[d]) ** 2) * np.exp(-b * (x - B[d]) ** 2), x)

    def lap(d):
        gb = np.exp(-b * (x - B[d]) ** 2)
        d2 = (4.0 * b * b * (x - B[d]) ** 2 - 2.0 * b) * gb
        return np.trapezoid(np.exp(-a * (x - A[d]) ** 2) * d2, x)

    o = [ov(d) for d in range(3)]
    l = [lap(d) for d in range(3)]
    lapl = l[0] * o[1] * o[2] + o[0] * l[1] * o[2] + o[0] * o[1] * l[2]
    ref = -0.5 * I.norm_s(a) * I.norm_s(b) * lapl
    assert abs(T[0, 1] - ref) < 1e-10


def test_sto3g_h2_textbook_values():
    g = json.load(open(os.path.join(GOLDEN, "sto3g_h2.json")))
    zeta = g["zeta"]
    alphas = np.array(g["sto3g_1s_exponents_zeta1"]) * zeta ** 2
    coef = np.array(g["sto3g_1s_coefficients"])
    R = g["R_bohr"]
    s = _toy_system([[0, 0, 0], [0, 0, R]], [1, 1], [0, 0, 0, 1, 1, 1], np.concatenate([alphas, alphas]))
    D = np.zeros((6, 2))
    D[:3, 0] = coef
    D[3:, 1] = coef
    S = D.T @ I.overlap(s) @ D
    T = D.T @ I.kinetic(s) @ D
    V = D.T @ I.nuclear(s) @ D
    one = _toy_system([[0, 0, 0], [0, 0, R]], [1, 0], [0, 0, 0, 1, 1, 1], np.concatenate([alphas, alphas]))
    V1 = D.T @ I.nuclear(one) @ D
    e4 = np.einsum("abcd,ai,bj,ck,dl->ijkl", I.eri4(s), D, D, D, D)
    v = g["values"]
    tol = g["tolerance"]
    got = {
        "S12": S[0, 1], "T11": T[0, 0], "T12": T[0, 1],
        "V1_11": V1[0, 0], "V1_12": V1[0, 1], "V1_22": V1[1, 1],
        "Hcore11": (T + V)[0, 0], "Hcore12": (T + V)[0, 1],
        "eri_1111": e4[0, 0, 0, 0], "eri_1122": e4[0, 0, 1, 1],
        "eri_2111": e4[1, 0, 0, 0], "eri_2121": e4[1, 0, 1, 0],
    }
    for key, ref in v.items():
        assert abs(got[key] - ref) <= tol, (key, got[key], ref)
    np.testing.assert_allclose(np.diag(S), 1.0, atol=2e-6)


def test_nuclear_repulsion():
    s = _toy_system([[0, 0, 0], [0, 0, 2.0], [0, 3.0, 0]], [1, 2, 3], [0], [1.0])
    ref = 1 * 2 / 2.0 + 1 * 3 / 3.0 + 2 * 3 / np.sqrt(13.0)
    assert abs(I.nuclear_repulsion(s) - ref) < 1e-14
