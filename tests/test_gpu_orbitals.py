"""GPU orbital rotation step and the outer / inner iterations.

* donof_ri_rotate_orbitals against oracle/orbopt.rotation_step (scipy's expm) at
  the oracle's own Lagrangian: the FP64 engine to 1e-10, orthonormal in the
  overlap metric (C^T S C = I) to 1e-13;
* 100 inner iterations of the rotation driver follow the oracle's driver
  (oracle/orbopt.optimize) and keep C^T S C = I to 1e-12;
* the inner iterations never raise the energy and shrink the rotation gradient;
* the outer / inner driver (solve.py) lowers the energy over its iterations, and
  the FP64 and SLICE4 engines follow the same path within the energy bar.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import integrals as I, orbopt, ri  # noqa: E402
from synthetic import pairing_columns, standard_gamma  # noqa: E402
from tests.workloads import make_workload  # noqa: E402


@pytest.mark.parametrize("name", ["square4", "c6h12"])
def test_rotation_step_matches_oracle(name):
    from paper_2012_15662_gb300 import binding as bd
    w = make_workload(name)
    s = w.system
    eng = bd.Engine(s, bd.DONOF_RI_FP64)
    eng.transform(w.C, bd.DONOF_RI_HALF)
    eng.jk_ao(want=False)
    E, lam = eng.energy_lagrangian(w.gamma)
    C1, gmax = eng.rotate(0.1)
    eng.close()
    B, L, G = ri.setup(s)
    sub, rank = pairing_columns(s.n_strong, s.n_weak_per)
    Eo, lamo = orbopt.energy_lambda(s, B, I.core_hamiltonian(s), I.nuclear_repulsion(s), w.C, w.gamma, sub, rank)
    assert gmax == pytest.approx(np.abs(lamo - lamo.T).max(), rel=1e-10)
    Co = orbopt.rotation_step(w.C, lamo, 0.1)
    assert np.abs(C1 - Co).max() <= 1e-10
    S = I.overlap(s)
    assert np.abs(C1.T @ S @ C1 - np.eye(s.nbf)).max() <= 1e-13


@pytest.mark.parametrize("name,iters", [("square4", 100), ("c6h12", 25)])
def test_inner_iterations_follow_oracle_and_stay_orthonormal(name, iters):
    from paper_2012_15662_gb300 import binding as bd, solve
    w = make_workload(name)
    s = w.system
    sub, rank = pairing_columns(s.n_strong, s.n_weak_per)
    Co, Eo, go, ito = orbopt.optimize(s, w.C, w.gamma, sub, rank, max_iter=iters, gtol=0.0)
    eng = bd.Engine(s, bd.DONOF_RI_FP64)
    r = solve.orbital_iterations(eng, bd.Engine.colmajor(w.C), w.gamma, max_iter=iters, gtol=0.0, etol=0.0)
    eng.close()
    C = r["C"].reshape(s.nbf, s.nbf).T
    S = I.overlap(s)
    assert r["iterations"] == ito == iters
    assert np.abs(C.T @ S @ C - np.eye(s.nbf)).max() <= 1e-12
    assert abs(r["E"] - Eo) <= 1e-9 * max(1.0, abs(Eo))
    assert np.abs(C - Co).max() <= 1e-8


def test_inner_iterations_descend():
    from paper_2012_15662_gb300 import binding as bd, solve
    w = make_workload("square4")
    eng = bd.Engine(w.system, bd.DONOF_RI_FP64)
    E0 = None
    r = solve.orbital_iterations(eng, bd.Engine.colmajor(w.C), w.gamma, max_iter=1)
    E0, g0 = r["E"], r["gmax"]
    r = solve.orbital_iterations(eng, bd.Engine.colmajor(w.C), w.gamma, max_iter=40)
    assert r["E"] < E0 and r["gmax"] < g0
    eng.close()


def test_outer_inner_driver_fp64_and_slice4_agree():
    """Both engines' drivers descend; the SLICE4 driver's final energy is its FP64
    value: the FP64 engine at the SLICE4 driver's final orbitals and angles gives the
    same energy within the 1e-6 Eh bar.  (From these random orbitals the occupation
    landscape has several minima, so the two drivers need not end in the same one.)"""
    from paper_2012_15662_gb300 import binding as bd, solve
    w = make_workload("square4")
    s = w.system
    g0 = standard_gamma(s.n_strong, s.n_weak_per)
    out = {}
    for name, prec in [("fp64", bd.DONOF_RI_FP64), ("slice4", bd.DONOF_RI_SLICE4)]:
        eng = bd.Engine(s, prec)
        out[name] = solve.solve(eng, w.C, g0, max_outer=3, max_inner=15)
        eng.close()
    for name in out:
        h = out[name]["history"]
        assert all(h[i + 1]["E"] <= h[i]["E"] + 1e-9 for i in range(len(h) - 1)), name
    r = out["slice4"]
    eng = bd.Engine(s, bd.DONOF_RI_FP64)
    eng.transform(r["C"], bd.DONOF_RI_HALF)
    eng.jk_ao(want=False)
    E64, _ = eng.energy_lagrangian(r["gamma"])
    eng.close()
    assert abs(E64 - r["E"]) <= 1e-6
