"""The paper's scheme to convergence on the device and the RI -> exact restart.

From the device RI-HF orbitals (donof_ri_rhf), solve.converge runs the outer /
inner iterations (occupation optimisation, then F^lambda orbital steps) to
|dE| < 1e-6 Eh with max |lambda - lambda^T| <= 1e-4, in FP64 and in the digit-plane
form; then the converged FP64 RI run is restarted with exact four-centre
integrals (donof_ri_exact_jk), which must converge in at most two outer
iterations (Sec. 4 and the Abstract).  Checked against the oracle's driver
(oracle/orbopt.converge, pinned in tests/test_oracle_convergence.py): the device's
final point has the energy the oracle computes there (to 1e-9 in FP64) and is
stationary by the oracle's Lagrangian; the converged energies agree with the
oracle's run to 2e-5 Eh (both stop once an outer iteration changes E by less than
1e-6 while E still drifts by a few 1e-7 per outer iteration, and the device's
occupation optimiser is its own L-BFGS, so the two paths are not step for step the
same).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import integrals as I, orbopt, rhf, ri  # noqa: E402
from synthetic import pairing_columns, standard_gamma  # noqa: E402
from tests.workloads import make_workload  # noqa: E402

PATH_TOL = 2e-5


@pytest.fixture(scope="module")
def oracle_runs():
    w = make_workload("square4")
    s = w.system
    B, L, G = ri.setup(s)
    hf = rhf.scf(I.core_hamiltonian(s), I.overlap(s), rhf.jk_ri(B), s.n_strong, I.nuclear_repulsion(s), tol=1e-9)
    sub, rank = pairing_columns(s.n_strong, s.n_weak_per)
    r = orbopt.converge(s, hf["C"], standard_gamma(s.n_strong, s.n_weak_per), hf["eps"], sub, rank, B=B)
    x = orbopt.converge(s, r["C"], r["gamma"], r["diag"], sub, rank, eri=I.eri4(s))
    return w, B, sub, rank, r, x


def test_device_scheme_converges_and_exact_restart_takes_two_outer_iterations(oracle_runs):
    from paper_2012_15662_gb300 import binding as bd, solve
    w, B, sub, rank, ro, xo = oracle_runs
    s = w.system
    g0 = standard_gamma(s.n_strong, s.n_weak_per)
    eng = bd.Engine(s, bd.DONOF_RI_FP64)
    C0, eps0, E_hf, it, com = eng.rhf(max_iter=100, tol=1e-9)
    r = solve.converge(eng, C0, g0, eps0)
    assert r["converged"], r["history"][-3:]
    assert abs(r["E"] - ro["E"]) <= PATH_TOL, (r["E"], ro["E"])
    # the final point by the oracle: its energy, and stationarity
    Eo, lam = orbopt.energy_lambda(s, B, I.core_hamiltonian(s), I.nuclear_repulsion(s), r["C"], r["gamma"], sub, rank)
    assert abs(Eo - r["E"]) <= 1e-9 * max(1.0, abs(Eo))
    assert np.abs(lam - lam.T).max() <= 1.01e-4
    x = solve.converge(eng, r["C"], r["gamma"], r["diag"], exact=True)
    eng.close()
    assert x["converged"] and x["outer"] <= 2, x["history"]
    assert abs(x["E"] - xo["E"]) <= PATH_TOL, (x["E"], xo["E"])
    assert x["E"] < r["E"]


def test_digit_plane_form_converges_to_the_same_energy(oracle_runs):
    from paper_2012_15662_gb300 import binding as bd, solve
    w, B, sub, rank, ro, xo = oracle_runs
    s = w.system
    eng = bd.Engine(s, bd.DONOF_RI_SLICE4)
    C0, eps0, E_hf, it, com = eng.rhf(max_iter=100, tol=1e-9)
    r = solve.converge(eng, C0, standard_gamma(s.n_strong, s.n_weak_per), eps0)
    eng.close()
    assert r["converged"]
    assert abs(r["E"] - ro["E"]) <= PATH_TOL, (r["E"], ro["E"])
    Eo, _ = orbopt.energy_lambda(s, B, I.core_hamiltonian(s), I.nuclear_repulsion(s), r["C"], r["gamma"], sub, rank)
    assert abs(Eo - r["E"]) <= 1e-6


def test_quasi_newton_inner_step_converges(oracle_runs):
    """The quasi-Newton orbital step (solve.lbfgs_iterations: L-BFGS on the rotation
    generator through donof_ri_apply_rotation) converges the same scheme in fewer inner
    iterations, to a stationary point at least as low as the F^lambda run's, whose
    energy the oracle confirms."""
    from paper_2012_15662_gb300 import binding as bd, solve
    w, B, sub, rank, ro, xo = oracle_runs
    s = w.system
    eng = bd.Engine(s, bd.DONOF_RI_FP64)
    C0, eps0, E_hf, it, com = eng.rhf(max_iter=100, tol=1e-9)
    r = solve.converge(eng, C0, standard_gamma(s.n_strong, s.n_weak_per), eps0, inner="lbfgs", max_inner=300)
    eng.close()
    assert r["converged"], r["history"][-3:]
    assert r["inner_total"] < ro["inner_total"]
    assert r["E"] <= ro["E"] + PATH_TOL
    Eo, lam = orbopt.energy_lambda(s, B, I.core_hamiltonian(s), I.nuclear_repulsion(s), r["C"], r["gamma"], sub, rank)
    assert abs(Eo - r["E"]) <= 1e-9 * max(1.0, abs(Eo))
    assert np.abs(lam - lam.T).max() <= 1.01e-4


def test_apply_rotation_matches_expm():
    """donof_ri_apply_rotation against scipy's expm: C expm(kappa), C^T S C = I."""
    from scipy.linalg import expm
    from paper_2012_15662_gb300 import binding as bd
    w = make_workload("c6h12")
    s = w.system
    rng = np.random.default_rng(11)
    X = rng.standard_normal((s.nbf, s.nbf)) * 0.3
    kappa = np.ascontiguousarray(X - X.T)
    eng = bd.Engine(s, bd.DONOF_RI_FP64)
    eng.transform(w.C, bd.DONOF_RI_HALF)          # the context's orbitals
    Ccm = np.empty(s.nbf * s.nbf)
    bd.donof_ri_apply_rotation(eng.ctx, kappa, Ccm)
    eng.close()
    C1 = Ccm.reshape(s.nbf, s.nbf).T
    np.testing.assert_allclose(C1, w.C @ expm(kappa), atol=1e-10)
    np.testing.assert_allclose(C1.T @ I.overlap(s) @ C1, np.eye(s.nbf), atol=1e-12)
