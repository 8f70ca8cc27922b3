"""GPU occupation optimisation (donof_ri_optimize_occupations) against the oracle.

* evaluation parity: E(gamma) and dE/dgamma of the device kernel against
  oracle/onopt.py at random angles (FP64 engine: to rounding; SLICE4: within
  the energy bar, the gradient within the same relative budget);
* optimisation: the device L-BFGS from the standard guess reaches a point whose
  gradient is below gtol, whose energy equals the oracle optimiser's minimum
  (the two optimisers take different paths to the same local minimum) and whose
  occupations agree (n, not gamma, is unique: gamma and -gamma give the same n);
* call order and argument errors.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import integrals as I, onopt, pnof7, ri  # noqa: E402
from synthetic import pairing_columns  # noqa: E402
from tests.workloads import make_workload  # noqa: E402


def _oracle_jk(w):
    s = w.system
    B, L, G = ri.setup(s)
    m = s.n_omega
    bh = ri.half_transform(B, w.C, m)
    J, K = ri.jk_mo(ri.full_transform(bh, w.C), ri.diagonal(bh, w.C))
    H = I.core_hamiltonian(s)
    Hd = np.einsum("mp,mn,np->p", w.C[:, :m], H, w.C[:, :m])
    return J, K, Hd, I.nuclear_repulsion(s)


@pytest.fixture(scope="module", params=[("square4", "fp64"), ("c6h12", "fp64"), ("c6h12", "slice4")])
def case(request):
    from paper_2012_15662_gb300 import binding as bd
    name, prec = request.param
    w = make_workload(name)
    eng = bd.Engine(w.system, bd.DONOF_RI_FP64 if prec == "fp64" else bd.DONOF_RI_SLICE4)
    eng.transform(w.C, bd.DONOF_RI_FULL)
    yield w, prec, eng, _oracle_jk(w)
    eng.close()


def test_energy_and_gradient_match_oracle(case):
    w, prec, eng, (J, K, Hd, enuc) = case
    s = w.system
    sub, rank = pairing_columns(s.n_strong, s.n_weak_per)
    rng = np.random.default_rng(5)
    for _ in range(3):
        g0 = rng.uniform(0.05, 1.4, s.n_strong * s.n_weak_per)
        gam, E, grad, it, reason = eng.optimize_occupations(g0, max_iter=0)
        assert np.array_equal(gam, g0) and it == 0
        Eo, go = onopt.energy_and_gradient(g0, s.n_strong, s.n_weak_per, sub, rank, Hd, J, K, enuc)
        scale = max(1.0, np.abs(go).max())
        if prec == "fp64":
            assert abs(E - Eo) <= 1e-12 * max(1.0, abs(Eo))
            assert np.abs(grad - go).max() <= 1e-10 * scale
        else:
            assert abs(E - Eo) <= 1e-6
            assert np.abs(grad - go).max() <= 1e-6 * scale


def test_optimisation_reaches_the_oracle_minimum(case):
    w, prec, eng, (J, K, Hd, enuc) = case
    s = w.system
    sub, rank = pairing_columns(s.n_strong, s.n_weak_per)
    g0 = onopt.standard_guess(s.n_strong, s.n_weak_per)
    gam, E, grad, it, reason = eng.optimize_occupations(g0, max_iter=5000, gtol=1e-8, etol=1e-14)
    assert reason in (0, 3) and it > 0
    go, Eo, no, ito, gmo = onopt.optimize(g0, s.n_strong, s.n_weak_per, sub, rank, Hd, J, K, enuc, gtol=1e-9)
    n = pnof7.occupations(gam, s.n_strong, s.n_weak_per, sub, rank)
    # Minima of these systems put some occupations at 0 or at the strong bound 1/2,
    # on kinks of E(gamma) where both optimisers end on the energy criterion; the
    # device optimiser must reach the oracle's minimum energy to 1e-8 relative.
    assert abs(E - Eo) <= 1e-8 * max(1.0, abs(Eo))
    assert np.abs(n - no).max() <= 1e-3
    E0, _ = onopt.energy_and_gradient(g0, s.n_strong, s.n_weak_per, sub, rank, Hd, J, K, enuc)
    assert E < E0


def test_call_order_and_arguments():
    from paper_2012_15662_gb300 import binding as bd
    w = make_workload("square4")
    eng = bd.Engine(w.system, bd.DONOF_RI_FP64)
    g0 = np.full(w.system.n_strong * w.system.n_weak_per, 0.2)
    with pytest.raises(bd.DonofError) as e:
        eng.optimize_occupations(g0)
    assert e.value.status == bd.DONOF_RI_E_STATE
    eng.transform(w.C, bd.DONOF_RI_HALF)
    with pytest.raises(bd.DonofError):
        eng.optimize_occupations(g0)  # a HALF transform has no J, K
    eng.transform(w.C, bd.DONOF_RI_FULL)
    with pytest.raises(bd.DonofError) as e:
        eng.optimize_occupations(g0, gtol=-1.0)
    assert e.value.status == bd.DONOF_RI_E_ARG
    eng.close()
