"""The device RI-HF guess (donof_ri_rhf) against the oracle's SCF (oracle/rhf.scf).

The oracle is pinned separately (tests/test_oracle_rhf.py: the printed minimal-
basis H2 result, the determinant energy, convergence, a minimum).  Here, on the
same system, the device SCF must reach the oracle's energy, density and orbital
energies; its orbitals must be orthonormal in the overlap metric; and at its
orbitals, with every strong orbital fully occupied, the engine's PNOF7 energy must
equal the SCF energy and its Lagrangian must be symmetric (the closed-shell energy
is stationary there), in FP64 and in the digit-plane form.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import integrals as I, rhf, ri  # noqa: E402
from tests.workloads import make_workload  # noqa: E402


@pytest.fixture(scope="module", params=["square4", "c6h12"])
def ref(request):
    w = make_workload(request.param)
    s = w.system
    B, L, G = ri.setup(s)
    S = I.overlap(s)
    out = rhf.scf(I.core_hamiltonian(s), S, rhf.jk_ri(B), s.n_strong, I.nuclear_repulsion(s), tol=1e-9)
    return w, S, out


@pytest.mark.parametrize("prec_name", ["fp64", "slice4"])
def test_rhf_matches_oracle_scf(ref, prec_name):
    from paper_2012_15662_gb300 import binding as bd
    w, S, o = ref
    s = w.system
    prec = bd.DONOF_RI_FP64 if prec_name == "fp64" else bd.DONOF_RI_SLICE4
    eng = bd.Engine(s, prec)
    # the FP64 commutator F D S - S D F has a rounding floor near 1e-9 at C6H12 (|F| reaches
    # the kinetic energies of the tightest functions), so the device stops at 1e-8
    C, eps, E, it, com = eng.rhf(max_iter=100, tol=1e-8)
    no = s.n_strong
    assert com <= 1e-8
    assert abs(E - o["E"]) <= 1e-9 * max(1.0, abs(o["E"])), (E, o["E"])
    assert it <= o["iterations"] + 3, (it, o["iterations"])
    np.testing.assert_allclose(C.T @ S @ C, np.eye(s.nbf), atol=1e-12)
    D = 2.0 * C[:, :no] @ C[:, :no].T
    Do = 2.0 * o["C"][:, :no] @ o["C"][:, :no].T
    # the density to the accuracy the commutator tolerance allows (about tol / HOMO-LUMO gap)
    assert np.abs(D - Do).max() <= 1e-6 * max(1.0, np.abs(Do).max())
    # occupied orbital energies to 1e-8 of their scale; the virtual ones of nearly
    # degenerate pairs keep the FP32 Jacobi start's absolute accuracy (about 1e-7 of the
    # largest |F'| element, the kinetic energy of the tightest function, ~1e4 Eh), which
    # the density does not feel
    np.testing.assert_allclose(eps[:no], o["eps"][:no], atol=1e-8 * np.abs(o["eps"][:no]).max())
    np.testing.assert_allclose(eps[no:2 * no], o["eps"][no:2 * no], atol=1e-7 * np.abs(o["eps"]).max())
    # PNOF7 at the SCF orbitals with every strong orbital full (strong angles 0) is the
    # closed-shell determinant: E equals the SCF energy and lambda is symmetric
    gamma = np.concatenate([np.zeros(no), np.full(no * (s.n_weak_per - 1), 0.3)])
    eng.transform(C, bd.DONOF_RI_HALF)
    eng.jk_ao(want=False)
    Ep, lam = eng.energy_lagrangian(gamma)
    eng.close()
    tol_e = 1e-9 * max(1.0, abs(E)) if prec_name == "fp64" else 1e-6
    assert abs(Ep - E) <= tol_e, (Ep, E)
    assert np.abs(lam - lam.T).max() <= (1e-7 if prec_name == "fp64" else 1e-6)


def test_rhf_arguments():
    from paper_2012_15662_gb300 import binding as bd
    w = make_workload("square4")
    eng = bd.Engine(w.system, bd.DONOF_RI_FP64)
    for args in ((0, 1e-9), (10, 0.0)):
        with pytest.raises(bd.DonofError) as e:
            eng.rhf(*args)
        assert e.value.status == bd.DONOF_RI_E_ARG
    # a limit too small to converge returns the last iteration with the commutator above tol
    C, eps, E, it, com = eng.rhf(max_iter=2, tol=1e-12)
    assert it == 2 and com > 1e-12 and np.isfinite(E)
    eng.close()
