"""GPU parity of the split-precision tensor-core path (DONOF_RI_TF32X3) vs the oracle.

Tolerance, derived from the arithmetic: each operand is carried as
hi + lo with TF32 pieces (representation error <= 2^-22 relative), the
dropped lo*lo term is <= 2^-22 relative, and products are accumulated in
FP32 (2^-24 per addition) over K = nbf or naux terms.  Every result is a
one- or two-level contraction of such sums, so its error is a small multiple
of sqrt(K) 2^-22 relative to the largest term: 2e-5 of the result's largest
magnitude bounds it with margin at these sizes (observed: ~1e-6 to 3e-6).
The energy is a sum of N_Omega^2 such terms: |dE| <= 1e-6 |E|.
This FP32-class path does not reach an absolute 1e-7 on J/K.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import integrals as I, pnof7, ri  # noqa: E402
from synthetic import pairing_columns  # noqa: E402
from tests.workloads import make_workload  # noqa: E402

REL = 2e-5


def _oracle(w):
    s = w.system
    B, L, G = ri.setup(s)
    m = s.n_omega
    rows = ri.all_rows(B, w.C, m)
    H = I.core_hamiltonian(s)
    sub, rank = pairing_columns(s.n_strong, s.n_weak_per)
    n = pnof7.occupations(w.gamma, s.n_strong, s.n_weak_per, sub, rank)
    A, Bc = pnof7.coupling(n, sub, rank)
    Hd = np.einsum("mp,mn,np->p", w.C[:, :m], H, w.C[:, :m])
    E = pnof7.energy(n, Hd, rows["J"], rows["K"], A, Bc, I.nuclear_repulsion(s))
    lam = pnof7.lagrangian(w.C, H, rows["Jao"], rows["Kao"], n, A, Bc)
    return dict(E=E, lam=lam, **rows)


@pytest.fixture(scope="module", params=["square4", "c6h12", "c10h20"])
def case(request):
    from paper_2012_15662_gb300 import binding as bd
    w = make_workload(request.param)
    ref = _oracle(w)
    eng = bd.Engine(w.system, bd.DONOF_RI_TF32X3)
    yield w, ref, eng
    eng.close()


def _close(got, ref, rel=REL):
    err = np.abs(got - ref).max()
    assert err <= rel * np.abs(ref).max(), (err, np.abs(ref).max())


def test_transform_and_jk_mo(case):
    from paper_2012_15662_gb300 import binding as bd
    w, ref, eng = case
    eng.transform(w.C, bd.DONOF_RI_FULL)
    _close(eng.fetch(bd.DONOF_RI_FETCH_BHALF), ref["bh"])
    _close(eng.fetch(bd.DONOF_RI_FETCH_DIAG), ref["d"])
    J, K = eng.jk_mo()
    _close(J, ref["J"])
    _close(K, ref["K"])
    # invariants that hold at any size
    assert np.abs(J - J.T).max() <= REL * np.abs(J).max()
    assert np.abs(np.diag(J) - np.diag(K)).max() <= REL * np.abs(J).max()


def test_jk_ao_energy(case):
    from paper_2012_15662_gb300 import binding as bd
    w, ref, eng = case
    eng.transform(w.C, bd.DONOF_RI_HALF)
    Jao, Kao = eng.jk_ao()
    _close(Jao, ref["Jao"])
    _close(Kao, ref["Kao"])
    E, lam = eng.energy_lagrangian(w.gamma)
    _close(lam, ref["lam"])
    assert abs(E - ref["E"]) <= 1e-6 * abs(ref["E"]), (E, ref["E"])


def test_repeat_is_deterministic(case):
    from paper_2012_15662_gb300 import binding as bd
    w, ref, eng = case
    out = []
    for _ in range(2):
        eng.transform(w.C, bd.DONOF_RI_FULL)
        J, K = eng.jk_mo()
        eng.jk_ao(want=False)
        E, lam = eng.energy_lagrangian(w.gamma)
        out.append((J, K, E, lam))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2]
    np.testing.assert_array_equal(out[0][3], out[1][3])
