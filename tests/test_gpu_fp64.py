"""GPU parity of the plain FP64 path against the oracle, element by element.

Sizes: the four-atom system (nbf=24, naux=80, N_Omega=12) and the C6H12-shaped
ring (nbf=144, naux=504, N_Omega=120): several GEMM tiles with ragged tails.
Tolerances: FP64 arithmetic on both sides, differing in summation order and in
the factorisation of a metric with condition number ~1e7, so results agree to
~1e-9 relative (stated per quantity below).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import integrals as I, pnof7, ri  # noqa: E402
from tests.workloads import make_workload  # noqa: E402


def _oracle(w):
    s = w.system
    B, L, G = ri.setup(s)
    m = s.n_omega
    rows = ri.all_rows(B, w.C, m)
    H = I.core_hamiltonian(s)
    from synthetic import pairing_columns
    sub, rank = pairing_columns(s.n_strong, s.n_weak_per)
    n = pnof7.occupations(w.gamma, s.n_strong, s.n_weak_per, sub, rank)
    A, Bc = pnof7.coupling(n, sub, rank)
    Hd = np.einsum("mp,mn,np->p", w.C[:, :m], H, w.C[:, :m])
    e_nuc = I.nuclear_repulsion(s)
    E = pnof7.energy(n, Hd, rows["J"], rows["K"], A, Bc, e_nuc)
    lam = pnof7.lagrangian(w.C, H, rows["Jao"], rows["Kao"], n, A, Bc)
    return dict(B=B, L=L, G=G, H=H, S=I.overlap(s), e_nuc=e_nuc, n=n, E=E, lam=lam, **rows)


@pytest.fixture(scope="module", params=["square4", "c6h12"])
def case(request):
    from paper_2012_15662_gb300 import binding as bd
    w = make_workload(request.param)
    ref = _oracle(w)
    eng = bd.Engine(w.system, bd.DONOF_RI_FP64)
    yield w, ref, eng
    eng.close()


def test_setup_matches_oracle(case):
    from paper_2012_15662_gb300 import binding as bd
    w, ref, eng = case
    np.testing.assert_allclose(eng.fetch(bd.DONOF_RI_FETCH_OVERLAP), ref["S"], atol=1e-13)
    np.testing.assert_allclose(eng.fetch(bd.DONOF_RI_FETCH_HCORE), ref["H"], atol=1e-12 * np.abs(ref["H"]).max())
    assert abs(eng.fetch(bd.DONOF_RI_FETCH_ENUC)[0] - ref["e_nuc"]) < 1e-12 * ref["e_nuc"]
    L = np.tril(eng.fetch(bd.DONOF_RI_FETCH_METRIC))
    np.testing.assert_allclose(L, ref["L"], atol=1e-10)
    B = eng.fetch(bd.DONOF_RI_FETCH_B)
    np.testing.assert_allclose(B, ref["B"], atol=1e-9 * np.abs(ref["B"]).max())


def test_transform_rows(case):
    from paper_2012_15662_gb300 import binding as bd
    w, ref, eng = case
    eng.transform(w.C, bd.DONOF_RI_FULL)
    sc = np.abs(ref["bh"]).max()
    np.testing.assert_allclose(eng.fetch(bd.DONOF_RI_FETCH_BHALF), ref["bh"], atol=1e-9 * sc)
    np.testing.assert_allclose(eng.fetch(bd.DONOF_RI_FETCH_DIAG), ref["d"], atol=1e-9 * sc)
    J, K = eng.jk_mo()
    np.testing.assert_allclose(J, ref["J"], atol=1e-9)
    np.testing.assert_allclose(K, ref["K"], atol=1e-9)


def test_jk_ao_energy_lambda(case):
    from paper_2012_15662_gb300 import binding as bd
    w, ref, eng = case
    eng.transform(w.C, bd.DONOF_RI_HALF)
    Jao, Kao = eng.jk_ao()
    np.testing.assert_allclose(Jao, ref["Jao"], atol=1e-9)
    np.testing.assert_allclose(Kao, ref["Kao"], atol=1e-9)
    E, lam = eng.energy_lagrangian(w.gamma)
    np.testing.assert_allclose(eng.fetch(bd.DONOF_RI_FETCH_OCC), ref["n"], atol=1e-15)
    assert abs(E - ref["E"]) < 1e-8, (E, ref["E"])
    np.testing.assert_allclose(lam, ref["lam"], atol=1e-8)


def test_status_codes(case):
    from paper_2012_15662_gb300 import binding as bd
    w, ref, eng = case
    # jk_mo after a HALF transform has no full transform to read
    eng.transform(w.C, bd.DONOF_RI_HALF)
    with pytest.raises(bd.DonofError) as ei:
        eng.jk_mo()
    assert ei.value.status == bd.DONOF_RI_E_STATE
    # a NaN orbital coefficient is reported at the next synchronising call
    C = w.C.copy()
    C[3, 1] = np.nan
    eng.transform(C, bd.DONOF_RI_FULL)
    with pytest.raises(bd.DonofError) as ei:
        eng.jk_mo()
    assert ei.value.status == bd.DONOF_RI_E_NONFINITE
    # the context stays usable
    eng.transform(w.C, bd.DONOF_RI_FULL)
    J, K = eng.jk_mo()
    np.testing.assert_allclose(J, ref["J"], atol=1e-9)


def test_metric_not_positive_definite():
    from paper_2012_15662_gb300 import binding as bd
    w = make_workload("square4")
    s = w.system
    # duplicate an auxiliary function: G becomes exactly singular
    s.aux_alpha = s.aux_alpha.copy()
    s.aux_alpha[1] = s.aux_alpha[0]
    with pytest.raises(bd.DonofError) as ei:
        bd.Engine(s, bd.DONOF_RI_FP64)
    assert ei.value.status == bd.DONOF_RI_E_METRIC_NOT_PD
