"""The contracted Lagrangian (donof_ri_energy_lagrangian_contracted): F^(p) C_p
straight from the RI transforms gives the energy and lambda of the per-orbital
form (J^(q), K^(q) then the Fock sum) and of the oracle's contracted form."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import integrals as I, pnof7, ri  # noqa: E402
from synthetic import pairing_columns  # noqa: E402
from tests.workloads import make_workload  # noqa: E402


@pytest.mark.parametrize("name", ["square4", "c6h12"])
def test_contracted_matches_per_orbital_form(name):
    from paper_2012_15662_gb300 import binding as bd
    w = make_workload(name)
    s = w.system
    nb, m = s.nbf, s.n_omega
    eng = bd.Engine(s, bd.DONOF_RI_FP64)
    eng.transform(w.C, bd.DONOF_RI_FULL)
    eng.jk_ao(want=False)
    E, lam = eng.energy_lagrangian(w.gamma)
    Ec = np.zeros(1)
    lam_cm = np.empty(nb * nb)
    bd.donof_ri_energy_lagrangian_contracted(eng.ctx, np.ascontiguousarray(w.gamma), Ec, lam_cm)
    lam_c = lam_cm.reshape(nb, nb).T
    eng.close()
    assert abs(Ec[0] - E) <= 1e-12 * max(1.0, abs(E))
    np.testing.assert_allclose(lam_c, lam, atol=1e-12 * np.abs(lam).max())
    B, L, G = ri.setup(s)
    r = ri.all_rows(B, w.C, m)
    sub, rank = pairing_columns(s.n_strong, s.n_weak_per)
    n = pnof7.occupations(w.gamma, s.n_strong, s.n_weak_per, sub, rank)
    A, Bc = pnof7.coupling(n, sub, rank)
    lam_o = pnof7.lagrangian_contracted(w.C, I.core_hamiltonian(s), r["bh"], r["d"], r["bf"], n, A, Bc)
    np.testing.assert_allclose(lam_c, lam_o, atol=1e-11 * np.abs(lam_o).max())


def test_contracted_call_order_and_precision():
    from paper_2012_15662_gb300 import binding as bd
    w = make_workload("square4")
    eng = bd.Engine(w.system, bd.DONOF_RI_FP64)
    eng.transform(w.C, bd.DONOF_RI_HALF)
    with pytest.raises(bd.DonofError) as e:
        bd.donof_ri_energy_lagrangian_contracted(eng.ctx, np.ascontiguousarray(w.gamma))
    assert e.value.status == bd.DONOF_RI_E_STATE
    eng.close()
    eng = bd.Engine(w.system, bd.DONOF_RI_SLICE4)
    eng.transform(w.C, bd.DONOF_RI_FULL)
    with pytest.raises(bd.DonofError) as e:
        bd.donof_ri_energy_lagrangian_contracted(eng.ctx, np.ascontiguousarray(w.gamma))
    assert e.value.status == bd.DONOF_RI_E_UNSUPPORTED
    eng.close()
