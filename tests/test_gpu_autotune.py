"""The SLICE4 tile-schedule autotuner: call order, and results that still meet
the parity bars after the tuned schedule (pipeline depth, split counts and the
symmetric J^(q) choice all change the kernels' work assignment)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import integrals as I, pnof7, ri  # noqa: E402
from synthetic import pairing_columns  # noqa: E402
from tests.workloads import make_workload  # noqa: E402


def test_autotune_call_order():
    from paper_2012_15662_gb300 import binding as bd
    w = make_workload("square4")
    eng = bd.Engine(w.system, bd.DONOF_RI_SLICE4)
    with pytest.raises(bd.DonofError) as e:
        bd.donof_ri_autotune(eng.ctx)
    assert e.value.status == bd.DONOF_RI_E_STATE
    eng.close()
    eng = bd.Engine(w.system, bd.DONOF_RI_FP64)
    eng.transform(w.C, bd.DONOF_RI_FULL)
    eng.jk_ao(want=False)
    with pytest.raises(bd.DonofError) as e:
        bd.donof_ri_autotune(eng.ctx)
    assert e.value.status == bd.DONOF_RI_E_UNSUPPORTED
    eng.close()


@pytest.mark.parametrize("name", ["c6h12", "c10h20"])
def test_tuned_schedule_keeps_parity(name):
    from paper_2012_15662_gb300 import binding as bd
    w = make_workload(name)
    s = w.system
    eng = bd.Engine(s, bd.DONOF_RI_SLICE4)
    eng.transform(w.C, bd.DONOF_RI_FULL)
    eng.jk_ao(want=False)
    rep, tried = bd.donof_ri_autotune(eng.ctx, reps=3)
    assert tried >= 6
    assert (rep[:, 0] >= 2).all() and (rep[:, 3] > 0).all()
    eng.transform(w.C, bd.DONOF_RI_FULL)
    J, K = eng.jk_mo()
    Jao, Kao = eng.jk_ao()
    E, lam = eng.energy_lagrangian(w.gamma)
    eng.close()
    B, L, G = ri.setup(s)
    m = s.n_omega
    r = ri.all_rows(B, w.C, m)
    H = I.core_hamiltonian(s)
    sub, rank = pairing_columns(s.n_strong, s.n_weak_per)
    n = pnof7.occupations(w.gamma, s.n_strong, s.n_weak_per, sub, rank)
    A, Bc = pnof7.coupling(n, sub, rank)
    Hd = np.einsum("mp,mn,np->p", w.C[:, :m], H, w.C[:, :m])
    Eo = pnof7.energy(n, Hd, r["J"], r["K"], A, Bc, I.nuclear_repulsion(s))
    assert np.abs(J - r["J"]).max() <= 1e-7 and np.abs(K - r["K"]).max() <= 1e-7
    assert np.abs(Jao - r["Jao"]).max() <= 1e-7 and np.abs(Kao - r["Kao"]).max() <= 1e-7
    assert abs(E - Eo) <= 1e-6


@pytest.mark.parametrize("name", ["square4", "c6h12"])
def test_every_schedule_variant_keeps_parity(name):
    """Each schedule the autotuner may choose, set directly: the one-CTA half
    transform, the full J^(q) (no symmetric skip), two waves for the split kinds,
    the shallowest pipelines: bit-identical where the arithmetic order is the
    same and within the SLICE4 bars everywhere."""
    from paper_2012_15662_gb300 import binding as bd
    w = make_workload(name)
    s = w.system
    B, L, G = ri.setup(s)
    r = ri.all_rows(B, w.C, s.n_omega)

    def run(eng):
        eng.transform(w.C, bd.DONOF_RI_FULL)
        J, K = eng.jk_mo()
        Jao, Kao = eng.jk_ao()
        E, lam = eng.energy_lagrangian(w.gamma)
        return J, K, Jao, Kao, E, lam

    eng = bd.Engine(s, bd.DONOF_RI_SLICE4)
    ref = run(eng)
    for kind, stages, option in [(0, 2, 1), (0, 3, 1), (3, 2, 0), (3, 3, 1), (1, 2, 2), (2, 2, 2), (5, 2, 2),
                                 (4, 2, 0)]:
        bd.donof_ri_set_schedule(eng.ctx, kind, stages, option)
    out = run(eng)
    with pytest.raises(bd.DonofError) as e:
        bd.donof_ri_set_schedule(eng.ctx, 0, 99, 0)
    assert e.value.status == bd.DONOF_RI_E_ARG
    eng.close()
    # the half transform's integers and the J^(q) / K^(q) values do not depend on the schedule
    np.testing.assert_array_equal(out[2], ref[2])
    np.testing.assert_array_equal(out[3], ref[3])
    for got in (out, ref):
        assert np.abs(got[0] - r["J"]).max() <= 1e-7 and np.abs(got[1] - r["K"]).max() <= 1e-7
        assert np.abs(got[2] - r["Jao"]).max() <= 1e-7 and np.abs(got[3] - r["Kao"]).max() <= 1e-7
