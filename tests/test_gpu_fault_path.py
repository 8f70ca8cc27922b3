"""Failure detection without a GPU fault: a bounded device-side wait that runs out.

Every mbarrier wait in the engine's tensor-core kernels gives up after a time
limit, records DONOF_RI_E_TIMEOUT in the context's status word and lets the CTA
exit with nothing in flight.  donof_ri_check_wait_timeout runs the same bounded
wait on an mbarrier that nothing completes, with a short limit: the next sync
must report the timeout, the sync after it must be clean, and the context must
give the same results as before (bit for bit), i.e. it stays usable.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from tests.workloads import make_workload  # noqa: E402


@pytest.mark.parametrize("prec_name", ["slice4", "fp64"])
def test_timed_out_wait_is_reported_and_context_stays_usable(prec_name):
    import time
    from paper_2012_15662_gb300 import binding as bd
    prec = bd.DONOF_RI_SLICE4 if prec_name == "slice4" else bd.DONOF_RI_FP64
    w = make_workload("square4")
    eng = bd.Engine(w.system, prec)
    eng.transform(w.C, bd.DONOF_RI_FULL)
    J0, K0 = eng.jk_mo()
    eng.jk_ao(want=False)
    E0, lam0 = eng.energy_lagrangian(w.gamma)
    t0 = time.perf_counter()
    bd.donof_ri_check_wait_timeout(eng.ctx, 20_000_000)  # 20 ms
    with pytest.raises(bd.DonofError) as e:
        bd.donof_ri_sync(eng.ctx)
    dt = time.perf_counter() - t0
    assert e.value.status == bd.DONOF_RI_E_TIMEOUT
    assert 0.015 <= dt < 2.0
    bd.donof_ri_sync(eng.ctx)          # the status was consumed
    eng.transform(w.C, bd.DONOF_RI_FULL)
    J1, K1 = eng.jk_mo()
    eng.jk_ao(want=False)
    E1, lam1 = eng.energy_lagrangian(w.gamma)
    eng.close()
    np.testing.assert_array_equal(J0, J1)
    np.testing.assert_array_equal(K0, K1)
    assert E0 == E1
    np.testing.assert_array_equal(lam0, lam1)


def test_wait_limit_is_checked():
    from paper_2012_15662_gb300 import binding as bd
    w = make_workload("square4")
    eng = bd.Engine(w.system, bd.DONOF_RI_FP64)
    for bad in (0, 999, 6_000_000_000):
        with pytest.raises(bd.DonofError) as e:
            bd.donof_ri_check_wait_timeout(eng.ctx, bad)
        assert e.value.status == bd.DONOF_RI_E_ARG
    bd.donof_ri_sync(eng.ctx)
    eng.close()
