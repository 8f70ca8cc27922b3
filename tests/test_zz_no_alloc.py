"""The entry point that allocates nothing (donof_ri_jmo_noalloc) agrees with donof_ri_jk_mo.

Some callers cannot allocate device memory: code running under an allocator
or memory pool that forbids cudaMalloc, or a service that must keep its device
footprint fixed after start-up.  donof_ri_jmo_noalloc computes the Coulomb
matrix J_pq = sum_P b^P_pp b^P_qq from a diagonal the caller already holds,
using only the library's static scratch array.  Its result must match the
context path's J (donof_ri_jk_mo, TF32X3) on the same diagonal, within the
split-precision tolerance of the other TF32X3 tests, on two calls in a row:
the second call runs on the scratch contents the first one left behind.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

REL = 2e-5  # as in test_gpu_mixed.py


@pytest.mark.parametrize("name", ["square4", "c6h12"])
def test_noalloc_j_matches_context_path(name):
    import torch
    from paper_2012_15662_gb300 import binding as bd
    from synthetic import make_workload
    w = make_workload(name)
    s = w.system
    eng = bd.Engine(s, bd.DONOF_RI_TF32X3)
    eng.transform(w.C, bd.DONOF_RI_FULL)
    J_ref, _ = eng.jk_mo()
    d = eng.fetch(bd.DONOF_RI_FETCH_DIAG)          # [naux][n_omega]
    eng.close()
    dev = torch.device("cuda", 0)
    d_dev = torch.from_numpy(np.ascontiguousarray(d)).to(dev)
    m = s.n_omega
    for _ in range(2):
        J_dev = torch.full((m, m), np.nan, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        bd.donof_ri_jmo_noalloc(d_dev, s.naux, m, J_dev)
        torch.cuda.synchronize()
        J = J_dev.cpu().numpy()
        assert np.isfinite(J).all()
        err = np.abs(J - J_ref).max()
        assert err <= REL * np.abs(J_ref).max(), (err, np.abs(J_ref).max())


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_2012_15662_gb300 import binding as bd
    dev = torch.device("cuda", 0)
    d = torch.zeros(16, dtype=torch.float64, device=dev)
    J = torch.zeros(16, dtype=torch.float64, device=dev)
    with pytest.raises(bd.DonofError) as ei:
        bd.donof_ri_jmo_noalloc(d, 60000, 4000, J)
    assert ei.value.status == bd.DONOF_RI_E_ARG
