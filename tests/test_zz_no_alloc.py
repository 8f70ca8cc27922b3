"""The entry point that allocates nothing (donof_ri_jmo_noalloc).

Some callers cannot allocate device memory: code running under an allocator
or memory pool that forbids cudaMalloc, or a service that must keep its device
footprint fixed after start-up.  donof_ri_jmo_noalloc computes the Coulomb
matrix J_pq = sum_P b^P_pp b^P_qq from a diagonal the caller already holds,
using only the library's static scratch array.  Two checks, each on two calls
in a row (the second call runs on the scratch contents the first one left):
* on the engine's own diagonal, its J matches the context path's J
  (donof_ri_jk_mo, TF32X3) within the split-precision tolerance of the other
  TF32X3 tests;
* on the oracle's diagonal, its J matches the oracle's J = d^T d within the
  same tolerance.
Sizes: square4, C6H12, C10H20 (naux 840: two K blocks per chunk, and the last
chunk's second block lies wholly past naux) and C10H20 trimmed to naux 523 (a
ragged chunk).  This file is collected last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

REL = 2e-5  # as in test_gpu_mixed.py


def _workload(name):
    from synthetic import without_basis_functions
    from tests.workloads import make_workload
    if name == "c10h20-naux523":
        w = make_workload("c10h20")
        w.system = without_basis_functions(w.system, 0, w.system.naux - 523)
        return w
    return make_workload(name)


def _noalloc_twice(d, naux, m):
    import torch
    from paper_2012_15662_gb300 import binding as bd
    dev = torch.device("cuda", 0)
    d_dev = torch.from_numpy(np.ascontiguousarray(d)).to(dev)
    out = []
    for _ in range(2):
        J_dev = torch.full((m, m), np.nan, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        bd.donof_ri_jmo_noalloc(d_dev, naux, m, J_dev)
        torch.cuda.synchronize()
        out.append(J_dev.cpu().numpy())
    return out


@pytest.mark.parametrize("name", ["square4", "c6h12", "c10h20", "c10h20-naux523"])
def test_noalloc_j_matches_context_path_and_oracle(name):
    from paper_2012_15662_gb300 import binding as bd
    from oracle import ri
    w = _workload(name)
    s = w.system
    m = s.n_omega
    eng = bd.Engine(s, bd.DONOF_RI_TF32X3)
    eng.transform(w.C, bd.DONOF_RI_FULL)
    J_ctx, _ = eng.jk_mo()
    d_eng = eng.fetch(bd.DONOF_RI_FETCH_DIAG)          # [naux][n_omega]
    eng.close()
    for J in _noalloc_twice(d_eng, s.naux, m):
        assert np.isfinite(J).all()
        err = np.abs(J - J_ctx).max()
        assert err <= REL * np.abs(J_ctx).max(), (err, np.abs(J_ctx).max())
    # the oracle's diagonal in, the oracle's J = d^T d to compare with
    B, L, G = ri.setup(s)
    d_or = ri.diagonal(ri.half_transform(B, w.C, m), w.C)
    J_or = d_or.T @ d_or
    for J in _noalloc_twice(d_or, s.naux, m):
        err = np.abs(J - J_or).max()
        assert err <= REL * np.abs(J_or).max(), (err, np.abs(J_or).max())


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_2012_15662_gb300 import binding as bd
    dev = torch.device("cuda", 0)
    d = torch.zeros(16, dtype=torch.float64, device=dev)
    J = torch.zeros(16, dtype=torch.float64, device=dev)
    with pytest.raises(bd.DonofError) as ei:
        bd.donof_ri_jmo_noalloc(d, 60000, 4000, J)
    assert ei.value.status == bd.DONOF_RI_E_ARG
