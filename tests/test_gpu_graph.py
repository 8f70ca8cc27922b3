"""donof_ri_iteration: the CUDA-graph replay gives the same bits as the eager calls.

The graph is keyed by the device pointers, so a replay must read the current
contents of the inputs: the test overwrites C in place between replays.  The
iteration forks the gamma-only part of the energy row onto a side stream; its
results must equal, bit for bit, those of the four public calls made one after
the other on the context's stream.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec_name", ["fp64", "tf32x3", "slice4"])
def test_graph_matches_eager(prec_name):
    import torch
    from paper_2012_15662_gb300 import binding as bd
    from oracle import integrals as I
    from synthetic import orthonormal_orbitals, random_orthogonal
    from tests.workloads import make_workload
    prec = {"fp64": bd.DONOF_RI_FP64, "tf32x3": bd.DONOF_RI_TF32X3, "slice4": bd.DONOF_RI_SLICE4}[prec_name]
    w = make_workload("c6h12")
    s = w.system
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    eng = bd.Engine(s, prec, stream=stream.cuda_stream)
    nb, m = s.nbf, s.n_omega
    C2 = orthonormal_orbitals(I.overlap(w.system), random_orthogonal(nb, np.random.default_rng(77)))
    C_dev = torch.from_numpy(bd.Engine.colmajor(w.C)).to(dev)
    g_dev = torch.from_numpy(np.ascontiguousarray(w.gamma)).to(dev)
    out = {k: torch.zeros(sz, dtype=torch.float64, device=dev)
           for k, sz in dict(J=m * m, K=m * m, E=1, L=nb * nb).items()}
    torch.cuda.synchronize()

    def run(graph):
        with torch.cuda.stream(stream):
            bd.donof_ri_iteration(eng.ctx, C_dev, g_dev, bd.DONOF_RI_FULL, out["J"], out["K"], out["E"], out["L"],
                                  use_graph=graph)
        stream.synchronize()
        bd.donof_ri_sync(eng.ctx)
        return {k: v.cpu().numpy().copy() for k, v in out.items()}

    def serial():
        with torch.cuda.stream(stream):
            bd.donof_ri_transform(eng.ctx, C_dev, bd.DONOF_RI_FULL)
            bd.donof_ri_jk_mo(eng.ctx, out["J"], out["K"])
            bd.donof_ri_jk_ao_batch(eng.ctx)
            bd.donof_ri_energy_lagrangian(eng.ctx, g_dev, out["E"], out["L"])
        stream.synchronize()
        bd.donof_ri_sync(eng.ctx)
        return {k: v.cpu().numpy().copy() for k, v in out.items()}

    ref = serial()
    eager = run(False)
    for k in eager:
        np.testing.assert_array_equal(eager[k], ref[k])
    l0 = bd.donof_ri_launch_count(eng.ctx)
    g1 = run(True)
    g2 = run(True)
    assert bd.donof_ri_launch_count(eng.ctx) - l0 >= 2 * 10
    for k in eager:
        np.testing.assert_array_equal(eager[k], g1[k])
        np.testing.assert_array_equal(eager[k], g2[k])
    # new contents behind the same pointer: the replay must see them
    C_dev.copy_(torch.from_numpy(bd.Engine.colmajor(C2)).to(dev))
    torch.cuda.synchronize()
    g3 = run(True)
    e3 = run(False)
    for k in eager:
        np.testing.assert_array_equal(g3[k], e3[k])
    assert not np.array_equal(g3["J"], eager["J"])
    eng.close()


def test_gemm_kernel_profile_rows():
    """Per-row profiling records one event pair per tensor-core GEMM launch (rows 8..13)
    and per memory-bound pass (rows 14, 15), nested inside its row, and the profiled (serial) iteration gives the forked one's bits."""
    import torch
    from paper_2012_15662_gb300 import binding as bd
    from tests.workloads import make_workload
    w = make_workload("square4")
    s = w.system
    eng = bd.Engine(s, bd.DONOF_RI_SLICE4)
    dev = torch.device("cuda", 0)
    nb = s.nbf
    C_dev = torch.from_numpy(bd.Engine.colmajor(w.C)).to(dev)
    g_dev = torch.from_numpy(np.ascontiguousarray(w.gamma)).to(dev)
    outs = []
    for prof in (False, True):
        E = torch.zeros(1, dtype=torch.float64, device=dev)
        L = torch.zeros(nb * nb, dtype=torch.float64, device=dev)
        bd.donof_ri_profile(eng.ctx, prof)
        bd.donof_ri_iteration(eng.ctx, C_dev, g_dev, bd.DONOF_RI_FULL, None, None, E, L, use_graph=False)
        torch.cuda.synchronize()
        bd.donof_ri_sync(eng.ctx)
        outs.append((E.cpu().numpy(), L.cpu().numpy()))
    rows = [bd.donof_ri_profile_read(eng.ctx, r) for r in range(8)]
    gemms = [bd.donof_ri_profile_read(eng.ctx, 8 + k) for k in range(6)]
    mems = [bd.donof_ri_profile_read(eng.ctx, 14 + k) for k in range(2)]
    bd.donof_ri_profile(eng.ctx, False)
    eng.close()
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])
    assert all(c == 1 for _, c in gemms), gemms
    # each GEMM lies inside its row: half, full_k, j, jao, kao, energy
    for k, r in enumerate([0, 2, 3, 4, 5, 6]):
        assert 0.0 < gemms[k][0] <= rows[r][0] + 1e-3, (k, gemms[k], rows[r])
    # the digit pass inside the half-transform row, the J^(q)/K^(q) split inside "other"
    assert all(c == 1 for _, c in mems), mems
    for k, r in enumerate([0, 7]):
        assert 0.0 < mems[k][0] <= rows[r][0] + 1e-3, (k, mems[k], rows[r])


@pytest.mark.parametrize("prec_name", ["fp64", "slice4"])
def test_graph_with_pinned_host_buffers(prec_name):
    """Page-locked host inputs and outputs go through the captured graph (host copies
    inside it): same bits as device buffers, and a replay reads the host input's
    current contents."""
    import torch
    from paper_2012_15662_gb300 import binding as bd
    from oracle import integrals as I
    from synthetic import orthonormal_orbitals, random_orthogonal
    from tests.workloads import make_workload
    prec = {"fp64": bd.DONOF_RI_FP64, "slice4": bd.DONOF_RI_SLICE4}[prec_name]
    w = make_workload("square4")
    s = w.system
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    eng = bd.Engine(s, prec, stream=stream.cuda_stream)
    nb, m = s.nbf, s.n_omega
    sizes = dict(J=m * m, K=m * m, E=1, L=nb * nb)

    def run(C, g, out, graph):
        with torch.cuda.stream(stream):
            bd.donof_ri_iteration(eng.ctx, C, g, bd.DONOF_RI_FULL, out["J"], out["K"], out["E"], out["L"],
                                  use_graph=graph)
        stream.synchronize()
        bd.donof_ri_sync(eng.ctx)
        return {k: v.cpu().numpy().copy() for k, v in out.items()}

    C_dev = torch.from_numpy(bd.Engine.colmajor(w.C)).to(dev)
    g_dev = torch.from_numpy(np.ascontiguousarray(w.gamma)).to(dev)
    dev_out = {k: torch.zeros(n, dtype=torch.float64, device=dev) for k, n in sizes.items()}
    ref = run(C_dev, g_dev, dev_out, False)
    C_h = torch.from_numpy(bd.Engine.colmajor(w.C)).pin_memory()
    g_h = torch.from_numpy(np.ascontiguousarray(w.gamma)).pin_memory()
    host_out = {k: torch.zeros(n, dtype=torch.float64).pin_memory() for k, n in sizes.items()}
    l0 = bd.donof_ri_launch_count(eng.ctx)
    h1 = run(C_h, g_h, host_out, True)
    h2 = run(C_h, g_h, host_out, True)
    assert bd.donof_ri_launch_count(eng.ctx) - l0 >= 2 * 10
    for k in ref:
        np.testing.assert_array_equal(h1[k], ref[k])
        np.testing.assert_array_equal(h2[k], ref[k])
    C2 = orthonormal_orbitals(I.overlap(w.system), random_orthogonal(nb, np.random.default_rng(78)))
    C_h.copy_(torch.from_numpy(bd.Engine.colmajor(C2)))
    h3 = run(C_h, g_h, host_out, True)
    C_dev.copy_(torch.from_numpy(bd.Engine.colmajor(C2)).to(dev))
    torch.cuda.synchronize()
    ref3 = run(C_dev, g_dev, dev_out, False)
    for k in ref:
        np.testing.assert_array_equal(h3[k], ref3[k])
    assert not np.array_equal(h3["E"], ref["E"])
    eng.close()
