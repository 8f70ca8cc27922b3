"""donof_ri_iteration: the CUDA-graph replay gives the same bits as the eager calls.

The graph is keyed by the device pointers, so a replay must read the current
contents of the inputs: the test overwrites C in place between replays.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec_name", ["fp64", "tf32x3"])
def test_graph_matches_eager(prec_name):
    import torch
    from paper_2012_15662_gb300 import binding as bd
    from synthetic import make_workload, random_orthogonal
    prec = bd.DONOF_RI_FP64 if prec_name == "fp64" else bd.DONOF_RI_TF32X3
    w = make_workload("c6h12")
    s = w.system
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    eng = bd.Engine(s, prec, stream=stream.cuda_stream)
    nb, m = s.nbf, s.n_omega
    C2 = random_orthogonal(nb, np.random.default_rng(77))
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

    eager = run(False)
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
