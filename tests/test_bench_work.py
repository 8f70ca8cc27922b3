"""bench.py's algorithmic work per launch against the per-configuration operation
counts derived from the paper's Tables 2 and 3 (2 flops per multiply-add, the
symmetric halves of J^(p), K^(p) not counted), written out beforehand for the five
workloads: a1 2N_b^2N_xN_Omega, a3 2N_bN_xN_Omega^2, a5 / a6 N_b(N_b + 1)N_xN_Omega,
a7's GEMM 4N_b^2N_Omega^2.  The roofline fractions divide these by measured time,
so a slip here would mis-state every fraction.
"""
import pytest

import bench
from tests.workloads import make_workload

# (workload, a1, a3, a5 or a6, a7 GEMM), three significant digits
TABLE = [
    ("square4", 1.1e6, 5.5e5, 5.8e5, 3.3e5),
    ("c6h12", 2.51e9, 2.09e9, 1.26e9, 1.19e9),
    ("c10h20", 1.94e10, 1.61e10, 9.7e9, 9.2e9),
    ("c16h32", 2.48e11, 1.65e11, 1.24e11, 9.4e10),
    ("c20h40", 1.05e12, 5.81e11, 5.23e11, 3.3e11),
]


@pytest.mark.parametrize("name,a1,a3,a56,a7", TABLE)
def test_algorithmic_flops_match_the_operation_counts(name, a1, a3, a56, a7):
    s = make_workload(name).system
    f = bench.algorithmic_flops(s)
    assert f["half"] == pytest.approx(a1, rel=0.02)
    # a3 adds the K_pq square-sum, 2 N_x N_Omega^2, to the transform's count
    assert f["full_k"] - 2.0 * s.naux * s.n_omega ** 2 == pytest.approx(a3, rel=0.02)
    assert f["jao"] == pytest.approx(a56, rel=0.02)
    assert f["kao"] == pytest.approx(a56, rel=0.02)
    assert f["fock"] == pytest.approx(a7, rel=0.02)
