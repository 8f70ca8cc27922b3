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
    eng = bd.Engine(w.system, bd.DONOF_RI_TF32X3)
    eng.transform(w.C, bd.DONOF_RI_FULL)
    with pytest.raises(bd.DonofError) as e:
        bd.donof_ri_energy_lagrangian_contracted(eng.ctx, np.ascontiguousarray(w.gamma))
    assert e.value.status == bd.DONOF_RI_E_UNSUPPORTED
    eng.close()
    # the digit path needs the half transform only (it runs the full transform's GEMM itself)
    eng = bd.Engine(w.system, bd.DONOF_RI_SLICE4)
    with pytest.raises(bd.DonofError) as e:
        bd.donof_ri_energy_lagrangian_contracted(eng.ctx, np.ascontiguousarray(w.gamma))
    assert e.value.status == bd.DONOF_RI_E_STATE
    eng.transform(w.C, bd.DONOF_RI_HALF)
    E, lam = eng.energy_lagrangian_contracted(w.gamma)
    eng.close()
    assert np.isfinite(E) and np.isfinite(lam).all()


def _ragged(n_c, nbf, naux, n_weak):
    from synthetic import Workload, draw_gamma, make_system, orthonormal_orbitals, random_orthogonal, without_basis_functions
    full = make_system("ring", n_c=n_c, seed=n_c, jitter=0.02, n_weak_per=n_weak)
    s = without_basis_functions(full, full.nbf - nbf, full.naux - naux)
    rng = np.random.default_rng(nbf + naux)
    C = orthonormal_orbitals(I.overlap(s), random_orthogonal(s.nbf, rng))
    return Workload(name=f"c{n_c}-{nbf}-{naux}", system=s, C=C, gamma=draw_gamma(s.n_strong, s.n_weak_per, rng))


# square4 and C6H12: one K chunk over P; C10H20: two; nbf 229 with naux 811 (every
# tile edge ragged, a ragged third chunk); nbf 761 (the full transform's GEMM, which
# stores b^P_qp here, in two K chunks over the basis; one weak orbital per pair).
SLICE4_CASES = ["square4", "c6h12", "c10h20", (10, 229, 811, 4), (24, 761, 301, 1)]


@pytest.mark.parametrize("case", SLICE4_CASES, ids=lambda c: c if isinstance(c, str) else "ring-%d-%d-%d" % c[:3])
def test_slice4_contracted_against_oracle(case):
    """The digit path's contracted form (one digit-plane GEMM over K = (q, P) on the
    b_half digits and X^P_qp = [q = p] w_pP - B_pq b^P_qp) against the oracle's
    contracted Lagrangian and its energy, at the digit path's tolerances (E 1e-6 Eh,
    lambda 1e-6), and against the digit path's per-orbital form."""
    from paper_2012_15662_gb300 import binding as bd
    w = make_workload(case) if isinstance(case, str) else _ragged(*case)
    s = w.system
    m = s.n_omega
    eng = bd.Engine(s, bd.DONOF_RI_SLICE4)
    eng.transform(w.C, bd.DONOF_RI_HALF)
    Ec, lam_c = eng.energy_lagrangian_contracted(w.gamma)
    eng.jk_ao(want=False)
    E, lam = eng.energy_lagrangian(w.gamma)
    # the contracted call leaves the per-orbital state usable, and repeats bit for bit
    eng.transform(w.C, bd.DONOF_RI_FULL)
    Ec2, lam_c2 = eng.energy_lagrangian_contracted(w.gamma)
    eng.close()
    assert Ec2 == Ec
    np.testing.assert_array_equal(lam_c2, lam_c)
    B, L, G = ri.setup(s)
    bh = ri.half_transform(B, w.C, m)
    del B
    d = ri.diagonal(bh, w.C)
    bf = ri.full_transform(bh, w.C)
    J, K = ri.jk_mo(bf, d)
    H = I.core_hamiltonian(s)
    sub, rank = pairing_columns(s.n_strong, s.n_weak_per)
    n = pnof7.occupations(w.gamma, s.n_strong, s.n_weak_per, sub, rank)
    A, Bc = pnof7.coupling(n, sub, rank)
    lam_o = pnof7.lagrangian_contracted(w.C, H, bh, d, bf, n, A, Bc)
    Hd = np.einsum("mp,mn,np->p", w.C[:, :m], H, w.C[:, :m])
    E_o = pnof7.energy(n, Hd, J, K, A, Bc, I.nuclear_repulsion(s))
    err = dict(E=abs(Ec - E_o), lam=np.abs(lam_c - lam_o).max(), E_pf=abs(Ec - E), lam_pf=np.abs(lam_c - lam).max())
    print(case, err)
    assert err["E"] <= 1e-6 and err["lam"] <= 1e-6, err
    assert err["E_pf"] <= 1e-6 and err["lam_pf"] <= 1e-6, err
