"""GPU parity of the BF16 digit-plane path (DONOF_RI_SLICE4) at the target tolerance.

Target (stated per result): |dJ|, |dK| <= 1e-7 absolute and |dE| <= 1e-6 Eh
against the FP64 oracle.  The arithmetic behind it: each operand row carries
32 bits below its power-of-two scale, the digit-pair products are summed
exactly (integers below 2^24 in FP32, then int64), and only products 2^-40 or
more below the leading pair are dropped, so each GEMM result is good to about
2^-31 of its row scale (observed J, K ~2e-9, dE ~1e-8 Eh).
Sizes: square4, C6H12, C10H20 and C16H32 element by element; rings trimmed to
nbf 523 and 761 with naux 301 element by element (at 761 the contractions over
the orbital basis span two K chunks, the second one ragged; every tile edge is
ragged); C20H40 (nbf 720, naux 2520) on outputs the oracle
computes one by one (b_half rows of the first auxiliary functions, from a
partial forward substitution) and on properties that hold at any size.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import integrals as I, pnof7, ri  # noqa: E402
from synthetic import pairing_columns  # noqa: E402
from tests.workloads import make_workload  # noqa: E402

TOL_JK = 1e-7
TOL_E = 1e-6


def _oracle(w):
    s = w.system
    B, L, G = ri.setup(s)
    m = s.n_omega
    rows = ri.all_rows(B, w.C, m)
    H = I.core_hamiltonian(s)
    sub, rank = pairing_columns(s.n_strong, s.n_weak_per)
    n = pnof7.occupations(w.gamma, s.n_strong, s.n_weak_per, sub, rank)
    A, Bc = pnof7.coupling(n, sub, rank)
    Hd = np.einsum("mp,mn,np->p", w.C[:, :m], H, w.C[:, :m])
    E = pnof7.energy(n, Hd, rows["J"], rows["K"], A, Bc, I.nuclear_repulsion(s))
    lam = pnof7.lagrangian(w.C, H, rows["Jao"], rows["Kao"], n, A, Bc)
    return dict(E=E, lam=lam, **rows)


@pytest.fixture(scope="module", params=["square4", "c6h12", "c10h20", "c16h32"])
def case(request):
    from paper_2012_15662_gb300 import binding as bd
    w = make_workload(request.param)
    ref = _oracle(w)
    eng = bd.Engine(w.system, bd.DONOF_RI_SLICE4)
    yield w, ref, eng
    eng.close()


def test_jk_mo_and_transforms(case):
    from paper_2012_15662_gb300 import binding as bd
    w, ref, eng = case
    eng.transform(w.C, bd.DONOF_RI_FULL)
    J, K = eng.jk_mo()
    assert np.abs(J - ref["J"]).max() <= TOL_JK
    assert np.abs(K - ref["K"]).max() <= TOL_JK
    bh = eng.fetch(bd.DONOF_RI_FETCH_BHALF)
    assert np.abs(bh - ref["bh"]).max() <= 1e-8 * max(1.0, np.abs(ref["bh"]).max())
    d = eng.fetch(bd.DONOF_RI_FETCH_DIAG)
    assert np.abs(d - ref["d"]).max() <= 1e-8 * max(1.0, np.abs(ref["d"]).max())


def test_jk_ao_energy_lambda(case):
    from paper_2012_15662_gb300 import binding as bd
    w, ref, eng = case
    eng.transform(w.C, bd.DONOF_RI_HALF)
    Jao, Kao = eng.jk_ao()
    assert np.abs(Jao - ref["Jao"]).max() <= TOL_JK
    assert np.abs(Kao - ref["Kao"]).max() <= TOL_JK
    E, lam = eng.energy_lagrangian(w.gamma)
    assert abs(E - ref["E"]) <= TOL_E, (E, ref["E"])
    assert np.abs(lam - ref["lam"]).max() <= 1e-6


def test_bitwise_reproducible(case):
    from paper_2012_15662_gb300 import binding as bd
    w, ref, eng = case
    out = []
    for _ in range(2):
        eng.transform(w.C, bd.DONOF_RI_FULL)
        J, K = eng.jk_mo()
        eng.jk_ao(want=False)
        out.append((J, K) + eng.energy_lagrangian(w.gamma))
    for a, b in zip(out[0], out[1]):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("n_c,nbf,naux,n_weak", [(20, 523, 301, 4), (24, 761, 301, 1)])
def test_large_basis_odd_sizes(n_c, nbf, naux, n_weak):
    """Odd sizes with a large orbital basis: nbf 523 (the contractions over the basis
    in one K chunk, every tile edge ragged) and nbf 761 (the half and full transforms
    and F^(p) C_p in two K chunks, the second of 25 elements; one weak orbital per
    pair, N_Omega 192), naux 301."""
    from paper_2012_15662_gb300 import binding as bd
    from synthetic import Workload, draw_gamma, make_system, orthonormal_orbitals, random_orthogonal, without_basis_functions
    full = make_system("ring", n_c=n_c, seed=n_c, jitter=0.02, n_weak_per=n_weak)
    s = without_basis_functions(full, full.nbf - nbf, full.naux - naux)
    assert (s.nbf, s.naux) == (nbf, naux)
    rng = np.random.default_rng(nbf)
    C = orthonormal_orbitals(I.overlap(s), random_orthogonal(s.nbf, rng))
    w = Workload(name=f"c{n_c}-{nbf}", system=s, C=C, gamma=draw_gamma(s.n_strong, s.n_weak_per, rng))
    ref = _oracle(w)
    eng = bd.Engine(s, bd.DONOF_RI_SLICE4)
    eng.transform(w.C, bd.DONOF_RI_FULL)
    J, K = eng.jk_mo()
    bh = eng.fetch(bd.DONOF_RI_FETCH_BHALF)
    d = eng.fetch(bd.DONOF_RI_FETCH_DIAG)
    Jao, Kao = eng.jk_ao()
    E, lam = eng.energy_lagrangian(w.gamma)
    eng.close()
    assert np.abs(bh - ref["bh"]).max() <= 1e-8 * max(1.0, np.abs(ref["bh"]).max())
    assert np.abs(d - ref["d"]).max() <= 1e-8 * max(1.0, np.abs(ref["d"]).max())
    assert np.abs(J - ref["J"]).max() <= TOL_JK
    assert np.abs(K - ref["K"]).max() <= TOL_JK
    assert np.abs(Jao - ref["Jao"]).max() <= TOL_JK
    assert np.abs(Kao - ref["Kao"]).max() <= TOL_JK
    assert abs(E - ref["E"]) <= TOL_E, (E, ref["E"])
    assert np.abs(lam - ref["lam"]).max() <= 1e-6


def test_full_size_c20h40():
    """nbf 720, naux 2520, N_Omega 400: sampled b_half rows and size-independent properties."""
    from scipy.linalg import solve_triangular
    from paper_2012_15662_gb300 import binding as bd
    w = make_workload("c20h40")
    s = w.system
    eng = bd.Engine(s, bd.DONOF_RI_SLICE4)
    eng.transform(w.C, bd.DONOF_RI_FULL)
    J, K = eng.jk_mo()
    bh = eng.fetch(bd.DONOF_RI_FETCH_BHALF)
    d = eng.fetch(bd.DONOF_RI_FETCH_DIAG)
    Jao, Kao = eng.jk_ao()
    E, lam = eng.energy_lagrangian(w.gamma)
    eng.close()
    # oracle, one output at a time: B^P for the first auxiliary functions needs only the
    # leading block of the metric's Cholesky factor and the matching (P|mu nu)
    npick = 6
    G = I.metric(s)
    L = np.linalg.cholesky(G[:npick, :npick])
    e3 = I.eri3(s, slice(0, npick))
    Bp = solve_triangular(L, e3.reshape(npick, -1), lower=True).reshape(npick, s.nbf, s.nbf)
    m = s.n_omega
    bh_ref = np.einsum("pm,Pmn->Ppn", w.C[:, :m].T, Bp)
    assert np.abs(bh[:npick] - bh_ref).max() <= 1e-8 * max(1.0, np.abs(bh_ref).max())
    d_ref = np.einsum("Ppn,np->Pp", bh_ref, w.C[:, :m])
    assert np.abs(d[:npick] - d_ref).max() <= 1e-8 * max(1.0, np.abs(d_ref).max())
    # properties at any size
    assert np.abs(J - J.T).max() <= TOL_JK
    assert np.abs(K - K.T).max() <= TOL_JK
    assert np.abs(np.diag(J) - np.diag(K)).max() <= TOL_JK
    assert K.min() >= -TOL_JK
    np.testing.assert_allclose(J, d.T @ d, atol=TOL_JK)
    C = w.C[:, :m]
    for q in (0, 57, 399):
        assert abs(C[:, q] @ Jao[q] @ C[:, q] - J[q, q]) <= TOL_JK
        assert abs(C[:, q] @ Kao[q] @ C[:, q] - K[q, q]) <= TOL_JK
    H = I.core_hamiltonian(s)
    sub, rank = pairing_columns(s.n_strong, s.n_weak_per)
    n = pnof7.occupations(w.gamma, s.n_strong, s.n_weak_per, sub, rank)
    A, Bc = pnof7.coupling(n, sub, rank)
    Hd = np.einsum("mp,mn,np->p", C, H, C)
    # energy from this path's own J, K (Eq. PNOF) equals the energy from lambda
    E2 = pnof7.energy(n, Hd, J, K, A, Bc, I.nuclear_repulsion(s))
    assert abs(E - E2) <= TOL_E


def test_full_size_c20h40_against_oracle():
    """C20H40, the benchmark's workload: J, K, E and lambda against the FP64 oracle (a
    few minutes of host time: the three-centre integrals and the fit at full size)."""
    from paper_2012_15662_gb300 import binding as bd
    w = make_workload("c20h40")
    s = w.system
    eng = bd.Engine(s, bd.DONOF_RI_SLICE4)
    eng.transform(w.C, bd.DONOF_RI_FULL)
    J, K = eng.jk_mo()
    eng.jk_ao(want=False)
    E, lam = eng.energy_lagrangian(w.gamma)
    eng.close()
    B, L, G = ri.setup(s)
    m = s.n_omega
    bh = ri.half_transform(B, w.C, m)
    del B, L, G
    d = ri.diagonal(bh, w.C)
    bf = ri.full_transform(bh, w.C)
    Jo, Ko = ri.jk_mo(bf, d)
    assert np.abs(J - Jo).max() <= TOL_JK
    assert np.abs(K - Ko).max() <= TOL_JK
    H = I.core_hamiltonian(s)
    sub, rank = pairing_columns(s.n_strong, s.n_weak_per)
    n = pnof7.occupations(w.gamma, s.n_strong, s.n_weak_per, sub, rank)
    A, Bc = pnof7.coupling(n, sub, rank)
    lamo = pnof7.lagrangian_contracted(w.C, H, bh, d, bf, n, A, Bc)
    Hd = np.einsum("mp,mn,np->p", w.C[:, :m], H, w.C[:, :m])
    Eo = pnof7.energy(n, Hd, Jo, Ko, A, Bc, I.nuclear_repulsion(s))
    assert abs(E - Eo) <= TOL_E, (E, Eo)
    assert np.abs(lam - lamo).max() <= 1e-6


def test_ghost_centre_auxiliary_set():
    """C6H12 with the ghost-centre auxiliary set (N_aux 1140, Coulomb metric condition
    number ~9e11 against ~1e7 for the on-atom sets): SLICE4 and the FP64 form against
    the oracle at the same tolerances."""
    from paper_2012_15662_gb300 import binding as bd
    w = make_workload("c6h12fit")
    ref = _oracle(w)
    for prec in (bd.DONOF_RI_SLICE4, bd.DONOF_RI_FP64):
        eng = bd.Engine(w.system, prec)
        eng.transform(w.C, bd.DONOF_RI_FULL)
        J, K = eng.jk_mo()
        Jao, Kao = eng.jk_ao()
        E, lam = eng.energy_lagrangian(w.gamma)
        eng.close()
        err = dict(J=np.abs(J - ref["J"]).max(), K=np.abs(K - ref["K"]).max(),
                   Jao=np.abs(Jao - ref["Jao"]).max(), Kao=np.abs(Kao - ref["Kao"]).max(),
                   E=abs(E - ref["E"]), lam=np.abs(lam - ref["lam"]).max())
        print(prec, err)
        assert max(err["J"], err["K"], err["Jao"], err["Kao"]) <= TOL_JK, (prec, err)
        assert err["E"] <= TOL_E and err["lam"] <= 1e-6, (prec, err)
