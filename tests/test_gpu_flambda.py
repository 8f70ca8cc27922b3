"""The F^lambda orbital step on the device (donof_ri_flambda_step) against the
oracle's (oracle.orbopt.flambda_step, numpy eigh in FP64).

With a distinct, ascending diagonal the eigenvectors are unique up to sign: the
device's rotated orbitals match the oracle's column by column (to the FP32
precision of the device eigensolver), stay orthonormal to FP64 rounding, and give
the oracle's energy after the step.  With the first-step diagonal (lambda_pp) the
eigenvalues match.  The F^lambda driver lowers the energy monotonically.
square4 and C6H12 (nbf 24, 144) run the one-CTA Jacobi; C10H20 (nbf 240) the
block Jacobi, against the same oracle; C16H32 (nbf 480) checks the block path on
properties that hold at any size.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

from oracle import integrals as I, orbopt, ri  # noqa: E402
from synthetic import pairing_columns  # noqa: E402
from tests.workloads import make_workload  # noqa: E402


@pytest.mark.parametrize("name", ["square4", "c6h12", "c10h20"])
def test_flambda_step_matches_oracle(name):
    from paper_2012_15662_gb300 import binding as bd
    w = make_workload(name)
    s = w.system
    nb = s.nbf
    B, L, G = ri.setup(s)
    H = I.core_hamiltonian(s)
    enuc = I.nuclear_repulsion(s)
    sub, rank = pairing_columns(s.n_strong, s.n_weak_per)
    E0, lam = orbopt.energy_lambda(s, B, H, enuc, w.C, w.gamma, sub, rank)
    gmax_o = np.abs(lam - lam.T).max()
    # not a power of ten times an element (the largest one, gmax, would then sit on the
    # boundary of two scaling decades, where either choice is correct)
    bound = 1.234e-3 * gmax_o
    D = np.linspace(-2.0, 2.0, nb)
    C_o, eps_o = orbopt.flambda_step(w.C, lam, D, bound)
    eng = bd.Engine(s, bd.DONOF_RI_FP64)
    eng.transform(w.C, bd.DONOF_RI_HALF)
    eng.jk_ao(want=False)
    eng.energy_lagrangian(w.gamma)
    diag = D.copy()
    Ccm = np.empty(nb * nb)
    gmax, sweeps = bd.donof_ri_flambda_step(eng.ctx, diag, False, bound, Ccm)
    C_g = Ccm.reshape(nb, nb).T
    assert abs(gmax - gmax_o) <= 1e-10 * gmax_o
    assert 1 <= sweeps < 30
    np.testing.assert_allclose(C_g.T @ I.overlap(s) @ C_g, np.eye(nb), atol=1e-13)
    np.testing.assert_allclose(diag, eps_o, atol=1e-9 * np.abs(eps_o).max())
    # eigenvectors column by column where the eigenvalue is separated (FP32 Jacobi,
    # then two FP64 first-order refinements)
    overlap = np.abs(C_g.T @ I.overlap(s) @ C_o)
    gaps = np.minimum(np.r_[np.inf, np.diff(eps_o)], np.r_[np.diff(eps_o), np.inf])
    sep = gaps > 1e-3 * np.abs(eps_o).max()
    assert sep.sum() >= nb // 2
    np.testing.assert_allclose(np.diag(overlap)[sep], 1.0, atol=1e-10)
    E_g, _ = orbopt.energy_lambda(s, B, H, enuc, C_g, w.gamma, sub, rank)
    E_o, _ = orbopt.energy_lambda(s, B, H, enuc, C_o, w.gamma, sub, rank)
    assert abs(E_g - E_o) <= 1e-9 * max(1.0, abs(E_o))
    # the first step: diagonal lambda_pp
    eng.transform(w.C, bd.DONOF_RI_HALF)
    eng.jk_ao(want=False)
    eng.energy_lagrangian(w.gamma)
    diag1 = np.empty(nb)
    bd.donof_ri_flambda_step(eng.ctx, diag1, True, bound)
    eng.close()
    ev = np.linalg.eigvalsh(orbopt.flambda_matrix(lam, np.diag(lam), bound))
    # lambda_pp = 0 for every orbital outside the pairing space: their eigenvalues
    # nearly coincide, and a pair the FP64 refinement cannot resolve keeps the FP32
    # solver's accuracy
    np.testing.assert_allclose(diag1, ev, atol=1e-6 * np.abs(ev).max())


def test_flambda_driver_descends():
    from paper_2012_15662_gb300 import binding as bd
    from paper_2012_15662_gb300 import solve
    w = make_workload("square4")
    eng = bd.Engine(w.system, bd.DONOF_RI_FP64)
    r = solve.flambda_iterations(eng, bd.Engine.colmajor(w.C), w.gamma, max_iter=40)
    eng.close()
    Es = r["energies"]
    assert all(b <= a for a, b in zip(Es, Es[1:]))
    assert Es[-1] < Es[0]


def test_flambda_call_order():
    from paper_2012_15662_gb300 import binding as bd
    w = make_workload("square4")
    eng = bd.Engine(w.system, bd.DONOF_RI_FP64)
    eng.transform(w.C, bd.DONOF_RI_HALF)
    with pytest.raises(bd.DonofError) as e:
        bd.donof_ri_flambda_step(eng.ctx, np.zeros(w.system.nbf), True, 0.1)
    assert e.value.status == bd.DONOF_RI_E_STATE
    eng.close()


def test_flambda_block_path_properties():
    """nbf 480 (block Jacobi): the step's rotation U = C0^T S C1 is orthogonal and
    diagonalises F^lambda (built here from the engine's own lambda by the stated
    rule), with the returned eigenvalues on the diagonal in increasing order (to the
    FP32 solver's accuracy)."""
    from paper_2012_15662_gb300 import binding as bd
    w = make_workload("c16h32")
    s = w.system
    nb = s.nbf
    eng = bd.Engine(s, bd.DONOF_RI_SLICE4)
    eng.transform(w.C, bd.DONOF_RI_HALF)
    eng.jk_ao(want=False)
    _, lam = eng.energy_lagrangian(w.gamma)
    g = np.abs(lam - lam.T).max()
    bound = 1.234e-2 * g
    diag = np.empty(nb)
    Ccm = np.empty(nb * nb)
    gmax, sweeps = bd.donof_ri_flambda_step(eng.ctx, diag, True, bound, Ccm)
    eng.close()
    assert gmax == pytest.approx(g, rel=1e-12)
    assert 1 <= sweeps < 30
    # ordered by the FP32 solve; the returned values are the FP64-refined ones
    assert np.diff(diag).min() >= -2e-6 * np.abs(diag).max()
    C1 = Ccm.reshape(nb, nb).T
    S = I.overlap(s)
    np.testing.assert_allclose(C1.T @ S @ C1, np.eye(nb), atol=1e-12)
    # F^lambda: F_qp = lambda_qp - lambda_pq below the diagonal, mirrored, each element
    # above the bound multiplied by 1/10 until it is not
    F = np.tril(lam - lam.T, -1)
    a = np.abs(F)
    for _ in range(700):
        big = a > bound
        if not big.any():
            break
        F[big] *= 0.1
        a[big] *= 0.1
    F = F + F.T + np.diag(np.diag(lam))
    U = w.C.T @ S @ C1
    A = U.T @ F @ U
    off = A - np.diag(np.diag(A))
    scale = np.abs(F).max()
    # pairs of separated eigenvalues are refined to FP64; a nearly degenerate pair the
    # first-order refinement cannot resolve keeps the FP32 solver's accuracy
    sep = np.abs(diag[:, None] - diag[None, :]) > 1e-3 * scale
    np.fill_diagonal(sep, False)
    assert sep.sum() >= nb * (nb - 1) // 2
    assert np.abs(off[sep]).max() <= 1e-9 * scale
    assert np.abs(off).max() <= 2e-6 * scale
    np.testing.assert_allclose(np.diag(A), diag, atol=1e-8 * scale)
